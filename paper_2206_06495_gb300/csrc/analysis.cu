// Accuracy analysis of the stencil operators on the GPU (Section 4 of the
// paper): the modified wavenumber of Eq. 2d_mw and the relative error of
// Eq. relative_error on the test function of Eq. test, for every alpha-node
// of an ELL operator.  One thread per row; every sum runs over the row's
// stencil slots in slot order, so results do not depend on the launch.
#include <cmath>

#include "common.cuh"

namespace rbffd {
namespace {

constexpr int kAThreads = 256;

// Modified wavenumbers at alpha-node i for the plane wave exp(i k.x):
//   k1 = -i [(kx D_x + ky D_y) / kt] exp(i k.x) exp(-i k.x_i) / kt   (k*/k~)
//   k2 = -[D_Lap exp(i k.x)] exp(-i k.x_i) / kt^2                     (k*^2/k~^2)
// with the phase of stencil node j taken relative to the alpha-node,
// k.(x_j - x_i), so that large coordinates lose no digits.
__global__ void __launch_bounds__(kAThreads)
    k_modified_wavenumber(int64_t n, int64_t ld, int k, const int32_t* __restrict__ ix,
                          const double* __restrict__ wx, const int32_t* __restrict__ iy,
                          const double* __restrict__ wy, int64_t ld2, int k2n,
                          const int32_t* __restrict__ il, const double* __restrict__ wl,
                          const double* __restrict__ ax, const double* __restrict__ ay,
                          const double* __restrict__ bx, const double* __restrict__ by,
                          double kx, double ky, double2* __restrict__ k1,
                          double2* __restrict__ k2) {
  const double kt = sqrt(kx * kx + ky * ky), ikt2 = 1.0 / (kt * kt);
  for (int64_t i = blockIdx.x * (int64_t)kAThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kAThreads) {
    const double x0 = ax[i], y0 = ay[i];
    double re = 0.0, im = 0.0;
    for (int s = 0; s < k; ++s) {
      const int32_t jx = ix[s * ld + i], jy = iy[s * ld + i];
      double sx, cx, sy, cy;
      sincos(kx * (bx[jx] - x0) + ky * (by[jx] - y0), &sx, &cx);
      const double ax_ = kx * wx[s * ld + i];
      re += ax_ * cx;
      im += ax_ * sx;
      if (jy != jx) sincos(kx * (bx[jy] - x0) + ky * (by[jy] - y0), &sy, &cy);
      else { sy = sx; cy = cx; }
      const double ay_ = ky * wy[s * ld + i];
      re += ay_ * cy;
      im += ay_ * sy;
    }
    // -i (re + i im) = im - i re
    k1[i] = make_double2(im * ikt2, -re * ikt2);
    if (k2) {
      double lr = 0.0, li = 0.0;
      for (int s = 0; s < k2n; ++s) {
        const int32_t j = il[s * ld2 + i];
        double sn, cs;
        sincos(kx * (bx[j] - x0) + ky * (by[j] - y0), &sn, &cs);
        lr += wl[s * ld2 + i] * cs;
        li += wl[s * ld2 + i] * sn;
      }
      k2[i] = make_double2(-lr * ikt2, -li * ikt2);
    }
  }
}

// Relative error of one operator row on the node-scaled test function
// g_i(x, y) = cos(x / dr_i) cos(y / dr_i): |sum_s w_s g_i(x_j) - L g_i(x_i)|
// divided by max |L g_i| (1 for interpolation, 1/dr for first derivatives,
// 2/dr^2 for the Laplacian).  dr_i from dr, or, when dr is null, the mean
// distance from the alpha-node to stencil slots 1..6 (a collocated operator,
// whose slot 0 is the node itself).  The mean over rows is reduced
// deterministically into *mean.
__global__ void __launch_bounds__(kAThreads)
    k_stencil_error(int64_t n, int64_t ld, int k, const int32_t* __restrict__ idx,
                    const double* __restrict__ w, int op, const double* __restrict__ ax,
                    const double* __restrict__ ay, const double* __restrict__ bx,
                    const double* __restrict__ by, const double* __restrict__ dr,
                    double* __restrict__ err, GridReduce gr, double* __restrict__ mean) {
  __shared__ double sh[kAThreads];
  double part[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kAThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kAThreads) {
    const double x0 = ax[i], y0 = ay[i];
    double d;
    if (dr) {
      d = dr[i];
    } else {
      d = 0.0;
      for (int s = 1; s <= 6; ++s) {
        const int32_t j = idx[s * ld + i];
        const double ex = bx[j] - x0, ey = by[j] - y0;
        d += sqrt(ex * ex + ey * ey);
      }
      d /= 6.0;
    }
    const double id = 1.0 / d;
    double acc = 0.0;
    for (int s = 0; s < k; ++s) {
      const int32_t j = idx[s * ld + i];
      acc += w[s * ld + i] * (cos(bx[j] * id) * cos(by[j] * id));
    }
    double sx0, cx0, sy0, cy0;
    sincos(x0 * id, &sx0, &cx0);
    sincos(y0 * id, &sy0, &cy0);
    double exact, scale;
    if (op == 1) {
      exact = -sx0 * cy0 * id;
      scale = id;
    } else if (op == 2) {
      exact = -cx0 * sy0 * id;
      scale = id;
    } else if (op == 3) {
      exact = -2.0 * cx0 * cy0 * id * id;
      scale = 2.0 * id * id;
    } else {
      exact = cx0 * cy0;
      scale = 1.0;
    }
    const double e = fabs(acc - exact) / scale;
    err[i] = e;
    part[0] += e;
  }
  grid_reduce<1>(part, gr, sh, [&](double* t) { *mean = t[0] / (double)n; });
}

// Force of the fluid on a circular body (Section 5.2): the traction
// (-p I + (grad U + grad U^T) / Re) n at each of the n_c surface P-nodes
// (rows, in increasing angle; n from the centre through the node, i.e. from
// the body into the fluid), the velocity gradient from the D^(P,V) rows,
// integrated in angle by composite Simpson's rule (weights 2, 4, 2, 4, ... of
// h/3 on the periodic grid) times the radius.  One block; the sums run in a
// fixed order.  out[0], out[1]: C_D, C_L = F / (1/2 D) (rho = U = 1).
constexpr int kFThreads = 256;
__global__ void __launch_bounds__(kFThreads)
    k_cylinder_forces(int n_c, const int32_t* __restrict__ rows, int64_t ld, int k,
                      const int32_t* __restrict__ idx, const double* __restrict__ wdx,
                      const double* __restrict__ wdy, const double* __restrict__ u,
                      const double* __restrict__ v, const double* __restrict__ p,
                      const double* __restrict__ px, const double* __restrict__ py, double cx,
                      double cy, double radius, double inv_re, double* __restrict__ out) {
  __shared__ double sx[kFThreads], sy[kFThreads];
  double fx = 0.0, fy = 0.0;
  for (int q = threadIdx.x; q < n_c; q += kFThreads) {
    const int64_t i = rows[q];
    double ux = 0.0, uy = 0.0, vx = 0.0, vy = 0.0;
    for (int s = 0; s < k; ++s) {
      const int32_t j = idx[s * ld + i];
      const double ax = wdx[s * ld + i], ay = wdy[s * ld + i];
      ux += ax * u[j];
      uy += ay * u[j];
      vx += ax * v[j];
      vy += ay * v[j];
    }
    const double ex = px[i] - cx, ey = py[i] - cy, r = sqrt(ex * ex + ey * ey);
    const double nx = ex / r, ny = ey / r;
    const double tx = -p[i] * nx + (2.0 * ux * nx + (uy + vx) * ny) * inv_re;
    const double ty = -p[i] * ny + ((uy + vx) * nx + 2.0 * vy * ny) * inv_re;
    const double w = (q % 2) ? 4.0 : 2.0;
    fx += w * tx;
    fy += w * ty;
  }
  sx[threadIdx.x] = fx;
  sy[threadIdx.x] = fy;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ax = 0.0, ay = 0.0;
    for (int t = 0; t < kFThreads; ++t) {
      ax += sx[t];
      ay += sy[t];
    }
    const double h = 2.0 * 3.14159265358979323846 / (double)n_c;
    const double scale = h / 3.0 * radius * 2.0 / (2.0 * radius);  // Simpson, ds, 1/(D/2)
    out[0] = ax * scale;
    out[1] = ay * scale;
  }
}

}  // namespace

int analysis_forces(rbffd_ctx* ctx, const rbffd_flow& f, const double* u, const double* v,
                    const double* p, const int32_t* rows, int32_t n_c, double cx, double cy,
                    double radius, double Re, double* out_host, cudaStream_t st) {
  void* base = nullptr;
  int rc = ctx_scratch(ctx, 2 * sizeof(double), &base);
  if (rc) return rc;
  k_cylinder_forces<<<1, kFThreads, 0, st>>>(n_c, rows, f.ld_p, ctx->prm.n, f.pv_idx, f.pv_dx,
                                             f.pv_dy, u, v, p, f.p_x, f.p_y, cx, cy, radius,
                                             1.0 / Re, (double*)base);
  rc = check_cuda(ctx, cudaGetLastError(), "forces kernel");
  if (rc) return rc;
  rc = check_cuda(ctx, cudaMemcpyAsync(out_host, base, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                       st), "forces copy");
  if (rc) return rc;
  return check_cuda(ctx, cudaStreamSynchronize(st), "forces sync");
}

int analysis_mw(rbffd_ctx* ctx, const rbffd_ell* Dx, const rbffd_ell* Dy, const rbffd_ell* Dl,
                const double* ax, const double* ay, const double* bx, const double* by,
                double kx, double ky, double* k1, double* k2, cudaStream_t st) {
  const int64_t n = Dx->n_rows;
  if (n == 0) return RBFFD_OK;
  const int blocks = (int)std::min<int64_t>((n + kAThreads - 1) / kAThreads,
                                            (int64_t)sm_count() * 8);
  k_modified_wavenumber<<<blocks, kAThreads, 0, st>>>(
      n, Dx->ld, Dx->n, Dx->idx, (const double*)Dx->w, Dy->idx, (const double*)Dy->w,
      Dl ? Dl->ld : 0, Dl ? Dl->n : 0, Dl ? Dl->idx : nullptr,
      Dl ? (const double*)Dl->w : nullptr, ax, ay, bx, by, kx, ky, (double2*)k1,
      Dl ? (double2*)k2 : nullptr);
  return check_cuda(ctx, cudaGetLastError(), "modified wavenumber kernel");
}

int analysis_error(rbffd_ctx* ctx, const rbffd_ell* D, int op, const double* ax,
                   const double* ay, const double* bx, const double* by, const double* dr,
                   double* err, double* mean, cudaStream_t st) {
  const int64_t n = D->n_rows;
  if (n == 0) return RBFFD_OK;
  const int blocks = (int)std::min<int64_t>((n + kAThreads - 1) / kAThreads,
                                            (int64_t)sm_count() * 8);
  void* base = nullptr;
  const size_t need = sizeof(double) * (size_t)blocks + 256;
  int rc = ctx_scratch(ctx, need, &base);
  if (rc) return rc;
  GridReduce gr;
  gr.counter = (unsigned int*)base;
  gr.partials = (double*)((char*)base + 256);
  if (!mean) mean = (double*)((char*)base + 128);  // the caller does not want the mean
  rc = check_cuda(ctx, cudaMemsetAsync(gr.counter, 0, sizeof(unsigned int), st), "memset");
  if (rc) return rc;
  k_stencil_error<<<blocks, kAThreads, 0, st>>>(n, D->ld, D->n, D->idx, (const double*)D->w, op,
                                                ax, ay, bx, by, dr, err, gr, mean);
  return check_cuda(ctx, cudaGetLastError(), "stencil error kernel");
}

}  // namespace rbffd
