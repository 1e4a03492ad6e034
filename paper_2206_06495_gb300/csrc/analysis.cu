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

}  // namespace

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
