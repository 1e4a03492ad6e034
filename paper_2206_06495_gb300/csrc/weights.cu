// Batched PHS+poly stencil weights (Section 2.1, Eq. rbf_poly_compact).
//
// One warp owns one stencil.  The augmented system [A P; P^T 0] (size
// S = n + (q+1)(q+2)/2) and its right-hand sides (one column per requested
// operator) live column-major in the warp's slice of shared memory, with an
// odd leading dimension so that a warp touching one column hits 32 banks.
// The warp factors the system by Gaussian elimination with partial pivoting
// (pivot: largest magnitude, lowest row on ties) applied to the right-hand
// sides in the same sweep, then back-substitutes.  Every elimination update is
// spread over the 32 lanes as a flat list of (row, column) pairs, so lanes stay
// busy down to the last columns.  All arithmetic is FP64.
//
// Local coordinates (the "shift and scale" of the implementation the paper
// follows): stencil nodes are shifted to the alpha-node and divided by the
// largest centre-to-node distance s; derivative weights are divided by s (first
// derivatives) or s^2 (Laplacian) afterwards.
#include <cmath>

#include "common.cuh"

namespace rbffd {
namespace {

constexpr int kMaxWarpsPerBlock = 4;
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// r^m for odd m from r^2: r^(m-1) * r
__device__ __forceinline__ double phs_from_r2(double r2, int m) {
  return ipow(r2, (m - 1) / 2) * sqrt(r2);
}

// (a, b) of the t-th monomial in graded lexicographic order 1, x, y, x^2, xy, y^2, ...
__device__ __forceinline__ void monomial(int t, int& a, int& b) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= t) ++d;
  int r = t - d * (d + 1) / 2;
  b = r;
  a = d - r;
}

// Right-hand side of operator `op` (bit index 0..3 = INTERP, DX, DY, LAP) in row `row`.
__device__ __forceinline__ double rhs_value(int op, int row, int n, int m, double X, double Y) {
  if (row < n) {
    const double r2 = X * X + Y * Y;
    switch (op) {
      case 0:  // phi(|0 - x_j|)
        return phs_from_r2(r2, m);
      case 1:  // d/dx |x - x_j|^m at x = 0: -m r^(m-2) x_j
        return -m * phs_from_r2(r2, m - 2) * X;
      case 2:
        return -m * phs_from_r2(r2, m - 2) * Y;
      default:  // 2-D Laplacian of r^m: m^2 r^(m-2)
        return (double)(m * m) * phs_from_r2(r2, m - 2);
    }
  }
  int a, b;
  monomial(row - n, a, b);
  switch (op) {
    case 0:
      return (a == 0 && b == 0) ? 1.0 : 0.0;
    case 1:
      return (a == 1 && b == 0) ? 1.0 : 0.0;
    case 2:
      return (a == 0 && b == 1) ? 1.0 : 0.0;
    default:
      return ((a == 2 && b == 0) || (a == 0 && b == 2)) ? 2.0 : 0.0;
  }
}

// Magnitude of a double as an ordered integer key: for non-negative values
// the IEEE bit pattern orders like the value, so the pivot search compares
// integers instead of spending FP64 instructions (NaN, with the largest
// patterns, wins and is then caught as a singular pivot).
__device__ __forceinline__ unsigned long long mag_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// One warp per stencil.  COND = false: the weights of the requested operators
// (right-hand sides per rhs_value), written to w.  COND = true: the 1-norm
// condition number ||A_aug||_1 ||A_aug^-1||_1 of the same local system (the
// right-hand sides are the S unit vectors, nrhs = S), written to w[i].
template <bool COND>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32)
    weights_kernel(const double* __restrict__ ax, const double* __restrict__ ay, int64_t na,
                   const double* __restrict__ bx, const double* __restrict__ by,
                   const int32_t* __restrict__ idx, int64_t ld, int n, int m, int q, int nrhs,
                   int4 ops, int LD, double* __restrict__ w,
                   unsigned long long* __restrict__ bad) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int np = q < 0 ? 0 : (q + 1) * (q + 2) / 2;
  const int S = n + np, NC = S + nrhs;
  double* Am = smem + (size_t)wib * (LD * NC + 2 * n + S);
  double* xs = Am + LD * NC;
  double* ys = xs + n;
  double* invd = ys + n;  // reciprocals of U's diagonal
  const int op_of[4] = {ops.x, ops.y, ops.z, ops.w};
  const int wpb = blockDim.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * wpb + wib;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  const int npair = n * (n - 1) / 2;
  for (int64_t i = gw; i < na; i += nwarps) {
    const double cx = ax[i], cy = ay[i];
    double r2max = 0.0;
    for (int s = lane; s < n; s += 32) {
      const int j = idx[s * ld + i];
      const double X = bx[j] - cx, Y = by[j] - cy;
      xs[s] = X;
      ys[s] = Y;
      r2max = fmax(r2max, X * X + Y * Y);
    }
    for (int o = 16; o > 0; o >>= 1) r2max = fmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
    const double sc = sqrt(r2max);
    const double isc = 1.0 / sc;
    __syncwarp();
    for (int s = lane; s < n; s += 32) {
      xs[s] = xs[s] * isc;
      ys[s] = ys[s] * isc;
    }
    __syncwarp();
    // ---- assemble [A P; P^T 0 | rhs] column-major: element (r, c) at Am[c*LD + r].
    // A is symmetric with phi(0) = 0 on its diagonal: each pair (r < c) is
    // evaluated once and stored twice.
    double amax = 0.0;
    for (int p = lane; p < npair; p += 32) {
      int c = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
      while (c * (c - 1) / 2 > p) --c;
      while (c * (c + 1) / 2 <= p) ++c;
      const int r = p - c * (c - 1) / 2;
      const double dx = xs[r] - xs[c], dy = ys[r] - ys[c];
      const double v = phs_from_r2(dx * dx + dy * dy, m);
      Am[c * LD + r] = v;
      Am[r * LD + c] = v;
      amax = fmax(amax, fabs(v));
    }
    for (int r = lane; r < n; r += 32) Am[r * LD + r] = 0.0;
    for (int e = lane; e < n * np; e += 32) {  // P (row r, monomial t) and P^T
      const int t = e / n, r = e - t * n;
      int a, b;
      monomial(t, a, b);
      const double v = ipow(xs[r], a) * ipow(ys[r], b);
      Am[(n + t) * LD + r] = v;
      Am[r * LD + n + t] = v;
      amax = fmax(amax, fabs(v));
    }
    for (int e = lane; e < np * np; e += 32) {
      const int c = e / np, r = e - c * np;
      Am[(n + c) * LD + n + r] = 0.0;
    }
    if (COND) {
      for (int e = lane; e < S * S; e += 32) {
        const int o = e / S, r = e - o * S;
        Am[(S + o) * LD + r] = r == o ? 1.0 : 0.0;
      }
    } else {
      for (int e = lane; e < S * nrhs; e += 32) {
        const int o = e / S, r = e - o * S;
        const double X = r < n ? xs[r] : 0.0, Y = r < n ? ys[r] : 0.0;
        Am[(S + o) * LD + r] = rhs_value(op_of[o], r, n, m, X, Y);
      }
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncwarp();
    double anorm = 0.0;  // ||A_aug||_1, the largest column sum
    if (COND) {
      for (int c = lane; c < S; c += 32) {
        double cs = 0.0;
        for (int r = 0; r < S; ++r) cs += fabs(Am[c * LD + r]);
        anorm = fmax(anorm, cs);
      }
      for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    }
    // ---- elimination with partial pivoting
    bool singular = false;
    for (int kk = 0; kk < S; ++kk) {
      unsigned long long bk = 0ull;
      int br = S;
      for (int r = kk + lane; r < S; r += 32) {
        const unsigned long long key = mag_key(Am[kk * LD + r]);
        if (br == S || key > bk) {
          bk = key;
          br = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ok > bk || (ok == bk && orr < br)) {
          bk = ok;
          br = orr;
        }
      }
      const double bv = __longlong_as_double((long long)bk);
      if (!(bv > 1e-14 * amax) || !isfinite(bv)) {
        singular = true;
        break;
      }
      if (br != kk) {
        for (int c = kk + lane; c < NC; c += 32) {
          const double t = Am[c * LD + kk];
          Am[c * LD + kk] = Am[c * LD + br];
          Am[c * LD + br] = t;
        }
      }
      __syncwarp();
      const double inv = 1.0 / Am[kk * LD + kk];
      if (lane == 0) invd[kk] = inv;
      for (int r = kk + 1 + lane; r < S; r += 32) Am[kk * LD + r] *= inv;
      __syncwarp();
      const int R = S - 1 - kk, C = NC - 1 - kk;
      for (int p = lane; p < R * C; p += 32) {
        const int c = kk + 1 + p / R, r = kk + 1 + (p - (p / R) * R);
        Am[c * LD + r] -= Am[kk * LD + r] * Am[c * LD + kk];
      }
      __syncwarp();
    }
    if (singular) {
      if (lane == 0) atomicMin(bad, (unsigned long long)i);
      if (COND) {
        if (lane == 0) w[i] = INFINITY;
      } else {
        for (int e = lane; e < nrhs * n; e += 32) {
          const int o = e / n, s = e - o * n;
          w[(int64_t)o * n * ld + (int64_t)s * ld + i] = 0.0;
        }
      }
      __syncwarp();
      continue;
    }
    // ---- back substitution on the upper triangle, all right-hand sides
    for (int c = S - 1; c >= 0; --c) {
      const double ic = invd[c];
      for (int o = lane; o < nrhs; o += 32) Am[(S + o) * LD + c] *= ic;
      __syncwarp();
      for (int p = lane; p < c * nrhs; p += 32) {
        const int o = p / c, r = p - o * c;
        Am[(S + o) * LD + r] -= Am[c * LD + r] * Am[(S + o) * LD + c];
      }
      __syncwarp();
    }
    if (COND) {
      double inorm = 0.0;  // ||A_aug^-1||_1 from the solved unit vectors
      for (int o = lane; o < S; o += 32) {
        double cs = 0.0;
        for (int r = 0; r < S; ++r) cs += fabs(Am[(S + o) * LD + r]);
        inorm = fmax(inorm, cs);
      }
      for (int o = 16; o > 0; o >>= 1) inorm = fmax(inorm, __shfl_xor_sync(0xffffffffu, inorm, o));
      if (lane == 0) w[i] = anorm * inorm;
      __syncwarp();
      continue;
    }
    // ---- unscale and store w (the first n entries of each solution)
    for (int e = lane; e < nrhs * n; e += 32) {
      const int o = e / n, s = e - o * n;
      const int op = op_of[o];
      double v = Am[(S + o) * LD + s];
      if (op == 1 || op == 2) v *= isc;
      else if (op == 3) v *= isc * isc;
      w[(int64_t)o * n * ld + (int64_t)s * ld + i] = v;
    }
    __syncwarp();
  }
}

// shared memory of one warp (the system with its right-hand sides, the local
// coordinates and the pivot reciprocals) and the launch shape
struct WShape {
  int LD, wpb;
  size_t smem;
};
inline WShape weights_shape(int n, int S, int nrhs) {
  WShape sh;
  sh.LD = (S % 2) ? S : S + 1;
  const size_t per_warp = sizeof(double) * ((size_t)sh.LD * (S + nrhs) + 2 * n + S);
  sh.wpb = (int)std::max<size_t>(1, std::min<size_t>(kMaxWarpsPerBlock, kSmemBudget / per_warp));
  sh.smem = per_warp * sh.wpb;
  return sh;
}

}  // namespace

int weights_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
                  const double* by, const int32_t* idx, int64_t ld, uint32_t op_mask, double* w,
                  int64_t* bad_node, cudaStream_t st) {
  const int n = ctx->prm.n, m = ctx->prm.m, q = ctx->prm.q;
  const int np = q < 0 ? 0 : (q + 1) * (q + 2) / 2;
  const int S = n + np;
  int opv[4] = {0, 0, 0, 0};
  int nrhs = 0;
  for (int b = 0; b < 4; ++b)
    if (op_mask & (1u << b)) opv[nrhs++] = b;
  const WShape sh = weights_shape(n, S, nrhs);
  const int LD = sh.LD, wpb = sh.wpb;
  const size_t smem = sh.smem;
  int rc = check_cuda(ctx,
                      cudaFuncSetAttribute(weights_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                      "weights smem attribute");
  if (rc) return rc;
  void* base = nullptr;
  rc = ctx_scratch(ctx, 256, &base);
  if (rc) return rc;
  unsigned long long* d_bad = (unsigned long long*)base;
  rc = check_cuda(ctx, cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), st), "memset");
  if (rc) return rc;
  const int sms = sm_count();
  const int64_t need = (na + wpb - 1) / wpb;
  const int blocks = (int)std::min<int64_t>(need, (int64_t)sms * 16);
  weights_kernel<false><<<blocks, wpb * 32, smem, st>>>(
      ax, ay, na, bx, by, idx, ld, n, m, q, nrhs, make_int4(opv[0], opv[1], opv[2], opv[3]), LD,
      w, d_bad);
  rc = check_cuda(ctx, cudaGetLastError(), "weights kernel");
  if (rc) return rc;
  unsigned long long* h_bad = (unsigned long long*)ctx->host_pinned;
  rc = check_cuda(ctx, cudaMemcpyAsync(h_bad, d_bad, sizeof(*h_bad), cudaMemcpyDeviceToHost, st),
                  "status copy");
  if (rc) return rc;
  rc = check_cuda(ctx, cudaStreamSynchronize(st), "weights sync");
  if (rc) return rc;
  if (*h_bad != ~0ull) {
    if (bad_node) *bad_node = (int64_t)*h_bad;
    return set_error(ctx, RBFFD_ERR_SINGULAR_STENCIL, "singular stencil system at alpha-node %lld",
                     (long long)*h_bad);
  }
  return RBFFD_OK;
}

}  // namespace rbffd

namespace rbffd {

// The weight solves of weights_build with the singular-stencil status word in
// caller-provided device memory (no context, no allocation).  Returns an
// RBFFD status code; bad_node (host, may be null) as in weights_build.
int weights_build_scratch(int n, int m, int q, const double* ax, const double* ay, int64_t na,
                          const double* bx, const double* by, const int32_t* idx, int64_t ld,
                          uint32_t op_mask, double* w, unsigned long long* d_bad,
                          int64_t* bad_node, cudaStream_t st) {
  const int np = q < 0 ? 0 : (q + 1) * (q + 2) / 2;
  const int S = n + np;
  int opv[4] = {0, 0, 0, 0};
  int nrhs = 0;
  for (int b = 0; b < 4; ++b)
    if (op_mask & (1u << b)) opv[nrhs++] = b;
  const WShape sh = weights_shape(n, S, nrhs);
  const int LD = sh.LD, wpb = sh.wpb;
  const size_t smem = sh.smem;
  if (cudaFuncSetAttribute(weights_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return RBFFD_ERR_CUDA;
  // the status word keeps the previous call's value: reset it
  if (cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), st) != cudaSuccess)
    return RBFFD_ERR_CUDA;
  const int sms = sm_count();
  const int64_t need = (na + wpb - 1) / wpb;
  const int blocks = (int)std::min<int64_t>(need, (int64_t)sms * 16);
  weights_kernel<false><<<blocks, wpb * 32, smem, st>>>(ax, ay, na, bx, by, idx, ld, n, m, q,
                                                        nrhs,
                                                        make_int4(opv[0], opv[1], opv[2], opv[3]),
                                                        LD, w, d_bad);
  unsigned long long h_bad = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RBFFD_ERR_CUDA;
  if (h_bad != ~0ull) {
    if (bad_node) *bad_node = (int64_t)h_bad;
    return RBFFD_ERR_SINGULAR_STENCIL;
  }
  return RBFFD_OK;
}

}  // namespace rbffd

namespace rbffd {

// 1-norm condition numbers of the local systems the weight solves factor
// (rbffd_stencil_condition): the weight kernel in its COND mode.
int cond_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
               const double* by, const int32_t* idx, int64_t ld, double* cond,
               cudaStream_t st) {
  const int n = ctx->prm.n, m = ctx->prm.m, q = ctx->prm.q;
  const int np = q < 0 ? 0 : (q + 1) * (q + 2) / 2;
  const int S = n + np;
  const WShape sh = weights_shape(n, S, S);
  int rc = check_cuda(ctx,
                      cudaFuncSetAttribute(weights_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sh.smem),
                      "condition smem attribute");
  if (rc) return rc;
  void* base = nullptr;
  rc = ctx_scratch(ctx, 256, &base);
  if (rc) return rc;
  unsigned long long* d_bad = (unsigned long long*)base;
  rc = check_cuda(ctx, cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), st), "memset");
  if (rc) return rc;
  const int64_t need = (na + sh.wpb - 1) / sh.wpb;
  const int blocks = (int)std::min<int64_t>(need, (int64_t)sm_count() * 16);
  weights_kernel<true><<<blocks, sh.wpb * 32, sh.smem, st>>>(
      ax, ay, na, bx, by, idx, ld, n, m, q, S, make_int4(0, 0, 0, 0), sh.LD, cond, d_bad);
  rc = check_cuda(ctx, cudaGetLastError(), "condition kernel");
  if (rc) return rc;
  return check_cuda(ctx, cudaStreamSynchronize(st), "condition sync");
}

}  // namespace rbffd
