// The fractional step of Section 3 on the GPU: explicit stages as fused ELL
// kernels, implicit stages as BiCGSTAB solves built on the same ELL streams.
//
// Layout: every operator is slot-major ELL (idx[s*ld+i], w[s*ld+i]); state
// vectors are plain FP64 arrays.  In MIXED precision the explicit stages use
// FP32 weights, and every vector they gather also has a split FP32 copy
// (hi, lo) with hi + lo == x to about 2^-48 relative: FP32 derivative
// operators gather differences (x_j - x_ref) = (hi_j - hi_ref) + (lo_j - lo_ref)
// against the stencil's nearest node, so the cancellation of a derivative
// stencil happens before the rounding to FP32 rather than after it.  The
// divergence (the pressure solve's right side) keeps FP64 weights.
//
// Implicit solves (rows scaled as below, relative residual on the scaled
// system):
//   viscous:  H x = b, H = I - a_i D^(V,V)_Lap, a_i = dt/(2 Re) inside and 0
//             on wall rows, which are identity rows (Eq. u_ss);
//   pressure: S (L - e 1^T) x = S b, L = D^(P,P)_Lap inside and the Neumann
//             row n_x D_x + n_y D_y on boundary rows, e = indicator of the
//             boundary rows, S = diag(1/L_ii) (1/sum_j |L_ij| on a row whose
//             diagonal vanishes).  L annihilates constants, so the rank-one term
//             fixes the constant mode: x = p~ + c 1 for the mean-zero solution
//             p~ of the bordered system [L e; 1^T 0] (the multiplier c absorbs
//             the incompatibility of the non-symmetric L as a uniform normal
//             derivative on the Neumann rows, so every interior row is
//             Eq. pressure_Poisson exactly), and p~ = x - mean(x).
// FP64 precision: BiCGSTAB in FP64.  MIXED: FP64 iterative refinement whose
// corrections come from FP32 solves on FP32 copies of the scaled operators.
// Pressure solves are right-preconditioned by the multigrid V-cycle of
// amg.cuh (one application per search direction).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

#include "amg.cuh"
#include "common.cuh"

namespace rbffd {

namespace {

constexpr int kThreads = 256;
constexpr int kNV = 6;  // values reduced per kernel

// RBFFD_TRACE=1 in the environment prints one line per solve and refinement
// sweep to stderr (iterations, residuals, status).
bool trace_on() {
  static const bool on = [] {
    const char* e = getenv("RBFFD_TRACE");
    return e && *e && *e != '0';
  }();
  return on;
}

struct KScal {
  double rho[2], alpha[2], omega[2], beta[2];
  double rr[2], bb[2];
  double sum_p, sum_s;
  double cp, cs;  // preconditioned solves: (c . p), (c . s) of the multigrid's level-0 map
  double kap[2];  // preconditioned solves: B p = zp + kap[0], B s = zs + kap[1]
  double tol2;
  int active[2];
  int half[2];
  int iters;
  int maxit;
  int done;
  int status;  // 0 ok, 2 non-finite, 1/3/4 breakdown at (rh,v) = 0 / (t,t) = 0 / rho or
               // omega = 0, 5 residual grew beyond 1e4 ||b||
  int stage_err;  // nonzero: a tile copy did not complete within the bounded wait
};

__device__ __forceinline__ float2 split2(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

template <typename TW, typename TV>
struct KOp {
  const int32_t* idx;
  const TW* w;
  int64_t ld;
  int64_t n;
  int k;
  int diag1;       // add x_i (identity part of H)
  const TV* es;    // rank-one column, or null
  const TV* rdot;  // rank-one row (y += es * (rdot . x)); null = all ones
  const TV* a1 = nullptr;  // A 1 (row sums): the product with a constant shift
  // tile records of (idx, w) in the layout of one EllStage each (null: none):
  // a staged SpMV then moves a whole tile with one bulk copy
  const unsigned char* tiles = nullptr;
  // rows in difference form (needs a1): (A x)_i = sum_s w_s (x_j - x_i) + a1_i x_i
  int diff = 0;
};

template <typename T>
struct Acc;
template <>
struct Acc<double> {
  using t = double;
};
template <>
struct Acc<float> {
  using t = float;
};

// Self-checks of a diagnostic build (-DRBFFD_SELF_CHECK): an index outside
// its array is reported (first few, with the site, row and index) and the
// access is skipped instead of made.
#ifdef RBFFD_SELF_CHECK
__device__ int g_check_prints = 0;
__device__ __forceinline__ bool index_ok(long long j, long long n, int site, long long row) {
  if (j >= 0 && j < n) return true;
  if (atomicAdd(&g_check_prints, 1) < 20)
    printf("[rbffd self-check] site %d row %lld index %lld bound %lld\n", site, row, j, n);
  return false;
}
#define RBFFD_CHECK(j, n, site, row) \
  if (!index_ok((long long)(j), (long long)(n), (site), (long long)(row))) continue
#else
#define RBFFD_CHECK(j, n, site, row)
#endif

// sum_s w[s][i] * x[idx[s][i]] for one or two vectors sharing the stencil,
// accumulated in the precision of the vectors (in difference form when
// op.diff is set, as k_spmv_pc applies those rows)
template <int K, int NRHS, typename TW, typename TV>
__device__ __forceinline__ void gather_rows(const KOp<TW, TV>& op, int64_t i, const TV* const* x,
                                            typename Acc<TV>::t* acc) {
  using A = typename Acc<TV>::t;
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = 0;
  const int k = K > 0 ? K : op.k;
  if (op.diff) {
    A xi[NRHS];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) xi[r] = (A)x[r][i];
#pragma unroll(K > 0 ? K : 1)
    for (int s = 0; s < k; ++s) {
      const int j = op.idx[s * op.ld + i];
      if (K == 0) RBFFD_CHECK(j, op.n, 1, i);
      const A w = (A)op.w[s * op.ld + i];
#pragma unroll
      for (int r = 0; r < NRHS; ++r) acc[r] += w * ((A)x[r][j] - xi[r]);
    }
#pragma unroll
    for (int r = 0; r < NRHS; ++r) acc[r] += (A)op.a1[i] * xi[r];
    return;
  }
#pragma unroll(K > 0 ? K : 1)
  for (int s = 0; s < k; ++s) {
    const int j = op.idx[s * op.ld + i];
    if (K == 0) RBFFD_CHECK(j, op.n, 1, i);
    const A w = (A)op.w[s * op.ld + i];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) acc[r] += w * (A)x[r][j];
  }
}

// ------------------------------------------------ staged ELL tiles (bulk copies)
// A block stages the idx and weight columns of 256 consecutive rows into
// shared memory: one contiguous segment per stencil slot, moved by
// cp.async.bulk copies that complete on an mbarrier.  The threads then gather
// x for their own row with every address already on chip, so the streaming
// part of the SpMV never waits on the gathers.
constexpr int kTileRows = 256;
constexpr long long kSpinLimit = 1ll << 22;  // bounded mbarrier wait (a tile lands in microseconds)

// Polls of the first wait for a staged tile or record (kSpinLimit unless a
// test lowers it through rbffd_debug_set_wait_limit).  After a failed first
// wait the block still waits, up to kSpinLimit polls, for the copies it
// issued, so lowering it never leaves a copy in flight into a finished block.
__device__ long long g_wait_polls = kSpinLimit;

// Rows are staged whenever the stencil size is a compile-time constant: with
// every address on chip the gathers never stall the stream (measured at 1M
// rows: 63 us per FP32 launch staged against 102 us with direct loads).
template <int K, typename TW>
constexpr bool kStage = K > 0;

template <int K, typename TW>
struct EllStage {
  int32_t idx[K * kTileRows];
  TW w[K * kTileRows];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Stage rows [row0, row0 + 256) of (idx, w); every thread returns once the
// copies have landed, or false after kSpinLimit polls (then *err is set).
template <int K, typename TW>
__device__ __forceinline__ bool stage_tile(EllStage<K, TW>* tile, uint64_t* bar, uint32_t& phase,
                                           const int32_t* __restrict__ gidx,
                                           const TW* __restrict__ gw, int64_t ld, int64_t row0,
                                           int* err, const unsigned char* tiles = nullptr) {
  __syncthreads();  // every thread is done with the previous tile
  if (threadIdx.x == 0 && tiles) {
    // one record per tile, already in the EllStage layout: one copy
    constexpr uint32_t rec = (uint32_t)sizeof(EllStage<K, TW>);
    mbar_expect_tx(bar, rec);
    bulk_g2s(tile, tiles + (row0 / kTileRows) * (int64_t)rec, rec, bar);
  } else if (threadIdx.x == 0) {
    const int64_t left = ld - row0;
    const uint32_t rows = (uint32_t)(left < kTileRows ? left : kTileRows);  // multiple of 32
    const uint32_t bi = rows * 4u, bw = rows * (uint32_t)sizeof(TW);
    mbar_expect_tx(bar, (uint32_t)K * (bi + bw));
#pragma unroll 4
    for (int s = 0; s < K; ++s) {
      bulk_g2s(&tile->idx[s * kTileRows], gidx + s * ld + row0, bi, bar);
      bulk_g2s(&tile->w[s * kTileRows], gw + s * ld + row0, bw, bar);
    }
  }
  const long long limit = g_wait_polls;
  long long spins = 0;
  bool ok = false;
  while (spins < limit && !(ok = mbar_try_wait(bar, phase))) ++spins;
  // one verdict for the whole block, so every thread leaves the loop together
  if (!__syncthreads_and(ok ? 1 : 0)) {
    if (threadIdx.x == 0) atomicOr(err, 4);
    // give the copies in flight one more bounded chance to land before the block leaves
    spins = 0;
    while (!mbar_try_wait(bar, phase) && ++spins < kSpinLimit) {
    }
    return false;
  }
  phase ^= 1u;
  return true;
}

template <typename TV, int NRHS>
struct Vecs {
  TV* v[NRHS];
};

// the same sums with idx and w read from a staged tile
template <int K, int NRHS, typename TW, typename TV>
__device__ __forceinline__ void gather_tile(const EllStage<K, TW>* t, int tid, const TV* const* x,
                                            typename Acc<TV>::t* acc) {
  using A = typename Acc<TV>::t;
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r] = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int j = t->idx[s * kTileRows + tid];
    const A w = (A)t->w[s * kTileRows + tid];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) acc[r] += w * (A)x[r][j];
  }
}

// ----------------------------------------------------------- Krylov kernels
// sum_i x_i, or sum_i c_i x_i when c is given
template <typename TV>
__global__ void __launch_bounds__(kThreads) k_sum(const TV* __restrict__ x, int64_t n,
                                                  GridReduce gr, double* out,
                                                  const TV* __restrict__ c = nullptr) {
  constexpr int NU_ = 1;
  __shared__ double sh[NU_ * kThreads];
  float part = 0.f;
  double partd = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const TV xi = c ? c[i] * x[i] : x[i];
    if (sizeof(TV) == 8)
      partd += (double)xi;
    else
      part += (float)xi;
  }
  double v[NU_] = {partd + (double)part};
  grid_reduce<NU_>(v, gr, sh, [&](double* t) { *out = t[0]; });
}

// sign pattern of a restarted shadow residual (a 32-bit integer hash of i and the seed)
__device__ __forceinline__ float shadow_sign(int64_t i, uint32_t seed) {
  uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (h & 1u) ? 1.f : -1.f;
}

// r = b - A x ; p = r ; shadow residual rh = r (seed 0) or r with seeded signs
template <int K, int NRHS, bool RANK1, typename TW, typename TV>
__global__ void __launch_bounds__(kThreads)
    k_init(KOp<TW, TV> op, Vecs<TV, NRHS> x, Vecs<TV, NRHS> b, Vecs<TV, NRHS> r,
           Vecs<TV, NRHS> rh, Vecs<TV, NRHS> p, const double* sigma_x, KScal* sc, GridReduce gr,
           double tol2, int maxit, uint32_t seed, const float* __restrict__ pcc, int x_zero) {
  using A = typename Acc<TV>::t;
  constexpr int NU_ = kNV;
  __shared__ double sh[NU_ * kThreads];
  A prr[2] = {0, 0}, pbb[2] = {0, 0}, prh[2] = {0, 0}, psum = 0;
  const A sig = (RANK1 && !x_zero) ? (A)*sigma_x : (A)0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < op.n;
       i += (int64_t)gridDim.x * kThreads) {
    A acc[NRHS];
    if (x_zero) {  // x = 0: r = b without the product
#pragma unroll
      for (int q = 0; q < NRHS; ++q) acc[q] = 0;
    } else {
      gather_rows<K, NRHS>(op, i, (const TV* const*)x.v, acc);
    }
    const A sgn = seed ? (A)shadow_sign(i, seed) : (A)1;
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      A ax = acc[q];
      if (op.diag1) ax += (A)x.v[q][i];
      if (RANK1) ax += (A)op.es[i] * sig;
      const A bi = (A)b.v[q][i];
      const A ri = bi - ax;
      r.v[q][i] = (TV)ri;
      rh.v[q][i] = (TV)(sgn * ri);
      p.v[q][i] = (TV)ri;
      prr[q] += ri * ri;
      pbb[q] += bi * bi;
      prh[q] += sgn * ri * ri;
      if (RANK1) psum += pcc ? (A)pcc[i] * ri : (op.rdot ? (A)op.rdot[i] * ri : ri);
    }
  }
  double v[kNV] = {(double)prr[0], (double)pbb[0], (double)prr[1],
                   (double)pbb[1], (double)prh[0], (double)prh[1]};
  if (RANK1) v[5] = (double)psum;  // NRHS == 1 here: slot 5 carries sum(r)
  grid_reduce<NU_>(v, gr, sh, [&](double* t) {
    sc->tol2 = tol2;
    sc->maxit = maxit;
    sc->iters = 0;
    sc->status = 0;
    sc->stage_err = 0;
    int any = 0;
    for (int q = 0; q < NRHS; ++q) {
      const double rr = t[2 * q], bb = t[2 * q + 1];
      const double rho = q == 0 ? t[4] : t[5];
      sc->rr[q] = rr;
      sc->bb[q] = bb;
      sc->rho[q] = rho;
      sc->alpha[q] = 1.0;
      sc->omega[q] = 1.0;
      sc->half[q] = 0;
      if (!isfinite(rr)) sc->status = 2;
      sc->active[q] = (isfinite(rr) && rr > tol2 * bb && rho != 0.0) ? 1 : 0;
      any |= sc->active[q];
    }
    for (int q = NRHS; q < 2; ++q) sc->active[q] = 0;
    if (RANK1) {
      if (pcc)
        sc->cp = t[5];
      else
        sc->sum_p = t[5];
    }
    sc->done = (any && maxit > 0) ? 0 : 1;
  });
}

// v = A p ; reduce (rh, v).  K > 0: rows come in staged tiles (dynamic shared
// memory holds one EllStage); K == 0: rows are read directly.
template <int K, int NRHS, bool RANK1, typename TW, typename TV, int DIRECT = 0>
__global__ void __launch_bounds__(kThreads, DIRECT ? DIRECT : 1)
    k_spmv_p(KOp<TW, TV> op, Vecs<TV, NRHS> p, Vecs<TV, NRHS> v, Vecs<TV, NRHS> rh, KScal* sc,
             GridReduce gr, int* worked) {
  using A = typename Acc<TV>::t;
  if (sc->done) return;
  if (worked && blockIdx.x == 0 && threadIdx.x == 0) *worked = 1;
  constexpr int NU_ = NRHS;
  __shared__ double sh[NU_ * kThreads];
  const A sig = RANK1 ? (A)sc->sum_p : (A)0;
  A pd[2] = {0, 0};
  auto finish_row = [&](int64_t i, A* acc) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      A y = acc[q];
      if (op.diag1) y += (A)p.v[q][i];
      if (RANK1) y += (A)op.es[i] * sig;
      v.v[q][i] = (TV)y;
      pd[q] += (A)rh.v[q][i] * y;
    }
  };
  if constexpr (kStage<K, TW> && DIRECT == 0) {
    extern __shared__ __align__(128) unsigned char dsm[];
    auto* tile = reinterpret_cast<EllStage<K, TW>*>(dsm);
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const int64_t ntiles = (op.n + kTileRows - 1) / kTileRows;
    for (int64_t tix = blockIdx.x; tix < ntiles; tix += gridDim.x) {
      const int64_t row0 = tix * kTileRows;
      if (!stage_tile<K, TW>(tile, &bar, phase, op.idx, op.w, op.ld, row0, &sc->stage_err,
                             op.tiles))
        break;
      const int64_t i = row0 + threadIdx.x;
      if (i < op.n) {
        A acc[NRHS];
        gather_tile<K, NRHS>(tile, threadIdx.x, (const TV* const*)p.v, acc);
        finish_row(i, acc);
      }
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < op.n;
         i += (int64_t)gridDim.x * kThreads) {
      A acc[NRHS];
      gather_rows<K, NRHS>(op, i, (const TV* const*)p.v, acc);
      finish_row(i, acc);
    }
  }
  double vv[NU_];
#pragma unroll
  for (int q = 0; q < NU_; ++q) vv[q] = (double)pd[q];
  grid_reduce<NU_>(vv, gr, sh, [&](double* t) {
    if (sc->stage_err) sc->done = 1;
    for (int q = 0; q < NRHS; ++q) {
      if (!sc->active[q]) continue;
      const double rv = t[q];
      if (rv == 0.0 || !isfinite(rv)) {
        sc->active[q] = 0;
        sc->status = isfinite(rv) ? 1 : 2;
        continue;
      }
      sc->alpha[q] = sc->rho[q] / rv;
    }
  });
}

// s = r - alpha v ; reduce (s, s) and sum(s)
template <int NRHS, bool RANK1, typename TV>
__global__ void __launch_bounds__(kThreads)
    k_update_s(int64_t n, Vecs<TV, NRHS> r, Vecs<TV, NRHS> v, Vecs<TV, NRHS> s, KScal* sc,
               GridReduce gr, const TV* __restrict__ rdot, const float* __restrict__ pcc) {
  using A = TV;
  if (sc->done) return;
  constexpr int NU_ = 3;
  __shared__ double sh[NU_ * kThreads];
  A al[2];
  int act[2];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    al[q] = (A)sc->alpha[q];
    act[q] = sc->active[q];
  }
  A pss[2] = {0, 0}, psum = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      if (!act[q]) continue;
      const A si = r.v[q][i] - al[q] * v.v[q][i];
      s.v[q][i] = si;
      pss[q] += si * si;
      if (RANK1) psum += pcc ? (A)pcc[i] * si : (rdot ? rdot[i] * si : si);
    }
  }
  double vv[NU_] = {(double)pss[0], (double)pss[1], (double)psum};
  grid_reduce<NU_>(vv, gr, sh, [&](double* t) {
    for (int q = 0; q < NRHS; ++q)
      if (sc->active[q] && t[q] <= sc->tol2 * sc->bb[q]) sc->half[q] = 1;
    if (RANK1) {
      if (pcc)
        sc->cs = t[2];
      else
        sc->sum_s = t[2];
    }
  });
}

// t = A s^ ; reduce (t, s), (t, t)  (staged tiles when K > 0).  s^ = s, or the
// preconditioned B s in a preconditioned solve; sres = s.
template <int K, int NRHS, bool RANK1, typename TW, typename TV, int DIRECT = 0>
__global__ void __launch_bounds__(kThreads, DIRECT ? DIRECT : 1)
    k_spmv_s(KOp<TW, TV> op, Vecs<TV, NRHS> s, Vecs<TV, NRHS> sres, Vecs<TV, NRHS> t, KScal* sc,
             GridReduce gr, int* worked) {
  using A = typename Acc<TV>::t;
  if (sc->done) return;
  if (worked && blockIdx.x == 0 && threadIdx.x == 0) *worked = 1;
  constexpr int NU_ = 2 * NRHS;
  __shared__ double sh[NU_ * kThreads];
  const A sig = RANK1 ? (A)sc->sum_s : (A)0;
  A pts[2] = {0, 0}, ptt[2] = {0, 0};
  auto finish_row = [&](int64_t i, A* acc) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      A y = acc[q];
      if (op.diag1) y += (A)s.v[q][i];
      if (RANK1) y += (A)op.es[i] * sig;
      t.v[q][i] = (TV)y;
      pts[q] += y * (A)sres.v[q][i];
      ptt[q] += y * y;
    }
  };
  if constexpr (kStage<K, TW> && DIRECT == 0) {
    extern __shared__ __align__(128) unsigned char dsm[];
    auto* tile = reinterpret_cast<EllStage<K, TW>*>(dsm);
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const int64_t ntiles = (op.n + kTileRows - 1) / kTileRows;
    for (int64_t tix = blockIdx.x; tix < ntiles; tix += gridDim.x) {
      const int64_t row0 = tix * kTileRows;
      if (!stage_tile<K, TW>(tile, &bar, phase, op.idx, op.w, op.ld, row0, &sc->stage_err,
                             op.tiles))
        break;
      const int64_t i = row0 + threadIdx.x;
      if (i < op.n) {
        A acc[NRHS];
        gather_tile<K, NRHS>(tile, threadIdx.x, (const TV* const*)s.v, acc);
        finish_row(i, acc);
      }
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < op.n;
         i += (int64_t)gridDim.x * kThreads) {
      A acc[NRHS];
      gather_rows<K, NRHS>(op, i, (const TV* const*)s.v, acc);
      finish_row(i, acc);
    }
  }
  double vv[NU_];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    vv[2 * q] = (double)pts[q];
    vv[2 * q + 1] = (double)ptt[q];
  }
  grid_reduce<NU_>(vv, gr, sh, [&](double* tt) {
    if (sc->stage_err) sc->done = 1;
    for (int q = 0; q < NRHS; ++q) {
      if (!sc->active[q] || sc->half[q]) continue;
      const double ts = tt[2 * q], t2 = tt[2 * q + 1];
      if (!(t2 > 0.0) || !isfinite(ts)) {
        sc->omega[q] = 0.0;
        sc->active[q] = 0;
        sc->status = isfinite(t2) ? 3 : 2;
        continue;
      }
      sc->omega[q] = ts / t2;
    }
  });
}

// x += alpha p^ + omega s^ ; r = s - omega t ; reduce (rh, r), (r, r).
// p^, s^ = p, s, or their preconditioned images in a preconditioned solve.
template <int NRHS, typename TV>
__global__ void __launch_bounds__(kThreads)
    k_update_xr(int64_t n, Vecs<TV, NRHS> x, Vecs<TV, NRHS> r, Vecs<TV, NRHS> rh,
                Vecs<TV, NRHS> p, Vecs<TV, NRHS> shat, Vecs<TV, NRHS> s, Vecs<TV, NRHS> t,
                KScal* sc, GridReduce gr) {
  using A = TV;
  if (sc->done) return;
  constexpr int NU_ = 2 * NRHS;
  __shared__ double sh[NU_ * kThreads];
  A al[2], om[2];
  int act[2], hf[2];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    al[q] = (A)sc->alpha[q];
    om[q] = (A)sc->omega[q];
    act[q] = sc->active[q];
    hf[q] = sc->half[q];
  }
  A prh[2] = {0, 0}, prr[2] = {0, 0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      if (!act[q]) continue;
      const A si = s.v[q][i];
      A ri;
      if (hf[q]) {
        x.v[q][i] += al[q] * p.v[q][i];
        ri = si;
      } else {
        x.v[q][i] += al[q] * p.v[q][i] + om[q] * shat.v[q][i];
        ri = si - om[q] * t.v[q][i];
      }
      r.v[q][i] = ri;
      prh[q] += rh.v[q][i] * ri;
      prr[q] += ri * ri;
    }
  }
  double vv[NU_];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    vv[2 * q] = (double)prh[q];
    vv[2 * q + 1] = (double)prr[q];
  }
  grid_reduce<NU_>(vv, gr, sh, [&](double* tt) {
    sc->iters += 1;
    int any = 0;
    for (int q = 0; q < NRHS; ++q) {
      if (!sc->active[q]) continue;
      const double rho_new = tt[2 * q], rr = tt[2 * q + 1];
      sc->rr[q] = rr;
      if (!isfinite(rr)) {
        sc->status = 2;
        sc->active[q] = 0;
        continue;
      }
      if (rr > 1e8 * sc->bb[q] && sc->bb[q] > 0.0) {  // the recurrence has blown up
        sc->status = 5;
        sc->active[q] = 0;
        continue;
      }
      if (sc->half[q] || rr <= sc->tol2 * sc->bb[q]) {
        sc->active[q] = 0;
        continue;
      }
      if (rho_new == 0.0 || sc->omega[q] == 0.0) {
        sc->status = 4;
        sc->active[q] = 0;
        continue;
      }
      sc->beta[q] = (rho_new / sc->rho[q]) * (sc->alpha[q] / sc->omega[q]);
      sc->rho[q] = rho_new;
      any = 1;
    }
    if (!any || sc->iters >= sc->maxit) sc->done = 1;
  });
}

// p = r + beta (p - omega v) ; reduce sum(p)
template <int NRHS, bool RANK1, typename TV>
__global__ void __launch_bounds__(kThreads)
    k_update_p(int64_t n, Vecs<TV, NRHS> r, Vecs<TV, NRHS> p, Vecs<TV, NRHS> v, KScal* sc,
               GridReduce gr, const TV* __restrict__ rdot, const float* __restrict__ pcc) {
  using A = TV;
  if (sc->done) return;
  constexpr int NU_ = 1;
  __shared__ double sh[NU_ * kThreads];
  A be[2], om[2];
  int act[2];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    be[q] = (A)sc->beta[q];
    om[q] = (A)sc->omega[q];
    act[q] = sc->active[q];
  }
  A psum = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      if (!act[q]) continue;
      const A pi = r.v[q][i] + be[q] * (p.v[q][i] - om[q] * v.v[q][i]);
      p.v[q][i] = pi;
      if (RANK1) psum += pcc ? (A)pcc[i] * pi : (rdot ? rdot[i] * pi : pi);
    }
  }
  double vv[NU_] = {(double)psum};
  grid_reduce<NU_>(vv, gr, sh, [&](double* tt) {
    if (RANK1) {
      if (pcc)
        sc->cp = tt[0];
      else
        sc->sum_p = tt[0];
    }
  });
}

// ------------------------------------------- multigrid preconditioner (amg.cuh)
// z = B v for a residual v of the scaled pressure system A_f = A + es 1^T:
//   mu = (c . v) / (c . es);  r0 = c v - mu ce;  y = one V-cycle on G for r0;
//   z = y - mean(y) + mu / M.
// Since A is close to diag(1/c) G and A 1 = 0, this inverts the constant mode
// exactly (B es = 1 / M, and A_f 1 / M = es) and G on the rest.  (c . v) and
// (c . s) come from the reductions of the kernels that produce p and s.

// B v = z + kap with kap = (mu - sum(z)) / M, so that B v = z - mean(z) + mu / M;
// the rank-one sum of B v is then mu.
__device__ __forceinline__ void pc_finish(KScal* sc, int which, double zsum, double inv_ces,
                                          double inv_R) {
  const double mu = (which ? sc->cs : sc->cp) * inv_ces;
  sc->kap[which] = (mu - zsum) * inv_R;
  if (which)
    sc->sum_s = mu;
  else
    sc->sum_p = mu;
}

// r0 = c v - mu ce in the hierarchy's level-0 order (row p is P-node perm0[p];
// which = 0: v = p, mu from sc->cp; 1: v = s, from sc->cs)
template <typename TV>
__global__ void __launch_bounds__(kThreads)
    k_pc_in(int64_t n, const TV* __restrict__ v, const float* __restrict__ c,
            const float* __restrict__ ce, const int32_t* __restrict__ perm0, int which,
            double inv_ces, const KScal* sc, float* __restrict__ r0) {
  if (sc->done) return;
  const float mu = (float)((which ? sc->cs : sc->cp) * inv_ces);
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads)
    r0[i] = c[i] * (float)v[perm0[i]] - mu * ce[i];
}

// sum_s G_off[i][s] * get(column) over a level's off-diagonal row.  W > 0:
// the loop is unrolled to W predicated slots so that every load of the row is
// in flight at once (the level's width is at most W); W = 0: a plain loop.
template <int W, typename Get>
__device__ __forceinline__ float graph_row(const AmgLevel& F, int64_t i, Get get) {
  float ax = 0.f;
  if constexpr (W > 0) {
#pragma unroll
    for (int s = 0; s < W; ++s)
      if (s < F.width) ax += F.val[s * F.ld + i] * get(F.idx[s * F.ld + i]);
  } else {
    for (int s = 0; s < F.width; ++s) ax += F.val[s * F.ld + i] * get(F.idx[s * F.ld + i]);
  }
  return ax;
}

// the unrolled width for a level: 8, 16 or 32 slots, or 0 (plain loop)
inline int width_bucket(int w) { return w <= 8 ? 8 : w <= 16 ? 16 : w <= 32 ? 32 : 0; }

// Pre-smoothing from zero (x = omega D^-1 r) and restriction of its residual:
// rc[I] = sum over the rows i of aggregate I of (r - G x)_i.  A block takes 64
// consecutive aggregates, whose rows are the consecutive rows cptr[I0] ..
// (at most 256): one thread per row (coalesced), the residuals staged in
// shared memory and summed per aggregate in row order.  Neighbours' x values
// are formed from their r on the fly.
constexpr int kRB = 64;  // aggregates per block (at most 4 rows each)

template <int W>
__global__ void __launch_bounds__(kThreads)
    k_pc_restrict(AmgLevel F, int64_t nc, float* __restrict__ rc, const KScal* sc) {
  if (sc->done) return;
  __shared__ float res[kThreads];
  for (int64_t I0 = blockIdx.x * (int64_t)kRB; I0 < nc; I0 += (int64_t)gridDim.x * kRB) {
    const int64_t I1 = I0 + kRB < nc ? I0 + kRB : nc;
    const int64_t f0 = F.cptr[I0], f1 = F.cptr[I1];
    const int64_t i = f0 + threadIdx.x;
    float rv = 0.f;
    if (i < f1) {
      const float ri = F.r[i];
      const float xi = F.wd[i] * ri;
      F.x[i] = xi;
      const float ax =
          F.diag[i] * xi + graph_row<W>(F, i, [&](int32_t j) { return F.wd[j] * F.r[j]; });
      rv = ri - ax;
    }
    res[threadIdx.x] = rv;
    __syncthreads();
    if (threadIdx.x < kRB && I0 + threadIdx.x < I1) {
      const int64_t I = I0 + threadIdx.x;
      float acc = 0.f;
      for (int64_t c = F.cptr[I]; c < F.cptr[I + 1]; ++c) acc += res[c - f0];
      rc[I] = acc;
    }
    __syncthreads();
  }
}

// x_fine[i] += s * z for the rows i of aggregate `row` (the coarse-grid
// correction of the finer level, written by the coarse level's thread; the
// rows are consecutive)
__device__ __forceinline__ void prolong_to(const AmgLevel& Fine, int64_t row, float z) {
  const float v = kAmgCoarseScale * z;
  const int32_t c1 = Fine.cptr[row + 1];
  for (int32_t c = Fine.cptr[row]; c < c1; ++c) Fine.x[c] += v;
}

// Coarsest level: z = X r with the dense inverse X (one warp per row), then
// the correction of the next finer level (has_fine) or the result itself.
template <typename TZ>
__global__ void __launch_bounds__(kThreads)
    k_pc_coarse(int64_t nc, const float* __restrict__ X, const float* __restrict__ r,
                TZ* __restrict__ z, AmgLevel Fine, int has_fine, const KScal* sc) {
  if (sc->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t row = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; row < nc; row += nw) {
    float acc = 0.f;
#pragma unroll 8
    for (int64_t j = lane; j < nc; j += 32) acc += X[row * nc + j] * r[j];
    acc = warp_sum(acc);
    if (lane == 0) {
      if (has_fine)
        prolong_to(Fine, row, acc);
      else
        z[row] = (TZ)acc;
    }
  }
}

// One post-smoothing sweep on a level whose x already holds the coarse-grid
// correction: z = x + omega D^-1 (r - G x).  Levels above 0 then add their
// correction to the next finer level (PROLONG; z is not stored); level 0
// stores z in the solve's precision and reduces its sum (REDUCE).
template <bool PROLONG, bool REDUCE, typename TZ, int W>
__global__ void __launch_bounds__(kThreads)
    k_pc_up(AmgLevel F, AmgLevel Fine, TZ* __restrict__ z, const int32_t* __restrict__ perm0,
            KScal* sc, GridReduce gr, int which, double inv_ces, double inv_R) {
  if (sc->done) return;
  constexpr int NU_ = 1;
  __shared__ double sh[NU_ * kThreads];
  float part = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < F.n;
       i += (int64_t)gridDim.x * kThreads) {
    const float xi = F.x[i];
    const float ax = F.diag[i] * xi + graph_row<W>(F, i, [&](int32_t j) { return F.x[j]; });
    const float zi = xi + F.wd[i] * (F.r[i] - ax);
    if (PROLONG) {
      prolong_to(Fine, i, zi);
    } else {
      z[perm0[i]] = (TZ)zi;  // back to P-node order
      if (REDUCE) part += zi;
    }
  }
  if (REDUCE) {
    double v[NU_] = {(double)part};
    grid_reduce<NU_>(v, gr, sh, [&](double* t) { pc_finish(sc, which, t[0], inv_ces, inv_R); });
  }
}

// Levels from block records (LevelRec): a block stages the record of its 64
// aggregates with one bulk copy (bounded wait; a copy that does not land sets
// the solve's stage error and ends the block's work), then runs the same
// arithmetic in the same order as k_pc_restrict / k_pc_up on those rows.
static_assert(kRB == kRecAggs && kThreads == kRecRows, "level-0 record shape");

template <int W>
__device__ __forceinline__ bool stage_rec(LevelRec<W>* rec, uint64_t* bar, uint32_t& phase,
                                          const unsigned char* __restrict__ recs, int64_t b,
                                          int* err) {
  __syncthreads();  // every thread is done with the previous record
  if (threadIdx.x == 0) {
    constexpr uint32_t bytes = (uint32_t)sizeof(LevelRec<W>);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(rec, recs + b * (int64_t)bytes, bytes, bar);
  }
  const long long limit = g_wait_polls;
  long long spins = 0;
  bool ok = false;
  while (spins < limit && !(ok = mbar_try_wait(bar, phase))) ++spins;
  if (!__syncthreads_and(ok ? 1 : 0)) {
    if (threadIdx.x == 0) atomicOr(err, 4);
    spins = 0;
    while (!mbar_try_wait(bar, phase) && ++spins < kSpinLimit) {
    }
    return false;
  }
  phase ^= 1u;
  return true;
}

// sum_s val[s] * get(idx[s]) over a record row's slots (slot s < width)
template <int W, typename Get>
__device__ __forceinline__ float rec_row(const LevelRec<W>& R, int width, int r, Get get) {
  float ax = 0.f;
#pragma unroll
  for (int s = 0; s < W; ++s)
    if (s < width) ax += R.val[s * kRecRows + r] * get(R.idx[s * kRecRows + r]);
  return ax;
}

template <int W>
__global__ void __launch_bounds__(kThreads)
    k_pc_restrict_rec(AmgLevel F, int64_t nrec, const unsigned char* __restrict__ recs,
                   float* __restrict__ rc, KScal* sc) {
  if (sc->done) return;
  __shared__ __align__(128) LevelRec<W> rec;
  __shared__ float res[kThreads];
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < nrec; b += gridDim.x) {
    if (!stage_rec<W>(&rec, &bar, phase, recs, b, &sc->stage_err)) break;
    float rv = 0.f;
    if (t < rec.nrows) {
      const int64_t i = (int64_t)rec.f0 + t;
      const float ri = F.r[i];
      const float xi = rec.wd[t] * ri;
      F.x[i] = xi;
      const float ax =
          rec.diag[t] * xi + rec_row<W>(rec, F.width, t, [&](int32_t j) { return F.wd[j] * F.r[j]; });
      rv = ri - ax;
    }
    res[t] = rv;
    __syncthreads();
    if (t < rec.nagg) {
      float acc = 0.f;
      for (int c = rec.off[t]; c < rec.off[t + 1]; ++c) acc += res[c];
      rc[b * kRB + t] = acc;
    }
  }
}

template <typename TZ, int W>
__global__ void __launch_bounds__(kThreads)
    k_pc_up0(AmgLevel F, int64_t nrec, const unsigned char* __restrict__ recs,
             TZ* __restrict__ z, KScal* sc, GridReduce gr, int which, double inv_ces,
             double inv_R) {
  if (sc->done) return;
  constexpr int NU_ = 1;
  __shared__ double sh[NU_ * kThreads];
  __shared__ __align__(128) LevelRec<W> rec;
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int t = threadIdx.x;
  float part = 0.f;
  for (int64_t b = blockIdx.x; b < nrec; b += gridDim.x) {
    if (!stage_rec<W>(&rec, &bar, phase, recs, b, &sc->stage_err)) break;
    if (t < rec.nrows) {
      const int64_t i = (int64_t)rec.f0 + t;
      const float xi = F.x[i];
      const float ax = rec.diag[t] * xi + rec_row<W>(rec, F.width, t, [&](int32_t j) { return F.x[j]; });
      const float zi = xi + rec.wd[t] * (F.r[i] - ax);
      z[rec.aux[t]] = (TZ)zi;  // back to P-node order
      part += zi;
    }
  }
  double v[NU_] = {(double)part};
  grid_reduce<NU_>(v, gr, sh, [&](double* t2) { pc_finish(sc, which, t2[0], inv_ces, inv_R); });
}

// levels above 0: the post-smoothing sweep adds its result, scaled, to the
// finer level's rows of each row's aggregate
template <int W>
__global__ void __launch_bounds__(kThreads)
    k_pc_up_rec(AmgLevel F, AmgLevel Fine, int64_t nrec, const unsigned char* __restrict__ recs,
                KScal* sc) {
  if (sc->done) return;
  __shared__ __align__(128) LevelRec<W> rec;
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < nrec; b += gridDim.x) {
    if (!stage_rec<W>(&rec, &bar, phase, recs, b, &sc->stage_err)) break;
    if (t < rec.nrows) {
      const int64_t i = (int64_t)rec.f0 + t;
      // the finer rows this row corrects (at most four), read with the gathers
      const int32_t c0 = rec.aux[t], c1 = rec.aux[t + 1];
      float xf[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xf[q] = c0 + q < c1 ? Fine.x[c0 + q] : 0.f;
      const float xi = F.x[i];
      const float ax = rec.diag[t] * xi + rec_row<W>(rec, F.width, t, [&](int32_t j) { return F.x[j]; });
      const float zi = xi + rec.wd[t] * (F.r[i] - ax);
      const float v = kAmgCoarseScale * zi;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c0 + q < c1) Fine.x[c0 + q] = xf[q] + v;
    }
  }
}

// one-level hierarchy: the lifted coarse solve is already mean-free
__global__ void k_pc_fin1(KScal* sc, int which, double inv_ces, double inv_R) {
  if (sc->done) return;
  pc_finish(sc, which, 0.0, inv_ces, inv_R);
}

// sum_s w[s][i] z[idx[s][i]]: FP64 sums in an FP64 solve, FP32 sums in an
// FP32 solve.
template <typename TW, typename TV>
struct ZAcc;
template <>
struct ZAcc<double, double> {
  double a = 0.0;
  __device__ __forceinline__ void add(double w, double z) { a += w * z; }
  __device__ __forceinline__ double get() const { return a; }
};
template <>
struct ZAcc<float, float> {  // FP32 inner solves: plain FP32 sums
  float a = 0.f;
  __device__ __forceinline__ void add(float w, float z) { a = fmaf(w, z, a); }
  __device__ __forceinline__ float get() const { return a; }
};

// Preconditioned-solve SpMVs with the operand B v = z + kap (pressure, one
// right side, staged tiles when K > 0):
//   y = A z + kap (A 1) + es mu,   mu = rank-one sum of B v (sc->sum_p / sum_s)
// WHICH = 0: v = A p^, reduce (rh, v) -> alpha;  WHICH = 1: t = A s^, reduce
// (t, s), (t, t) -> omega.
// op.diff (the FP32 rows of the MIXED inner solves): A z = sum_s w_s (z_j - z_i)
// + a1_i z_i with a1 the FP64 row sums.  Summed directly, FP32 rows of a
// Laplacian misrepresent the smooth modes: the row sum of the rounded weights
// is off by about eps32 times the largest weight, against an eigenvalue of
// order h^2 times it (a relative error near 6 % at 1M nodes).  In difference
// form a constant operand gives exactly a1_i z_i, and the rounding of each
// term scales with the differences, smaller by a factor h.  (On the 1M cavity
// the MIXED step measured the same either way.)
template <int K, typename TW, typename TV, int WHICH, int DIRECT = 0>
__global__ void __launch_bounds__(kThreads, DIRECT ? DIRECT : 1)
    k_spmv_pc(KOp<TW, TV> op, const TV* __restrict__ z, TV* __restrict__ y,
              const TV* __restrict__ dotv, KScal* sc, GridReduce gr, int* worked) {
  if (sc->done) return;
  // profiling: mark that this launch did the work its events bracket
  if (worked && blockIdx.x == 0 && threadIdx.x == 0) *worked = 1;
  constexpr int NU_ = 2;
  __shared__ double sh[NU_ * kThreads];
  const TV kap = (TV)sc->kap[WHICH];
  const TV sig = (TV)(WHICH ? sc->sum_s : sc->sum_p);
  TV d0 = 0, d1 = 0;
  // FP32 rows are always in difference form here (the plan sets op.diff
  // with a1 for every preconditioned FP32 operator); FP64 rows never are
  constexpr bool dif = std::is_same<TW, float>::value;
  auto finish_row = [&](int64_t i, TV acc, TV zi) {
    const TV yi = acc + (dif ? zi + kap : kap) * op.a1[i] + op.es[i] * sig;
    y[i] = yi;
    const TV di = dotv[i];  // rh for WHICH 0, s for WHICH 1
    d0 += di * yi;
    if (WHICH) d1 += yi * yi;
  };
  if constexpr (kStage<K, TW> && DIRECT == 0) {
    extern __shared__ __align__(128) unsigned char dsm[];
    auto* tile = reinterpret_cast<EllStage<K, TW>*>(dsm);
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const int64_t ntiles = (op.n + kTileRows - 1) / kTileRows;
    for (int64_t tix = blockIdx.x; tix < ntiles; tix += gridDim.x) {
      const int64_t row0 = tix * kTileRows;
      if (!stage_tile<K, TW>(tile, &bar, phase, op.idx, op.w, op.ld, row0, &sc->stage_err,
                             op.tiles))
        break;
      const int64_t i = row0 + threadIdx.x;
      if (i < op.n) {
        ZAcc<TW, TV> acc;
        const TV zi = dif ? z[i] : (TV)0;
#pragma unroll
        for (int q = 0; q < K; ++q)
          acc.add(tile->w[q * kTileRows + threadIdx.x],
                  z[tile->idx[q * kTileRows + threadIdx.x]] - zi);
        finish_row(i, (TV)acc.get(), zi);
      }
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < op.n;
         i += (int64_t)gridDim.x * kThreads) {
      ZAcc<TW, TV> acc;
      const int kk = K > 0 ? K : op.k;
      const TV zi = dif ? z[i] : (TV)0;
#pragma unroll(K > 0 ? K : 1)
      for (int q = 0; q < kk; ++q) {
        RBFFD_CHECK(op.idx[q * op.ld + i], op.n, 2, i);
        acc.add(op.w[q * op.ld + i], z[op.idx[q * op.ld + i]] - zi);
      }
      finish_row(i, (TV)acc.get(), zi);
    }
  }
  double vv[NU_] = {(double)d0, (double)d1};
  grid_reduce<NU_>(vv, gr, sh, [&](double* t) {
    if (sc->stage_err) sc->done = 1;
    if (!sc->active[0]) return;
    if (WHICH == 0) {
      const double rv = t[0];
      if (rv == 0.0 || !isfinite(rv)) {
        sc->active[0] = 0;
        sc->status = isfinite(rv) ? 1 : 2;
        return;
      }
      sc->alpha[0] = sc->rho[0] / rv;
    } else {
      if (sc->half[0]) return;
      const double ts = t[0], t2 = t[1];
      if (!(t2 > 0.0) || !isfinite(ts)) {
        sc->omega[0] = 0.0;
        sc->active[0] = 0;
        sc->status = isfinite(t2) ? 3 : 2;
        return;
      }
      sc->omega[0] = ts / t2;
    }
  });
}

// x += alpha (zp + kap_p) + omega (zs + kap_s) ; r = s - omega t ; reduce (rh, r), (r, r)
template <typename TV>
__global__ void __launch_bounds__(kThreads)
    k_update_xr_pc(int64_t n, TV* __restrict__ x, TV* __restrict__ r, const TV* __restrict__ rh,
                   const TV* __restrict__ zp, const TV* __restrict__ zs,
                   const TV* __restrict__ s, const TV* __restrict__ t, KScal* sc, GridReduce gr) {
  if (sc->done) return;
  constexpr int NU_ = 2;
  __shared__ double sh[NU_ * kThreads];
  const TV al = (TV)sc->alpha[0], om = (TV)sc->omega[0];
  const TV kp = (TV)sc->kap[0], ks = (TV)sc->kap[1];
  const int act = sc->active[0], hf = sc->half[0];
  TV prh = 0, prr = 0;
  if (act) {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads) {
      const TV si = s[i];
      TV ri;
      if (hf) {
        x[i] += al * ((TV)zp[i] + kp);
        ri = si;
      } else {
        x[i] += al * ((TV)zp[i] + kp) + om * ((TV)zs[i] + ks);
        ri = si - om * t[i];
      }
      r[i] = ri;
      prh += rh[i] * ri;
      prr += ri * ri;
    }
  }
  double vv[NU_] = {(double)prh, (double)prr};
  grid_reduce<NU_>(vv, gr, sh, [&](double* tt) {
    sc->iters += 1;
    if (!sc->active[0]) {
      sc->done = 1;
      return;
    }
    const double rho_new = tt[0], rr = tt[1];
    sc->rr[0] = rr;
    bool go = false;
    if (!isfinite(rr)) {
      sc->status = 2;
      sc->active[0] = 0;
    } else if (rr > 1e8 * sc->bb[0] && sc->bb[0] > 0.0) {
      sc->status = 5;
      sc->active[0] = 0;
    } else if (sc->half[0] || rr <= sc->tol2 * sc->bb[0]) {
      sc->active[0] = 0;
    } else if (rho_new == 0.0 || sc->omega[0] == 0.0) {
      sc->status = 4;
      sc->active[0] = 0;
    } else {
      sc->beta[0] = (rho_new / sc->rho[0]) * (sc->alpha[0] / sc->omega[0]);
      sc->rho[0] = rho_new;
      go = true;
    }
    if (!go || sc->iters >= sc->maxit) sc->done = 1;
  });
}

// Resumes a preconditioned solve whose right side was replaced between
// refinement sweeps, keeping its Krylov directions: r = b (the new normalised
// FP64 residual), x = 0, and beta from (rh, r) and the previous iteration's
// rho, alpha, omega.  s = (old residual norm) / (new residual norm) carries
// the old scale to the new one: p and v scale by s, so beta is stored times s
// and k_update_p forms p = r + beta s (p - omega v) unchanged.  A zero (rh, r)
// ends the call as a breakdown (status 4), which restarts the method.
template <typename TV>
__global__ void __launch_bounds__(kThreads)
    k_resume(int64_t n, const TV* __restrict__ b, TV* __restrict__ r, TV* __restrict__ x,
             const TV* __restrict__ rh, KScal* sc, GridReduce gr, double s, double tol2,
             int maxit) {
  constexpr int NU_ = 2;
  __shared__ double sh[NU_ * kThreads];
  TV prh = 0, prr = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const TV bi = b[i];
    r[i] = bi;
    x[i] = 0;
    prh += rh[i] * bi;
    prr += bi * bi;
  }
  double vv[NU_] = {(double)prh, (double)prr};
  grid_reduce<NU_>(vv, gr, sh, [&](double* t) {
    const double rho_new = t[0], rr = t[1], rho_old = sc->rho[0] * s;
    sc->tol2 = tol2;
    sc->maxit = maxit;
    sc->iters = 0;
    sc->status = 0;
    sc->stage_err = 0;
    sc->rr[0] = rr;
    sc->bb[0] = rr;
    sc->half[0] = 0;
    sc->active[1] = 0;
    const bool ok = isfinite(rr) && rho_new != 0.0 && rho_old != 0.0 && sc->omega[0] != 0.0;
    if (!ok) sc->status = isfinite(rr) ? 4 : 2;
    sc->active[0] = (ok && rr > 0.0) ? 1 : 0;
    if (ok) {
      sc->beta[0] = (rho_new / rho_old) * (sc->alpha[0] / sc->omega[0]) * s;
      sc->rho[0] = rho_new;
    }
    sc->done = (sc->active[0] && maxit > 0) ? 0 : 1;
  });
}

// row sums of an ELL operator in FP64 (A 1)
template <typename TW>
__global__ void k_rowsum(int64_t n, int64_t ld, int k, const TW* __restrict__ w,
                         double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < k; ++q) a += (double)w[q * ld + i];
    out[i] = a;
  }
}

// ------------------------------------------------- refinement helper kernels
// r = b - A x in FP64 (scaled system); reduce (r, r), (b, b) per right side
template <int K, int NRHS, bool RANK1>
__global__ void __launch_bounds__(kThreads)
    k_residual64(KOp<double, double> op, Vecs<double, NRHS> x, Vecs<double, NRHS> b,
                 Vecs<double, NRHS> r, const double* sigma_x, double* out4, GridReduce gr) {
  constexpr int NU_ = 2 * NRHS;
  __shared__ double sh[NU_ * kThreads];
  const double sig = RANK1 ? *sigma_x : 0.0;
  double prr[2] = {0, 0}, pbb[2] = {0, 0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < op.n;
       i += (int64_t)gridDim.x * kThreads) {
    double acc[NRHS];
    gather_rows<K, NRHS>(op, i, (const double* const*)x.v, acc);
#pragma unroll
    for (int q = 0; q < NRHS; ++q) {
      double ax = acc[q];
      if (op.diag1) ax += x.v[q][i];
      if (RANK1) ax += op.es[i] * sig;
      const double bi = b.v[q][i], ri = bi - ax;
      r.v[q][i] = ri;
      prr[q] += ri * ri;
      pbb[q] += bi * bi;
    }
  }
  double vv[NU_];
#pragma unroll
  for (int q = 0; q < NRHS; ++q) {
    vv[2 * q] = prr[q];
    vv[2 * q + 1] = pbb[q];
  }
  grid_reduce<NU_>(vv, gr, sh, [&](double* t) {
    for (int j = 0; j < NU_; ++j) out4[j] = t[j];
  });
}

// r32 = r64 * inv_norm ; e32 = 0
template <int NRHS>
__global__ void k_to32(int64_t n, Vecs<double, NRHS> r, Vecs<float, NRHS> r32,
                       Vecs<float, NRHS> e32, double inv0, double inv1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    r32.v[0][i] = (float)(r.v[0][i] * inv0);
    e32.v[0][i] = 0.f;
    if (NRHS > 1) {
      r32.v[NRHS - 1][i] = (float)(r.v[NRHS - 1][i] * inv1);
      e32.v[NRHS - 1][i] = 0.f;
    }
  }
}

// x64 += nrm * e32
template <int NRHS>
__global__ void k_addcorr(int64_t n, Vecs<double, NRHS> x, Vecs<float, NRHS> e32, double n0,
                          double n1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x.v[0][i] += n0 * (double)e32.v[0][i];
    if (NRHS > 1) x.v[NRHS - 1][i] += n1 * (double)e32.v[NRHS - 1][i];
  }
}

// Initial guess of a pressure solve by polynomial extrapolation in time
// through the last ord + 1 solutions: x holds the newest, h[0..] the older
// ones (newest first), and x <- sum_k (-1)^k C(ord + 1, k + 1) x_{j-k}
// (ord 1: 2 x - h0; ord 2: 3 x - 3 h0 + h1; ord 3: 4 x - 6 h0 + 4 h1 - h2;
// error O(dt^(ord+1)) for a smooth solution).  The old x goes to the oldest
// slot h[kMaxHist - 1], which the caller then takes as the newest.
constexpr int kMaxHist = 3;  // cubic: measured best on the 1M cavity (8.9 iterations per
                             // FP64 solve against 14.6 quadratic, 9.3 quartic, 10.2 quintic)
struct History {
  double* h[kMaxHist];
};
__global__ void k_extrapolate(int64_t n, int ord, double* __restrict__ x, History H) {
  double c[kMaxHist + 1];
  double b = ord + 1.0;  // C(ord + 1, k + 1) with alternating signs
  for (int k = 0; k <= ord; ++k) {
    c[k] = (k & 1) ? -b : b;
    b = b * (ord - k) / (k + 2.0);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t0 = x[i];
    double y = c[0] * t0;
    for (int k = 1; k <= ord; ++k) y += c[k] * H.h[k - 1][i];
    x[i] = y;
    H.h[kMaxHist - 1][i] = t0;
  }
}

__global__ void k_split(int64_t n, const double* __restrict__ x, float2* __restrict__ x2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x2[i] = split2(x[i]);
}

// ------------------------------------------------------- explicit stages
// sum_s w[s][i] * f(x[idx[s][i]]) for FP64 (plain) or FP32 (split differences)
template <int K, bool MIX, int NV>
struct Gather;

template <int K, int NV>
struct Gather<K, false, NV> {
  // NV operators (weights w[o]) applied to one vector x
  __device__ __forceinline__ static void run(const int32_t* idx, const void* const* w, int64_t ld,
                                             int k_rt, int64_t i, const double* x,
                                             const float2*, double* out) {
    const int k = K > 0 ? K : k_rt;
#pragma unroll
    for (int o = 0; o < NV; ++o) out[o] = 0.0;
#pragma unroll(K > 0 ? K : 1)
    for (int s = 0; s < k; ++s) {
      const double xj = x[idx[s * ld + i]];
#pragma unroll
      for (int o = 0; o < NV; ++o) out[o] += ((const double*)w[o])[s * ld + i] * xj;
    }
  }
};

template <int K, int NV>
struct Gather<K, true, NV> {
  __device__ __forceinline__ static void run(const int32_t* idx, const void* const* w, int64_t ld,
                                             int k_rt, int64_t i, const double*, const float2* x2,
                                             double* out) {
    const int k = K > 0 ? K : k_rt;
    float acc[NV];
#pragma unroll
    for (int o = 0; o < NV; ++o) acc[o] = 0.f;
    const float2 ref = x2[idx[i]];
#pragma unroll(K > 0 ? K : 1)
    for (int s = 0; s < k; ++s) {
      const float2 xj = x2[idx[s * ld + i]];
      const float d = (xj.x - ref.x) + (xj.y - ref.y);
#pragma unroll
      for (int o = 0; o < NV; ++o) acc[o] += ((const float*)w[o])[s * ld + i] * d;
    }
#pragma unroll
    for (int o = 0; o < NV; ++o) out[o] = (double)acc[o];
  }
};

struct ConvArgs {
  int64_t n, ld;
  int k;
  const int32_t* idx;
  const void *wdx, *wdy;
  const double *u, *v;
  const float2 *u2, *v2;
  double *cu_prev, *cv_prev, *us, *vs;
  float2 *us2, *vs2;
  double dt;
  int first;
};

// Stage 1: C_j(q) = -[u o D_x q + v o D_y q]; u* = u_j + dt (3/2 C_j - 1/2 C_{j-1})
template <int K, bool MIX>
__global__ void __launch_bounds__(kThreads) k_convect(ConvArgs a) {
  const void* w[2] = {a.wdx, a.wdy};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kThreads) {
    double du[2], dv[2];
    Gather<K, MIX, 2>::run(a.idx, w, a.ld, a.k, i, a.u, a.u2, du);
    Gather<K, MIX, 2>::run(a.idx, w, a.ld, a.k, i, a.v, a.v2, dv);
    const double ui = a.u[i], vi = a.v[i];
    const double cu = -(ui * du[0] + vi * du[1]);
    const double cv = -(ui * dv[0] + vi * dv[1]);
    const double cup = a.first ? cu : a.cu_prev[i];
    const double cvp = a.first ? cv : a.cv_prev[i];
    const double us = ui + a.dt * (1.5 * cu - 0.5 * cup);
    const double vs = vi + a.dt * (1.5 * cv - 0.5 * cvp);
    a.us[i] = us;
    a.vs[i] = vs;
    a.cu_prev[i] = cu;
    a.cv_prev[i] = cv;
    if (MIX) {
      a.us2[i] = split2(us);
      a.vs2[i] = split2(vs);
    }
  }
}

struct HelmRhsArgs {
  int64_t n, ld_v;
  int k;
  const int32_t* vv_idx;
  const void* lap;
  const double *us, *vs;
  const float2 *us2, *vs2;
  const int32_t* vp_idx;
  const void *vp_dx, *vp_dy;
  const double* pt;
  const float2* pt2;
  const uint8_t* v_bc;
  const double *v_nx, *v_ny, *gu, *gv;
  double a, dt;
  int km;
  double *ru, *rv, *xu, *xv;
  const double *u, *v;  // u_j, v_j (the Kim & Moin Crank-Nicolson form)
  const float2 *u2, *v2;
  int cn;    // RBFFD_CN_*
  int proj;  // RBFFD_PROJ_*
  const uint8_t *bcu, *bcv;  // open flows: per-component conditions (null: v_bc for both)
  // Initial guess of the viscous solves: vord < 0: the right side; else the
  // extrapolation of order vord through the previous solution (in xu, xv)
  // and the older ones in hu, hv (newest first), coefficients vc; the
  // previous solution then goes to the oldest slot.  Rows with a Dirichlet
  // condition start from their data.
  int vord = -1;
  double vc[kMaxHist + 1] = {};
  double* hu[kMaxHist] = {};
  double* hv[kMaxHist] = {};
};

// Stage 2 right side: u* + a D_Lap (u* or u_j) inside, minus dt G0 p~_j for
// the exact projection; wall rows: the wall data plus, for the paper's
// projection, the Kim & Moin term
template <int K, bool MIX>
__global__ void __launch_bounds__(kThreads) k_helm_rhs(HelmRhsArgs a) {
  const void* wl[1] = {a.lap};
  const void* wg[2] = {a.vp_dx, a.vp_dy};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kThreads) {
    double bu, bv;
    if (!a.v_bc[i]) {
      double lu, lv;
      const double* qu = a.cn ? a.u : a.us;
      const double* qv = a.cn ? a.v : a.vs;
      Gather<K, MIX, 1>::run(a.vv_idx, wl, a.ld_v, a.k, i, qu, a.cn ? a.u2 : a.us2, &lu);
      Gather<K, MIX, 1>::run(a.vv_idx, wl, a.ld_v, a.k, i, qv, a.cn ? a.v2 : a.vs2, &lv);
      bu = a.us[i] + a.a * lu;
      bv = a.vs[i] + a.a * lv;
      if (a.proj) {
        double g[2];
        Gather<K, MIX, 2>::run(a.vp_idx, wg, a.ld_v, a.k, i, a.pt, a.pt2, g);
        bu -= a.dt * g[0];
        bv -= a.dt * g[1];
      }
    } else if (a.bcu) {  // open flow: Dirichlet rows take the data, Neumann rows 0
      const bool du = a.bcu[i] == RBFFD_BC_DIRICHLET, dv = a.bcv[i] == RBFFD_BC_DIRICHLET;
      double g[2] = {0.0, 0.0};
      if (a.km && (du || dv)) Gather<K, MIX, 2>::run(a.vp_idx, wg, a.ld_v, a.k, i, a.pt, a.pt2, g);
      bu = du ? a.gu[i] + a.dt * g[0] : 0.0;
      bv = dv ? a.gv[i] + a.dt * g[1] : 0.0;
    } else {
      bu = a.gu[i];
      bv = a.gv[i];
      if (a.km && !a.proj) {
        double g[2];
        Gather<K, MIX, 2>::run(a.vp_idx, wg, a.ld_v, a.k, i, a.pt, a.pt2, g);
        if (a.km == 1) {
          const double tx = -a.v_ny[i], ty = a.v_nx[i];
          const double gt = tx * g[0] + ty * g[1];
          bu += a.dt * gt * tx;
          bv += a.dt * gt * ty;
        } else {
          bu += a.dt * g[0];
          bv += a.dt * g[1];
        }
      }
    }
    a.ru[i] = bu;
    a.rv[i] = bv;
    double xu = bu, xv = bv;
    if (a.vord >= 0) {
      const double pu = a.xu[i], pv = a.xv[i];
      const bool fu = a.bcu ? a.bcu[i] != RBFFD_BC_DIRICHLET : !a.v_bc[i];
      const bool fv = a.bcu ? a.bcv[i] != RBFFD_BC_DIRICHLET : !a.v_bc[i];
      if (fu) {
        xu = a.vc[0] * pu;
        for (int q = 1; q <= a.vord; ++q) xu += a.vc[q] * a.hu[q - 1][i];
      }
      if (fv) {
        xv = a.vc[0] * pv;
        for (int q = 1; q <= a.vord; ++q) xv += a.vc[q] * a.hv[q - 1][i];
      }
      a.hu[kMaxHist - 1][i] = pu;
      a.hv[kMaxHist - 1][i] = pv;
    }
    a.xu[i] = xu;
    a.xv[i] = xv;
  }
}

struct DivArgs {
  int64_t n, ld_p;
  int k;
  const int32_t* idx;
  const void *wdx, *wdy;
  const double *uss, *vss;
  const float2 *uss2, *vss2;
  const uint8_t* p_bc;
  const double* scale;
  double inv_dt;
  double* b;
  int proj;  // exact projection: every row is a divergence row
};

// Stage 3a: F = D^(P,V)_x u** + D^(P,V)_y v**; scaled Poisson right side
// (0 on the Neumann rows of the paper's projection)
template <int K, bool MIX>
__global__ void __launch_bounds__(kThreads) k_divergence(DivArgs a) {
  const void* wx[1] = {a.wdx};
  const void* wy[1] = {a.wdy};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kThreads) {
    double fx, fy;
    Gather<K, MIX, 1>::run(a.idx, wx, a.ld_p, a.k, i, a.uss, a.uss2, &fx);
    Gather<K, MIX, 1>::run(a.idx, wy, a.ld_p, a.k, i, a.vss, a.vss2, &fy);
    a.b[i] = (a.p_bc[i] && !a.proj) ? 0.0 : a.scale[i] * (fx + fy) * a.inv_dt;
  }
}

struct PresArgs {
  int64_t n, ld_p;
  int k;
  const int32_t* idx;
  const void* lap;
  const double* px;
  const float2* px2;
  const double* sum;
  double a;
  double *pt, *p;
  float2* pt2;
  int proj;
  int nomean;  // Dirichlet pressure rows: p~ = x, no shift to mean zero
};

// Stage 3c: p~ = x - mean(x); p = p~ - a D^(P,P)_Lap p~.  Exact projection:
// x - mean(x) is the increment phi, p~ += phi, p = p~ - a D^(P,P)_Lap phi
// (D_Lap annihilates constants, so it is applied to x).
template <int K, bool MIX>
__global__ void __launch_bounds__(kThreads) k_pressure(PresArgs a) {
  const void* wl[1] = {a.lap};
  const double mean = a.nomean ? 0.0 : *a.sum / (double)a.n;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kThreads) {
    double l;
    Gather<K, MIX, 1>::run(a.idx, wl, a.ld_p, a.k, i, a.px, a.px2, &l);
    const double pt = (a.proj ? a.pt[i] : 0.0) + (a.px[i] - mean);
    a.pt[i] = pt;
    a.p[i] = pt - a.a * l;
    if (MIX) a.pt2[i] = split2(pt);
  }
}

struct CorrArgs {
  int64_t n, ld_v;
  int k;
  const int32_t* idx;
  const void *wdx, *wdy;
  const double* pt;
  const float2* pt2;
  const double *uss, *vss;
  const uint8_t* v_bc;
  const double *gu, *gv;
  double dt;
  int overwrite;
  double *u, *v;
  float2 *u2, *v2;
  // exact projection: pt/pt2 hold x = phi + const, wall rows move by -c n with
  // c = -dt (sum x) / esn (the multiplier of the wall-flux column)
  int proj;
  const double *sum, *esn, *v_nx, *v_ny;
  const uint8_t *bcu, *bcv;  // open flows: only Dirichlet components are overwritten
};

// Stage 3d: u_{j+1} = u** - dt D^(V,P)_x p~ (Eq. velocity_next_timestep).
// Exact projection: u_{j+1} = u** - dt G0 phi - c w.
template <int K, bool MIX>
__global__ void __launch_bounds__(kThreads) k_correct(CorrArgs a) {
  const void* w[2] = {a.wdx, a.wdy};
  const double c = a.proj ? -a.dt * (*a.sum) / (*a.esn) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kThreads) {
    double un, vn;
    if (a.proj && a.v_bc[i]) {
      un = a.uss[i] - c * a.v_nx[i];
      vn = a.vss[i] - c * a.v_ny[i];
    } else {
      double g[2];
      Gather<K, MIX, 2>::run(a.idx, w, a.ld_v, a.k, i, a.pt, a.pt2, g);
      un = a.uss[i] - a.dt * g[0];
      vn = a.vss[i] - a.dt * g[1];
    }
    if (a.overwrite && !a.proj && a.v_bc[i]) {
      if (!a.bcu || a.bcu[i] == RBFFD_BC_DIRICHLET) un = a.gu[i];
      if (!a.bcv || a.bcv[i] == RBFFD_BC_DIRICHLET) vn = a.gv[i];
    }
    a.u[i] = un;
    a.v[i] = vn;
    if (MIX) {
      a.u2[i] = split2(un);
      a.v2[i] = split2(vn);
    }
  }
}

// --------------------------------------------------------------- set-up
// Row map of the one-sided Neumann operator: bmap[P-node] = its Neumann row.
// Rows outside [0, M) or repeated nodes raise the error flag.
__global__ void k_scatter_rows(int64_t nb, int64_t M, const int32_t* __restrict__ rows,
                               int32_t* __restrict__ bmap, int* __restrict__ err) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[b];
    if (r < 0 || r >= M) {
      atomicOr(err, 1);
      continue;
    }
    if (atomicCAS(&bmap[r], -1, (int32_t)b) != -1) atomicOr(err, 1);
  }
}

// Scaled pressure operator (see the file comment): Lidx/Lw = rows of L
// (interior: D^(P,P)_Lap on pp_idx; boundary: n_x D_x + n_y D_y on the
// one-sided stencil pn_idx), each divided by its diagonal; es = -S e.
__global__ void k_build_poisson(int64_t M, int64_t ld, int k, const int32_t* __restrict__ idx,
                                const double* __restrict__ lap, const uint8_t* __restrict__ p_bc,
                                const int32_t* __restrict__ bmap, int64_t ld_b,
                                const int32_t* __restrict__ pn_idx,
                                const double* __restrict__ pn_dx, const double* __restrict__ pn_dy,
                                const double* __restrict__ nx, const double* __restrict__ ny,
                                int32_t* __restrict__ Lidx, double* __restrict__ Lw,
                                double* __restrict__ es, double* __restrict__ scale,
                                int* __restrict__ err, int pdir) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (p_bc[i] == RBFFD_PBC_DIRICHLET) {  // p~ = 0: identity row, no rank-one entry
      for (int s = 0; s < k; ++s) {
        Lidx[s * ld + i] = (int32_t)i;
        Lw[s * ld + i] = s == 0 ? 1.0 : 0.0;
      }
      es[i] = 0.0;
      scale[i] = 1.0;
      continue;
    }
    const bool bnd = p_bc[i] != 0;
    const int32_t b = bnd ? bmap[i] : -1;
    if (bnd && b < 0) {  // a boundary node without a Neumann row
      atomicOr(err, 2);
      for (int s = 0; s < k; ++s) {
        Lidx[s * ld + i] = (int32_t)i;
        Lw[s * ld + i] = s == 0 ? 1.0 : 0.0;
      }
      es[i] = -1.0;
      scale[i] = 1.0;
      continue;
    }
    double diag = 0.0, sabs = 0.0;
    for (int s = 0; s < k; ++s) {
      int32_t c;
      double w;
      if (bnd) {
        c = pn_idx[s * ld_b + b];
        w = nx[i] * pn_dx[s * ld_b + b] + ny[i] * pn_dy[s * ld_b + b];
      } else {
        c = idx[s * ld + i];
        w = lap[s * ld + i];
      }
      sabs += fabs(w);
      if (c == (int32_t)i) diag += w;
      Lidx[s * ld + i] = c;
      Lw[s * ld + i] = w;
    }
    const double sc = diag != 0.0 ? 1.0 / diag : (sabs > 0.0 ? 1.0 / sabs : 1.0);
    for (int s = 0; s < k; ++s) Lw[s * ld + i] *= sc;
    es[i] = (bnd && !pdir) ? -sc : 0.0;  // with Dirichlet rows the system is nonsingular
    scale[i] = sc;
  }
}

// Composed pressure operator of the exact projection, L = D^(P,V) G0 (G0 =
// D^(V,P) with zero wall rows).  Row i merges, over the V-nodes v of its
// divergence stencil that are not on a wall, the products of its weights
// with the gradient stencil of v; columns appear in first-occurrence order
// (divergence slot, then gradient slot) and each weight is summed in that
// order, so the result does not depend on the launch.  Count pass (Lidx ==
// nullptr): count[i] = the row's distinct columns (kMaxComposed + 1 when it
// has more).  Build pass: width W (rows padded with (i, 0)), each row divided
// by its diagonal like the paper's operator, es = -S (D^(P,V) w)_i with w the
// wall normal at wall V-nodes (the wall-flux column); error bit 8 when a row
// does not fit.
constexpr int kMaxComposed = 128;

__global__ void __launch_bounds__(128)
    k_composed(int64_t M, int64_t ld_p, int k, const int32_t* __restrict__ pv_idx,
               const double* __restrict__ pv_dx, const double* __restrict__ pv_dy, int64_t ld_v,
               const int32_t* __restrict__ vp_idx, const double* __restrict__ vp_dx,
               const double* __restrict__ vp_dy, const uint8_t* __restrict__ v_bc,
               const double* __restrict__ v_nx, const double* __restrict__ v_ny, int W,
               int* __restrict__ count, int32_t* __restrict__ Lidx, double* __restrict__ Lw,
               double* __restrict__ es, double* __restrict__ scale, int* __restrict__ err) {
  int32_t cols[kMaxComposed];
  double ws[kMaxComposed];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    int nc = 0;
    bool over = false;
    double dw = 0.0;
    for (int s = 0; s < k; ++s) {
      const int32_t v = pv_idx[s * ld_p + i];
      RBFFD_CHECK(v, ld_v, 3, i);
      const double ax = pv_dx[s * ld_p + i], ay = pv_dy[s * ld_p + i];
      if (v_bc[v]) {
        dw += ax * v_nx[v] + ay * v_ny[v];
        continue;
      }
      for (int t = 0; t < k; ++t) {
        const int32_t c = vp_idx[t * ld_v + v];
        RBFFD_CHECK(c, M, 4, i);
        const double wt = ax * vp_dx[t * ld_v + v] + ay * vp_dy[t * ld_v + v];
        int q = 0;
        while (q < nc && cols[q] != c) ++q;
        if (q == nc) {
          if (nc == kMaxComposed) {
            over = true;
            continue;
          }
          cols[nc] = c;
          ws[nc] = 0.0;
          ++nc;
        }
        ws[q] += wt;
      }
    }
    if (!Lidx) {
      count[i] = over ? kMaxComposed + 1 : nc;
      continue;
    }
    if (over || nc > W) {
      atomicOr(err, 8);
      nc = 0;
    }
    double diag = 0.0, sabs = 0.0;
    for (int q = 0; q < nc; ++q) {
      if (cols[q] == (int32_t)i) diag += ws[q];
      sabs += fabs(ws[q]);
    }
    const double sc = diag != 0.0 ? 1.0 / diag : (sabs > 0.0 ? 1.0 / sabs : 1.0);
    for (int q = 0; q < W; ++q) {
      Lidx[q * ld_p + i] = q < nc ? cols[q] : (int32_t)i;
      Lw[q * ld_p + i] = q < nc ? ws[q] * sc : 0.0;
    }
    es[i] = -sc * dw;
    scale[i] = sc;
  }
}

__global__ void k_store_abs(const double* __restrict__ x, double* __restrict__ y) { *y = fabs(*x); }

// Viscous operator without its identity part: Hw = -a_i D_Lap
__global__ void k_build_helm(int64_t N, int64_t ld, int k, const double* __restrict__ lap,
                             const uint8_t* __restrict__ v_bc, double a, double* __restrict__ Hw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ai = v_bc[i] ? 0.0 : a;
    for (int s = 0; s < k; ++s) Hw[s * ld + i] = -ai * lap[s * ld + i];
  }
}

// Open flows (per-component conditions): the shared index array of the two
// viscous operators (the one-sided stencil of a Neumann V-row, the V->V
// stencil elsewhere) and, per component, Hw with x + Hw x = row i of H:
// interior -a D_Lap; Dirichlet 0 (identity row); Neumann N_i / N_ii - e_i,
// with N = v_nx D_x + v_ny D_y (the normalised Neumann row: its diagonal is
// the stencil's first slot, the node itself).
__global__ void k_build_hidx(int64_t N, int64_t ld, int k, const int32_t* __restrict__ vv_idx,
                             const int32_t* __restrict__ vmap, int64_t ld_b,
                             const int32_t* __restrict__ vn_idx, int32_t* __restrict__ Hidx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = vmap[i];
    for (int s = 0; s < k; ++s) Hidx[s * ld + i] = b >= 0 ? vn_idx[s * ld_b + b] : vv_idx[s * ld + i];
  }
}

__global__ void k_build_helm_open(int64_t N, int64_t ld, int k, const double* __restrict__ lap,
                                  const uint8_t* __restrict__ bc, const int32_t* __restrict__ vmap,
                                  int64_t ld_b, const double* __restrict__ vn_dx,
                                  const double* __restrict__ vn_dy, const double* __restrict__ nx,
                                  const double* __restrict__ ny, double a,
                                  double* __restrict__ Hw, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (bc[i] == RBFFD_BC_NEUMANN) {
      const int32_t b = vmap[i];
      if (b < 0) {  // a Neumann node without a Neumann row
        atomicOr(err, 16);
        for (int s = 0; s < k; ++s) Hw[s * ld + i] = 0.0;
        continue;
      }
      const double d = nx[i] * vn_dx[b] + ny[i] * vn_dy[b];  // slot 0: the node itself
      const double inv = d != 0.0 ? 1.0 / d : 0.0;
      if (!(d != 0.0)) atomicOr(err, 32);
      for (int s = 0; s < k; ++s) {
        const double w = nx[i] * vn_dx[s * ld_b + b] + ny[i] * vn_dy[s * ld_b + b];
        Hw[s * ld + i] = w * inv - (s == 0 ? 1.0 : 0.0);
      }
    } else {
      const double ai = bc[i] == RBFFD_BC_DIRICHLET ? 0.0 : a;
      for (int s = 0; s < k; ++s) Hw[s * ld + i] = -ai * lap[s * ld + i];
    }
  }
}

__global__ void k_count_eq(int64_t n, const uint8_t* __restrict__ x, uint8_t v, int* __restrict__ cnt) {
  int c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += x[i] == v;
  if (c) atomicAdd(cnt, c);
}

__global__ void k_scale_by_inv_abs(int64_t n, double* __restrict__ x, const double* sum) {
  const double s = *sum != 0.0 ? 1.0 / fabs(*sum) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

// diagonal of the scaled pressure operator (the sum of the slots on the row's own node)
__global__ void k_diag(int64_t M, int64_t ld, int k, const int32_t* __restrict__ idx,
                       const double* __restrict__ w, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < k; ++q)
      if (idx[q * ld + i] == (int32_t)i) s += w[q * ld + i];
    d[i] = s;
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

}  // namespace

// ------------------------------------------------------------------ plan
// Tile records of a slot-major ELL operator: record t holds idx[s][t*256 + r]
// and then w[s][t*256 + r] for s < k, r < 256 (rows past ld: index 0,
// weight 0), which is the layout of one EllStage.
template <typename TW>
__global__ void __launch_bounds__(kThreads)
    k_tile_records(int64_t ld, int k, int64_t ntiles, const int32_t* __restrict__ idx,
                   const TW* __restrict__ w, unsigned char* __restrict__ out) {
  const int64_t per = (int64_t)k * kTileRows;
  const int64_t rec = per * (int64_t)(sizeof(int32_t) + sizeof(TW));
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < ntiles * per;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t t = e / per, rem = e - t * per;
    const int64_t s = rem / kTileRows, row = t * kTileRows + (rem - s * kTileRows);
    const bool in = row < ld;
    reinterpret_cast<int32_t*>(out + t * rec)[rem] = in ? idx[s * ld + row] : 0;
    reinterpret_cast<TW*>(out + t * rec + per * (int64_t)sizeof(int32_t))[rem] =
        in ? w[s * ld + row] : (TW)0;
  }
}

struct StepPlan {
  rbffd_flow key;
  int k = 0;
  int kL = 0;         // row width of the pressure operator (k, or the composed width)
  int proj = 0;       // RBFFD_PROJ_*
  double* esn = nullptr;  // |sum of the raw rank-one column| (exact projection's multiplier scale)
  double esn_h = 0.0;
  int64_t N = 0, M = 0;
  int grid = 0;
  bool mix = false;
  std::vector<void*> allocs;
  // derived operators
  int32_t* Lidx = nullptr;
  int32_t* bmap = nullptr;
  int* err = nullptr;
  double *Lw = nullptr, *es = nullptr, *scale = nullptr, *Hw = nullptr;
  float *Lw32 = nullptr, *es32 = nullptr, *Hw32 = nullptr;
  float *vv_dx32 = nullptr, *vv_dy32 = nullptr, *vv_lap32 = nullptr, *pp_lap32 = nullptr,
        *vp_dx32 = nullptr, *vp_dy32 = nullptr;
  // stage vectors
  double *us = nullptr, *vs = nullptr, *ru = nullptr, *rv = nullptr, *uss = nullptr,
         *vss = nullptr, *pb = nullptr, *px = nullptr;
  int64_t px_step = -1;  // step index whose pressure solve left its solution in px
  // the pressure solutions of the steps before px's, newest first; the first
  // nhist of them are those of consecutive steps
  double* pxh[kMaxHist] = {};
  int nhist = 0;
  // the viscous solutions (u**, v**) of the steps before, as a ring like pxh
  double* vhu[kMaxHist] = {};
  double* vhv[kMaxHist] = {};
  int vhist = 0, vhead = 0;
  int hhead = 0;  // pxh[hhead] is the newest, then pxh[hhead + 1], ... (mod kMaxHist)
  float2 *u2 = nullptr, *v2 = nullptr, *us2 = nullptr, *vs2 = nullptr, *uss2 = nullptr,
         *vss2 = nullptr, *pt2 = nullptr, *px2 = nullptr;
  // Krylov work (6 vectors x 2 right sides) in FP64 and FP32
  double* kw64[7][2] = {};
  float* kw32[7][2] = {};
  float *e32[2] = {}, *r32[2] = {};
  double* r64[2] = {};
  KScal* sc = nullptr;
  double* dscal = nullptr;  // [0]: sum, [1..6]: residual norms
  struct AdjointPlan* adj = nullptr;  // transposed operators, built on first use
  Amg* amg = nullptr;                 // pressure preconditioner (precond = 1)
  double* a1 = nullptr;    // row sums of the FP64 pressure operator
  float* a1_32 = nullptr;  // the same in FP32 (complement of the difference-form FP32 rows)
  // tile records of the pressure and viscous operators the Krylov solves
  // apply (FP32 weights in MIXED precision, FP64 otherwise)
  unsigned char* Lt = nullptr;
  unsigned char* Ht = nullptr;
  // open flows (per-component velocity conditions): the viscous operators'
  // shared index array and v's own operator (Hw, Hw32, Ht serve u); pdir:
  // the pressure system has Dirichlet rows (nonsingular, no mean removal)
  bool open = false;
  int pdir = 0;
  int32_t* Hidx = nullptr;
  double* Hw_v = nullptr;
  float* Hw32_v = nullptr;
  unsigned char* Ht_v = nullptr;
  // CUDA graphs of Krylov iteration chunks: one per solve (its operator,
  // vectors and preconditioner) and chunk length, captured on first use on a
  // private stream and replayed on the caller's stream
  struct Graph {
    const void* key[10];
    int n;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;
  int64_t launches = 0;     // kernels launched by rbffd_step on this plan
  // optional per-launch timing of the pressure-solve SpMV kernels
  static constexpr int kEv = 512;
  cudaEvent_t ev[kEv] = {};
  int* evwork = nullptr;  // [kEv / 2] did-work flags of the profiled launches
  int ev_used = 0;
  double spmv_ms = 0.0;
  int64_t spmv_launches = 0;
  double spmv_batch_ms = 0.0;  // back-to-back SpMV launches of profiled solves
  int64_t spmv_batch_launches = 0;
  double vspmv_batch_ms = 0.0;  // the same for the viscous SpMV (two right sides)
  int64_t vspmv_batch_launches = 0;
  KScal* sc_timing = nullptr;
  GridReduce gr{};
};

void adjoint_plan_free(struct AdjointPlan* a);

void step_plan_free(StepPlan* p) {
  if (!p) return;
  adjoint_plan_free(p->adj);
  amg_free(p->amg);
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  for (int i = 0; i < StepPlan::kEv; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

namespace {

template <typename T>
int palloc(rbffd_ctx* ctx, StepPlan* p, T** out, size_t count) {
  void* ptr = nullptr;
  int rc = check_cuda(ctx, cudaMalloc(&ptr, sizeof(T) * (count > 0 ? count : 1)), "plan alloc");
  if (rc) return rc;
  p->allocs.push_back(ptr);
  *out = (T*)ptr;
  return RBFFD_OK;
}

int to32(rbffd_ctx* ctx, StepPlan* p, const double* src, int64_t n, float** dst,
         cudaStream_t st) {
  int rc = palloc(ctx, p, dst, n);
  if (rc) return rc;
  k_to_f32<<<p->grid, kThreads, 0, st>>>(n, src, *dst);
  return check_cuda(ctx, cudaGetLastError(), "to_f32");
}

// The fields a plan is built from: solver controls (tolerances, iteration
// cap, boundary modes, profiling) are read per call and do not key the plan.
rbffd_flow plan_key(const rbffd_flow& f) {
  rbffd_flow k = f;
  k.tol = k.inner_tol = 0.0;
  k.max_iter = k.km_mode = k.overwrite_bc = k.profile = k.cn_form = 0;
  return k;
}

int build_plan(rbffd_ctx* ctx, const rbffd_flow& f, StepPlan** out, cudaStream_t st) {
  StepPlan* p = new StepPlan();
  p->key = plan_key(f);
  p->k = ctx->prm.n;
  p->N = f.N;
  p->M = f.M;
  p->mix = f.precision == RBFFD_PREC_MIXED;
  p->grid = sm_count() * 8;  // 8 blocks of 256 per SM: full occupancy at 32 registers
  p->proj = f.projection;
  p->open = f.v_bcu != nullptr;
  p->kL = p->k;
  const int64_t nv = f.ld_v * p->k;
  const int64_t nmax = f.N > f.M ? f.N : f.M;
  int rc = 0;
#define TRY(x)                   \
  do {                           \
    rc = (x);                    \
    if (rc) {                    \
      step_plan_free(p);         \
      return rc;                 \
    }                            \
  } while (0)
  if (p->proj) {
    // width of the composed operator: the longest merged row
    int* cnt = nullptr;
    TRY(palloc(ctx, p, &cnt, f.M));
    k_composed<<<p->grid, 128, 0, st>>>(f.M, f.ld_p, p->k, f.pv_idx, f.pv_dx, f.pv_dy, f.ld_v,
                                        f.vp_idx, f.vp_dx, f.vp_dy, f.v_bc, f.v_nx, f.v_ny, 0,
                                        cnt, nullptr, nullptr, nullptr, nullptr, nullptr);
    TRY(check_cuda(ctx, cudaGetLastError(), "composed operator count"));
    std::vector<int> hc(f.M);
    TRY(check_cuda(ctx, cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * f.M,
                                        cudaMemcpyDeviceToHost, st), "count copy"));
    TRY(check_cuda(ctx, cudaStreamSynchronize(st), "count sync"));
    int W = 1;
    for (int c : hc) W = c > W ? c : W;
    if (W > kMaxComposed) {
      step_plan_free(p);
      return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                       "composed pressure operator has a row wider than %d entries", kMaxComposed);
    }
    p->kL = W;
  }
  const int64_t np = f.ld_p * p->kL;
  TRY(palloc(ctx, p, &p->Lw, np));
  TRY(palloc(ctx, p, &p->Lidx, np));
  TRY(palloc(ctx, p, &p->esn, 1));
  TRY(palloc(ctx, p, &p->bmap, f.M));
  TRY(palloc(ctx, p, &p->err, 1));
  TRY(palloc(ctx, p, &p->es, f.M));
  TRY(palloc(ctx, p, &p->scale, f.M));
  TRY(palloc(ctx, p, &p->Hw, nv));
  TRY(palloc(ctx, p, &p->us, f.N));
  TRY(palloc(ctx, p, &p->vs, f.N));
  TRY(palloc(ctx, p, &p->ru, f.N));
  TRY(palloc(ctx, p, &p->rv, f.N));
  TRY(palloc(ctx, p, &p->uss, f.N));
  TRY(palloc(ctx, p, &p->vss, f.N));
  TRY(palloc(ctx, p, &p->pb, f.M));
  TRY(palloc(ctx, p, &p->px, f.M));
  for (int q = 0; q < kMaxHist; ++q) {
    TRY(palloc(ctx, p, &p->pxh[q], f.M));
    TRY(palloc(ctx, p, &p->vhu[q], f.N));
    TRY(palloc(ctx, p, &p->vhv[q], f.N));
  }
  for (int a = 0; a < 7; ++a)
    for (int b = 0; b < 2; ++b) TRY(palloc(ctx, p, &p->kw64[a][b], nmax));
  TRY(palloc(ctx, p, &p->sc, 1));
  TRY(palloc(ctx, p, &p->dscal, 8));
  TRY(palloc(ctx, p, &p->gr.partials, (size_t)p->grid * kNV));
  TRY(palloc(ctx, p, &p->gr.counter, 1));
  TRY(check_cuda(ctx, cudaMemsetAsync(p->gr.counter, 0, sizeof(unsigned int), st), "memset"));
  const double a = f.dt / (2.0 * f.Re);
  TRY(check_cuda(ctx, cudaMemsetAsync(p->err, 0, sizeof(int), st), "memset"));
  TRY(check_cuda(ctx, cudaMemsetAsync(p->bmap, 0xff, sizeof(int32_t) * f.M, st), "memset"));
  if (p->proj) {
    k_composed<<<p->grid, 128, 0, st>>>(f.M, f.ld_p, p->k, f.pv_idx, f.pv_dx, f.pv_dy, f.ld_v,
                                        f.vp_idx, f.vp_dx, f.vp_dy, f.v_bc, f.v_nx, f.v_ny,
                                        p->kL, nullptr, p->Lidx, p->Lw, p->es, p->scale, p->err);
  } else {
    // Dirichlet pressure rows (open flows): counted first, since any one of
    // them removes the rank-one column from every row
    int* dcnt = nullptr;
    TRY(palloc(ctx, p, &dcnt, 1));
    TRY(check_cuda(ctx, cudaMemsetAsync(dcnt, 0, sizeof(int), st), "memset"));
    k_count_eq<<<p->grid, kThreads, 0, st>>>(f.M, f.p_bc, (uint8_t)RBFFD_PBC_DIRICHLET, dcnt);
    TRY(check_cuda(ctx, cudaMemcpyAsync(&p->pdir, dcnt, sizeof(int), cudaMemcpyDeviceToHost, st),
                   "Dirichlet rows"));
    TRY(check_cuda(ctx, cudaStreamSynchronize(st), "Dirichlet rows"));
    k_scatter_rows<<<p->grid, kThreads, 0, st>>>(f.nb_p, f.M, f.pn_rows, p->bmap, p->err);
    k_build_poisson<<<p->grid, kThreads, 0, st>>>(f.M, f.ld_p, p->k, f.pp_idx, f.pp_lap, f.p_bc,
                                                   p->bmap, f.ld_b, f.pn_idx, f.pn_dx, f.pn_dy,
                                                   f.p_nx, f.p_ny, p->Lidx, p->Lw, p->es,
                                                   p->scale, p->err, p->pdir > 0 ? 1 : 0);
  }
  // normalise the rank-one column so that the constant mode has eigenvalue 1
  k_sum<double><<<p->grid, kThreads, 0, st>>>(p->es, f.M, p->gr, p->dscal);
  k_store_abs<<<1, 1, 0, st>>>(p->dscal, p->esn);
  k_scale_by_inv_abs<<<p->grid, kThreads, 0, st>>>(f.M, p->es, p->dscal);
  if (p->open) {
    int32_t* vmap = nullptr;
    TRY(palloc(ctx, p, &vmap, f.N));
    TRY(palloc(ctx, p, &p->Hidx, nv));
    TRY(palloc(ctx, p, &p->Hw_v, nv));
    TRY(check_cuda(ctx, cudaMemsetAsync(vmap, 0xff, sizeof(int32_t) * f.N, st), "memset"));
    k_scatter_rows<<<p->grid, kThreads, 0, st>>>(f.nb_v, f.N, f.vn_rows, vmap, p->err);
    k_build_hidx<<<p->grid, kThreads, 0, st>>>(f.N, f.ld_v, p->k, f.vv_idx, vmap, f.ld_vb,
                                               f.vn_idx, p->Hidx);
    k_build_helm_open<<<p->grid, kThreads, 0, st>>>(f.N, f.ld_v, p->k, f.vv_lap, f.v_bcu, vmap,
                                                    f.ld_vb, f.vn_dx, f.vn_dy, f.v_nx, f.v_ny, a,
                                                    p->Hw, p->err);
    k_build_helm_open<<<p->grid, kThreads, 0, st>>>(f.N, f.ld_v, p->k, f.vv_lap, f.v_bcv, vmap,
                                                    f.ld_vb, f.vn_dx, f.vn_dy, f.v_nx, f.v_ny, a,
                                                    p->Hw_v, p->err);
  } else {
    k_build_helm<<<p->grid, kThreads, 0, st>>>(f.N, f.ld_v, p->k, f.vv_lap, f.v_bc, a, p->Hw);
  }
  TRY(check_cuda(ctx, cudaGetLastError(), "plan kernels"));
  {
    int herr = 0;
    TRY(check_cuda(ctx, cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st),
                   "plan status"));
    TRY(check_cuda(ctx, cudaStreamSynchronize(st), "plan sync"));
    TRY(check_cuda(ctx, cudaMemcpy(&p->esn_h, p->esn, sizeof(double), cudaMemcpyDeviceToHost),
                   "rank-one scale"));
    if (herr) {
      step_plan_free(p);
      if (herr & 8)
        return set_error(ctx, RBFFD_ERR_INVALID_ARG, "composed pressure operator overflow");
      if (herr & 48)
        return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                         "Neumann V-rows (vn_rows) must list every Neumann V-node once, each with "
                         "a nonzero normal derivative weight on the node itself (code %d)", herr);
      return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                       "Neumann rows (pn_rows) must list every boundary P-node once (code %d)",
                       herr);
    }
    if (p->proj && !(p->esn_h > 0.0))
      return (step_plan_free(p),
              set_error(ctx, RBFFD_ERR_INVALID_ARG,
                        "exact projection needs wall V-nodes with normals (v_bc, v_nx, v_ny)"));
  }
  if (f.precond) {
    // multigrid hierarchy of the P-node edge graph, scaled to the pressure rows
    std::vector<double> hd(f.M), hes(f.M);
    k_diag<<<p->grid, kThreads, 0, st>>>(f.M, f.ld_p, p->kL, p->Lidx, p->Lw, p->kw64[0][0]);
    TRY(check_cuda(ctx, cudaGetLastError(), "diagonal"));
    TRY(check_cuda(ctx, cudaMemcpyAsync(hd.data(), p->kw64[0][0], sizeof(double) * f.M,
                                        cudaMemcpyDeviceToHost, st),
                   "diagonal copy"));
    TRY(check_cuda(ctx, cudaMemcpyAsync(hes.data(), p->es, sizeof(double) * f.M,
                                        cudaMemcpyDeviceToHost, st),
                   "rank-one column copy"));
    TRY(check_cuda(ctx, cudaStreamSynchronize(st), "diagonal sync"));
    TRY(amg_build(ctx, f, hd.data(), hes.data(), &p->amg, st));
    TRY(palloc(ctx, p, &p->a1, f.M));
    k_rowsum<double><<<p->grid, kThreads, 0, st>>>(f.M, f.ld_p, p->kL, p->Lw, p->a1);
    TRY(check_cuda(ctx, cudaGetLastError(), "row sums"));
  }
  if (p->mix) {
    TRY(to32(ctx, p, p->Lw, np, &p->Lw32, st));
    // the FP32 pressure rows are applied in difference form with the FP64
    // row sums (near zero) as their diagonal complement (see k_spmv_pc)
    if (f.precond) TRY(to32(ctx, p, p->a1, f.M, &p->a1_32, st));
    TRY(to32(ctx, p, p->es, f.M, &p->es32, st));
    TRY(to32(ctx, p, p->Hw, nv, &p->Hw32, st));
    if (p->open) TRY(to32(ctx, p, p->Hw_v, nv, &p->Hw32_v, st));
    TRY(to32(ctx, p, f.vv_dx, nv, &p->vv_dx32, st));
    TRY(to32(ctx, p, f.vv_dy, nv, &p->vv_dy32, st));
    TRY(to32(ctx, p, f.vv_lap, nv, &p->vv_lap32, st));
    TRY(to32(ctx, p, f.pp_lap, f.ld_p * p->k, &p->pp_lap32, st));  // the caller's width
    TRY(to32(ctx, p, f.vp_dx, nv, &p->vp_dx32, st));
    TRY(to32(ctx, p, f.vp_dy, nv, &p->vp_dy32, st));
    TRY(palloc(ctx, p, &p->u2, f.N));
    TRY(palloc(ctx, p, &p->v2, f.N));
    TRY(palloc(ctx, p, &p->us2, f.N));
    TRY(palloc(ctx, p, &p->vs2, f.N));
    TRY(palloc(ctx, p, &p->uss2, f.N));
    TRY(palloc(ctx, p, &p->vss2, f.N));
    TRY(palloc(ctx, p, &p->pt2, f.M));
    TRY(palloc(ctx, p, &p->px2, f.M));
    for (int a2 = 0; a2 < 7; ++a2)
      for (int b = 0; b < 2; ++b) TRY(palloc(ctx, p, &p->kw32[a2][b], nmax));
    for (int b = 0; b < 2; ++b) {
      TRY(palloc(ctx, p, &p->e32[b], nmax));
      TRY(palloc(ctx, p, &p->r32[b], nmax));
      TRY(palloc(ctx, p, &p->r64[b], nmax));
    }
  }
  {
    const size_t wsz = p->mix ? sizeof(float) : sizeof(double);
    const size_t rec = (size_t)p->k * kTileRows * (sizeof(int32_t) + wsz);
    auto records = [&](int64_t rows, int64_t ld, const int32_t* idx, const double* w64,
                       const float* w32, unsigned char** out) -> int {
      const int64_t ntiles = (rows + kTileRows - 1) / kTileRows;
      int rc = palloc(ctx, p, out, rec * (size_t)ntiles);
      if (rc) return rc;
      if (p->mix)
        k_tile_records<float><<<p->grid, kThreads, 0, st>>>(ld, p->k, ntiles, idx, w32, *out);
      else
        k_tile_records<double><<<p->grid, kThreads, 0, st>>>(ld, p->k, ntiles, idx, w64, *out);
      return check_cuda(ctx, cudaGetLastError(), "tile records");
    };
    if (p->open) {
      TRY(records(f.N, f.ld_v, p->Hidx, p->Hw, p->Hw32, &p->Ht));
      TRY(records(f.N, f.ld_v, p->Hidx, p->Hw_v, p->Hw32_v, &p->Ht_v));
    } else {
      TRY(records(f.N, f.ld_v, f.vv_idx, p->Hw, p->Hw32, &p->Ht));
    }
    // the composed operator's width is not the staged tiles' k: its SpMVs
    // read rows directly
    if (f.precond && !p->proj) TRY(records(f.M, f.ld_p, p->Lidx, p->Lw, p->Lw32, &p->Lt));
  }
#undef TRY
  *out = p;
  return RBFFD_OK;
}

// ---------------------------------------------------------------- BiCGSTAB
struct SolveResult {
  int iters = 0;
  double relres = 0.0;
  int status = 0;  // as KScal::status
  bool converged = false;
  // a preconditioned solve that converged without breakdown on a full
  // iteration: k_resume can carry its directions to a new right side
  bool resumable = false;
};

// Add up the durations of the recorded SpMV launches (the stream is idle here).
// Only launches that did their work count (a launch issued after the solve
// converged returns at once and leaves its flag at 0).
void collect_events(StepPlan* P) {
  const int pairs = P->ev_used / 2;
  int flags[StepPlan::kEv / 2] = {};
  if (pairs > 0 &&
      cudaMemcpy(flags, P->evwork, sizeof(int) * pairs, cudaMemcpyDeviceToHost) == cudaSuccess) {
    for (int i = 0; i < pairs; ++i) {
      float ms = 0.f;
      if (flags[i] && cudaEventElapsedTime(&ms, P->ev[2 * i], P->ev[2 * i + 1]) == cudaSuccess) {
        P->spmv_ms += ms;
        P->spmv_launches += 1;
      }
    }
    cudaMemset(P->evwork, 0, sizeof(int) * pairs);
  }
  cudaGetLastError();  // a pair that could not be timed only goes uncounted
  P->ev_used = 0;
}

// The V-cycle results of p (which 0) and s (which 1) in the solve's precision.
template <typename TV>
TV* zbuf(const Amg* a, int which);
template <>
float* zbuf<float>(const Amg* a, int which) {
  return which ? a->zs : a->zp;
}
template <>
double* zbuf<double>(const Amg* a, int which) {
  return which ? a->zsd : a->zpd;
}

// B v = zout + kap[which] (one application of the multigrid preconditioner,
// 2 nlev launches)
template <typename TV>
void vcycle(StepPlan* P, const Amg* a, const TV* v, int which, TV* zout, cudaStream_t st) {
  const int G = P->grid;
  auto grid_for = [&](int64_t rows) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(G, (rows + kThreads - 1) / kThreads));
  };
  const int64_t n = a->lev[0].n;
  k_pc_in<TV><<<G, kThreads, 0, st>>>(n, v, a->c, a->ce, a->perm0, which, a->inv_ces, P->sc,
                                       a->lev[0].r);
  for (int l = 0; l + 1 < a->nlev; ++l) {
    const AmgLevel& F = a->lev[l];
    const int gb = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)G * 2, (a->lev[l + 1].n + kRB - 1) / kRB));
    if (a->rec[l]) {
      if (a->rec_w[l] == 8)
        k_pc_restrict_rec<8><<<gb, kThreads, 0, st>>>(F, a->rec_n[l], a->rec[l],
                                                      a->lev[l + 1].r, P->sc);
      else
        k_pc_restrict_rec<16><<<gb, kThreads, 0, st>>>(F, a->rec_n[l], a->rec[l],
                                                       a->lev[l + 1].r, P->sc);
      continue;
    }
    switch (width_bucket(F.width)) {
      case 8: k_pc_restrict<8><<<gb, kThreads, 0, st>>>(F, a->lev[l + 1].n, a->lev[l + 1].r, P->sc); break;
      case 16: k_pc_restrict<16><<<gb, kThreads, 0, st>>>(F, a->lev[l + 1].n, a->lev[l + 1].r, P->sc); break;
      case 32: k_pc_restrict<32><<<gb, kThreads, 0, st>>>(F, a->lev[l + 1].n, a->lev[l + 1].r, P->sc); break;
      default: k_pc_restrict<0><<<gb, kThreads, 0, st>>>(F, a->lev[l + 1].n, a->lev[l + 1].r, P->sc);
    }
  }
  const AmgLevel& C = a->lev[a->nlev - 1];
  const AmgLevel& Cf = a->lev[a->nlev >= 2 ? a->nlev - 2 : 0];
  k_pc_coarse<TV><<<grid_for(a->nc * 32), kThreads, 0, st>>>(a->nc, a->Xc, C.r, zout, Cf,
                                                             a->nlev >= 2 ? 1 : 0, P->sc);
  for (int l = a->nlev - 2; l >= 1; --l) {
    const AmgLevel& F = a->lev[l];
    if (a->rec[l]) {
      const int gbr = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)G * 2, a->rec_n[l]));
      if (a->rec_w[l] == 8)
        k_pc_up_rec<8><<<gbr, kThreads, 0, st>>>(F, a->lev[l - 1], a->rec_n[l], a->rec[l],
                                                 P->sc);
      else
        k_pc_up_rec<16><<<gbr, kThreads, 0, st>>>(F, a->lev[l - 1], a->rec_n[l], a->rec[l],
                                                  P->sc);
      continue;
    }
    const int gb = grid_for(F.n);
#define RBFFD_UP(Wb)                                                                         \
  k_pc_up<true, false, float, Wb><<<gb, kThreads, 0, st>>>(F, a->lev[l - 1], F.z, nullptr,   \
                                                           P->sc, P->gr, which, 0.0, 0.0)
    switch (width_bucket(F.width)) {
      case 8: RBFFD_UP(8); break;
      case 16: RBFFD_UP(16); break;
      case 32: RBFFD_UP(32); break;
      default: RBFFD_UP(0);
    }
#undef RBFFD_UP
  }
  if (a->nlev >= 2 && a->rec[0]) {
    const int gu = (int)std::max<int64_t>(1, std::min<int64_t>(G, a->rec_n[0]));
    if (a->rec_w[0] == 8)
      k_pc_up0<TV, 8><<<gu, kThreads, 0, st>>>(a->lev[0], a->rec_n[0], a->rec[0], zout, P->sc,
                                                P->gr, which, a->inv_ces, a->inv_R);
    else
      k_pc_up0<TV, 16><<<gu, kThreads, 0, st>>>(a->lev[0], a->rec_n[0], a->rec[0], zout, P->sc,
                                                 P->gr, which, a->inv_ces, a->inv_R);
  } else if (a->nlev >= 2) {
    const AmgLevel& F = a->lev[0];
#define RBFFD_UP0(Wb)                                                                      \
  k_pc_up<false, true, TV, Wb><<<G, kThreads, 0, st>>>(F, F, zout, a->perm0, P->sc, P->gr, \
                                                       which, a->inv_ces, a->inv_R)
    switch (width_bucket(F.width)) {
      case 8: RBFFD_UP0(8); break;
      case 16: RBFFD_UP0(16); break;
      case 32: RBFFD_UP0(32); break;
      default: RBFFD_UP0(0);
    }
#undef RBFFD_UP0
  }
  else
    k_pc_fin1<<<1, 1, 0, st>>>(P->sc, which, a->inv_ces, a->inv_R);
}

// The graph of `n` iterations of one solve, captured on first use.
int chunk_graph(rbffd_ctx* ctx, StepPlan* P, const void* const (&key)[10], int n,
                const std::function<void(cudaStream_t, int)>& issue, cudaGraphExec_t* out) {
  for (const auto& g : P->graphs)
    if (g.n == n && memcmp(g.key, key, sizeof(g.key)) == 0) {
      *out = g.exec;
      return RBFFD_OK;
    }
  int rc = 0;
  if (!P->cap &&
      (rc = check_cuda(ctx, cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking),
                       "capture stream")))
    return rc;
  if ((rc = check_cuda(ctx, cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal),
                       "begin capture")))
    return rc;
  issue(P->cap, n);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->cap, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return check_cuda(ctx, e, "end capture");
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if ((rc = check_cuda(ctx, e2, "graph instantiate"))) return rc;
  StepPlan::Graph entry;
  memcpy(entry.key, key, sizeof(entry.key));
  entry.n = n;
  entry.exec = ex;
  P->graphs.push_back(entry);
  *out = ex;
  return RBFFD_OK;
}

constexpr int kRestartLen = 50;    // preconditioned cycle length
constexpr int kMaxRestarts = 400;  // restarts of one solve before giving up

// BiCGSTAB on op x = b; with pc (pressure solves only, one right side, no
// rdot), right-preconditioned: p^ = B p, s^ = B s, the SpMVs act on p^ and s^,
// and x gathers alpha p^ + omega s^, so r stays the true residual recurrence.
template <int K, int NRHS, bool RANK1, typename TW, typename TV>
int bicgstab(rbffd_ctx* ctx, StepPlan* P, const KOp<TW, TV>& op, TV* const* x,
             const TV* const* b, TV* (*work)[2], double tol, int maxit, SolveResult* res,
             cudaStream_t st, bool prof = false, uint32_t seed_base = 0,
             const Amg* pc = nullptr, bool x_zero = false, double resume = 0.0,
             bool time_spmv = false) {
  Vecs<TV, NRHS> X, B, R, RH, PP, V, S, T;
  for (int q = 0; q < NRHS; ++q) {
    X.v[q] = x[q];
    B.v[q] = (TV*)b[q];
    R.v[q] = work[0][q];
    RH.v[q] = work[1][q];
    PP.v[q] = work[2][q];
    V.v[q] = work[3][q];
    S.v[q] = work[4][q];
    T.v[q] = work[5][q];
  }
  if (pc && (NRHS != 1 || !RANK1 || op.rdot || !op.a1))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "multigrid preconditioner: pressure solves only");
  // (c . v) of the rank-one completion pairs c with v node by node: the
  // P-node-ordered copy of c (the V-cycle's input map uses the level-0 one)
  const float* pcc = pc ? pc->cnode : nullptr;
  const int vc_launches = pc ? 2 * pc->nlev : 0;
  const int G = P->grid;
  double* sigx = P->dscal;
  KScal* h = (KScal*)ctx->host_pinned;
  int total = 0;
  // staged SpMV launches: one EllStage of dynamic shared memory per block
  size_t smem = 0;
  int Gs = G;
  if constexpr (kStage<K, TW>) {
    smem = sizeof(EllStage<K, TW>);
    const int bps = (int)std::max<size_t>(1, (200u * 1024u) / smem);
    const int64_t ntiles = (op.n + kTileRows - 1) / kTileRows;
    Gs = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * std::min(bps, 8));
    if (Gs < 1) Gs = 1;
    int rc0 = check_cuda(ctx,
                         cudaFuncSetAttribute(k_spmv_p<K, NRHS, RANK1, TW, TV>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "smem attribute");
    if (!rc0)
      rc0 = check_cuda(ctx,
                       cudaFuncSetAttribute(k_spmv_s<K, NRHS, RANK1, TW, TV>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem),
                       "smem attribute");
    if constexpr (NRHS == 1 && RANK1) {
      if (!rc0 && pc)
        rc0 = check_cuda(ctx,
                         cudaFuncSetAttribute(k_spmv_pc<K, TW, TV, 0>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "smem attribute");
      if (!rc0 && pc)
        rc0 = check_cuda(ctx,
                         cudaFuncSetAttribute(k_spmv_pc<K, TW, TV, 1>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                         "smem attribute");
    }
    if (rc0) return rc0;
  }
  // FP64 SpMVs with two right sides (the viscous solves) load directly at 3
  // blocks per SM, 85 registers a thread for the gathers of both right sides
  // in flight: 327 us per launch at 3M rows, against 347 at 4 blocks per SM
  // and 370 staged (an FP64 tile leaves room for two blocks per SM)
  constexpr int kVDirect = 3;
  const int vdir = (std::is_same<TW, double>::value && NRHS == 2 && !pc) ? kVDirect : 0;
  const int Gv = (int)std::max<int64_t>(
      1, std::min<int64_t>((op.n + kThreads - 1) / kThreads, (int64_t)sm_count() * kVDirect));
  // Pressure SpMVs of the preconditioned solve: FP32 operators stage 256-row
  // tiles (48 us per launch at 1M rows, against 50-61 us with direct loads at
  // 4-8 blocks per SM); FP64 operators load directly at 4 blocks per SM, 64
  // registers a thread for the gathers in flight (69.3 us at 1M rows, against
  // 70.2, 92.4 and 72.2 at 3, 6 and 8 blocks per SM and 97 staged: an FP64 tile
  // leaves room for two blocks per SM).
  constexpr int kPcDirect = std::is_same<TW, double>::value ? 4 : 0;
  const int Gd = (int)std::max<int64_t>(
      1, std::min<int64_t>((op.n + kThreads - 1) / kThreads, (int64_t)sm_count() * kPcDirect));
  auto spmv_pc = [&](auto W, cudaStream_t s, const TV* z, TV* y, const TV* dv, KScal* scp,
                     int* wf) {
    constexpr int WH = decltype(W)::value;
    if constexpr (kPcDirect > 0)
      k_spmv_pc<K, TW, TV, WH, kPcDirect><<<Gd, kThreads, 0, s>>>(op, z, y, dv, scp, P->gr, wf);
    else
      k_spmv_pc<K, TW, TV, WH><<<Gs, kThreads, smem, s>>>(op, z, y, dv, scp, P->gr, wf);
  };
  for (int q = 0; q < NRHS; ++q) {
    int rc = check_cuda(ctx, cudaMemcpyAsync(work[6][q], x[q], sizeof(TV) * op.n,
                                             cudaMemcpyDeviceToDevice, st),
                        "save x0");
    if (rc) return rc;
  }
  // A breakdown of the recurrences (a zero inner product) restarts the method
  // from the current iterate with a fresh shadow residual.
  for (int restart = 0;; ++restart) {
    // the caller's x0 = 0 holds only until the first restart
    const bool xz = x_zero && restart == 0;
    bool resumed = false;
    if constexpr (NRHS == 1 && RANK1) {
      // resume > 0: the previous call's directions carry over (k_resume)
      if (pc && restart == 0 && resume > 0.0) {
        k_resume<TV><<<G, kThreads, 0, st>>>(op.n, B.v[0], R.v[0], X.v[0], RH.v[0], P->sc, P->gr,
                                             resume, tol * tol, maxit - total);
        k_update_p<NRHS, RANK1><<<G, kThreads, 0, st>>>(op.n, R, PP, V, P->sc, P->gr, op.rdot,
                                                       pcc);
        P->launches += 2 + vc_launches;
        resumed = true;
      }
    }
    if (!resumed) {
      if (RANK1 && !xz) k_sum<TV><<<G, kThreads, 0, st>>>(x[0], op.n, P->gr, sigx, op.rdot);
      k_init<K, NRHS, RANK1><<<G, kThreads, 0, st>>>(op, X, B, R, RH, PP, sigx, P->sc, P->gr,
                                                      tol * tol, maxit - total,
                                                      (restart || seed_base)
                                                          ? 0x51ED27u + 977u * seed_base + restart
                                                          : 0u,
                                                      pcc, xz ? 1 : 0);
      P->launches += (RANK1 && !xz ? 2 : 1) + (pc ? vc_launches : 0);
    }
    if (pc) vcycle<TV>(P, pc, PP.v[0], 0, zbuf<TV>(pc, 0), st);
    int rc = check_cuda(ctx, cudaGetLastError(), "bicgstab init");
    if (rc) return rc;
    int issued = 0, chunk = 4, prev_iters = 0;
    double prev_rel = -1.0;
    // Preconditioned solves restart every kRestartLen iterations from the
    // current iterate (true residual, fresh shadow residual): on some node
    // sets the preconditioned BiCGSTAB recurrences otherwise stagnate for
    // thousands of iterations.
    const int budget = pc ? std::min(maxit - total, kRestartLen) : maxit - total;
    for (;;) {
      rc = check_cuda(ctx, cudaMemcpyAsync(h, P->sc, sizeof(KScal), cudaMemcpyDeviceToHost, st),
                      "scalar copy");
      if (rc) return rc;
      rc = check_cuda(ctx, cudaStreamSynchronize(st), "bicgstab sync");
      if (rc) return rc;
      if (prof) collect_events(P);
      if (trace_on())
        fprintf(stderr, "[rbffd]   %s iters=%d rr/bb=%.3e\n", sizeof(TV) == 8 ? "fp64" : "fp32",
                h->iters, h->bb[0] > 0 ? h->rr[0] / h->bb[0] : h->rr[0]);
      if (h->done || issued >= budget) break;
      // Next chunk: the iterations that the residual's rate over the last
      // chunk predicts are still needed, plus one (doubling while it has no rate).
      int n = chunk;
      double rel = 0.0;
      for (int q = 0; q < NRHS; ++q)
        if (h->active[q] && h->bb[q] > 0) rel = fmax(rel, sqrt(h->rr[q] / h->bb[q]));
      if (prev_rel > 0.0 && rel > 0.0 && rel < prev_rel && h->iters > prev_iters) {
        const double rate = pow(rel / prev_rel, 1.0 / (double)(h->iters - prev_iters));
        const double need = log(sqrt(h->tol2) / rel) / log(rate);
        if (std::isfinite(need)) n = (int)std::min(64.0, std::max(1.0, ceil(need) + 1.0));
      }
      prev_rel = rel;
      prev_iters = h->iters;
      n = std::min(n, budget - issued);
      if (prof) n = std::min(n, StepPlan::kEv / 4);
      // one chunk of iterations; every kernel returns at once after the solve
      // has finished (sc->done), so a chunk may overshoot harmlessly
      // profiled launches flag whether they did work (slot of their event pair)
      auto work_flag = [&]() -> int* { return prof ? P->evwork + P->ev_used / 2 : nullptr; };
      // external event-record nodes: recorded like stream events when the
      // graph runs, so their timestamps can be read on the host
      auto record_ev = [&](cudaStream_t s) {
        cudaEventRecordWithFlags(P->ev[P->ev_used++], s, cudaEventRecordExternal);
      };
      auto issue = [&](cudaStream_t s, int cnt) {
        for (int it = 0; it < cnt; ++it) {
          if (pc) {  // right-preconditioned: the SpMVs act on B p = zp + kap, B s = zs + kap
            if constexpr (NRHS == 1 && RANK1) {
              if (prof) record_ev(s);
              spmv_pc(std::integral_constant<int, 0>{}, s, zbuf<TV>(pc, 0), V.v[0], RH.v[0],
                      P->sc, work_flag());
              if (prof) record_ev(s);
              k_update_s<NRHS, RANK1><<<G, kThreads, 0, s>>>(op.n, R, V, S, P->sc, P->gr, op.rdot,
                                                             pcc);
              vcycle<TV>(P, pc, S.v[0], 1, zbuf<TV>(pc, 1), s);
              if (prof) record_ev(s);
              spmv_pc(std::integral_constant<int, 1>{}, s, zbuf<TV>(pc, 1), T.v[0], S.v[0],
                      P->sc, work_flag());
              if (prof) record_ev(s);
              k_update_xr_pc<TV><<<G, kThreads, 0, s>>>(op.n, X.v[0], R.v[0], RH.v[0],
                                                        zbuf<TV>(pc, 0), zbuf<TV>(pc, 1), S.v[0],
                                                        T.v[0], P->sc, P->gr);
              k_update_p<NRHS, RANK1><<<G, kThreads, 0, s>>>(op.n, R, PP, V, P->sc, P->gr, op.rdot,
                                                             pcc);
              vcycle<TV>(P, pc, PP.v[0], 0, zbuf<TV>(pc, 0), s);
            }
            continue;
          }
          if (prof) record_ev(s);
          if (vdir)
            k_spmv_p<K, NRHS, RANK1, TW, TV, kVDirect><<<Gv, kThreads, 0, s>>>(
                op, PP, V, RH, P->sc, P->gr, work_flag());
          else
            k_spmv_p<K, NRHS, RANK1><<<Gs, kThreads, smem, s>>>(op, PP, V, RH, P->sc, P->gr,
                                                                work_flag());
          if (prof) record_ev(s);
          k_update_s<NRHS, RANK1><<<G, kThreads, 0, s>>>(op.n, R, V, S, P->sc, P->gr, op.rdot,
                                                         pcc);
          if (prof) record_ev(s);
          if (vdir)
            k_spmv_s<K, NRHS, RANK1, TW, TV, kVDirect><<<Gv, kThreads, 0, s>>>(
                op, S, S, T, P->sc, P->gr, work_flag());
          else
            k_spmv_s<K, NRHS, RANK1><<<Gs, kThreads, smem, s>>>(op, S, S, T, P->sc, P->gr,
                                                                work_flag());
          if (prof) record_ev(s);
          k_update_xr<NRHS><<<G, kThreads, 0, s>>>(op.n, X, R, RH, PP, S, S, T, P->sc, P->gr);
          k_update_p<NRHS, RANK1><<<G, kThreads, 0, s>>>(op.n, R, PP, V, P->sc, P->gr, op.rdot,
                                                         pcc);
        }
      };
      if (prof) {
        // Profiled chunks are graphs too, with the SpMVs' event records as
        // graph nodes: their timestamps then bracket the kernels as they run
        // back to back, without the host's launch gaps of eager launches.
        // One graph per chunk (a power of two of iterations) so that the
        // event slots of one chunk do not overlap.
        int pw = 1;
        while (pw * 2 <= n) pw *= 2;
        n = pw;
        const void* const key[10] = {(const void*)&bicgstab<K, NRHS, RANK1, TW, TV>,
                                     op.idx, op.w, op.es, X.v[0], X.v[NRHS - 1], pc,
                                     work[0][0], (const void*)P->evwork, nullptr};
        P->ev_used = 0;
        cudaGraphExec_t g = nullptr;
        rc = chunk_graph(ctx, P, key, n, issue, &g);
        if (rc) return rc;
        P->ev_used = 4 * n;  // the events the graph records (also when it was cached)
        rc = check_cuda(ctx, cudaGraphLaunch(g, st), "graph launch");
        if (rc) return rc;
      } else {
        const void* const key[10] = {(const void*)&bicgstab<K, NRHS, RANK1, TW, TV>,
                                     op.idx, op.w, op.es, X.v[0], X.v[NRHS - 1], pc,
                                     work[0][0], nullptr, nullptr};
        for (int part = 64; part >= 1; part >>= 1) {  // n as a sum of powers of two
          if (!(n & part)) continue;
          cudaGraphExec_t g = nullptr;
          rc = chunk_graph(ctx, P, key, part, issue, &g);
          if (rc) return rc;
          rc = check_cuda(ctx, cudaGraphLaunch(g, st), "graph launch");
          if (rc) return rc;
        }
      }
      P->launches += (int64_t)(5 + 2 * vc_launches) * n;
      rc = check_cuda(ctx, cudaGetLastError(), "bicgstab iteration");
      if (rc) return rc;
      issued += n;
      chunk = std::min(chunk * 2, 64);
    }
    total += h->iters;
    if (h->stage_err)
      return set_error(ctx, RBFFD_ERR_CUDA, "SpMV tile copy did not complete (bounded wait)");
    double worst = 0.0;
    bool conv = true;
    for (int q = 0; q < NRHS; ++q) {
      const double rel = h->bb[q] > 0 ? sqrt(h->rr[q] / h->bb[q]) : sqrt(h->rr[q]);
      worst = fmax(worst, rel);
      if (!(h->rr[q] <= h->tol2 * h->bb[q])) conv = false;
    }
    res->iters = total;
    res->status = h->status;
    res->relres = worst;
    res->converged = conv;
    res->resumable = pc != nullptr && conv && h->status == 0 && !h->half[0];
    if (trace_on())
      fprintf(stderr, "[rbffd] bicgstab %s nrhs=%d restart=%d iters=%d relres=%.3e status=%d\n",
              sizeof(TV) == 8 ? "fp64" : "fp32", NRHS, restart, h->iters, worst, h->status);
    const bool breakdown = h->status == 1 || h->status == 3 || h->status == 4;
    const bool diverged = h->status == 5;
    const bool cycle_end = pc && !h->done && h->iters >= budget;  // restart, keep x
    if (conv || !(breakdown || diverged || cycle_end) || total >= maxit ||
        restart >= kMaxRestarts)
      break;
    if (diverged) {  // start again from the initial iterate
      for (int q = 0; q < NRHS; ++q) {
        rc = check_cuda(ctx, cudaMemcpyAsync(x[q], work[6][q], sizeof(TV) * op.n,
                                             cudaMemcpyDeviceToDevice, st),
                        "restore x0");
        if (rc) return rc;
      }
    }
  }
  if constexpr (NRHS == 1 && RANK1) {
    if (prof && pc) {
      // The pressure SpMV once more, 20 launches back to back on this solve's
      // operator and vectors (a scratch copy of the scalars, the output into
      // a work vector), bracketed by one event pair: its launch duration
      // without the event nodes between the solve's kernels.
      constexpr int kReps = 20;
      int rc = 0;
      if (!P->sc_timing) rc = palloc(ctx, P, &P->sc_timing, 1);
      if (!rc)
        rc = check_cuda(ctx, cudaMemcpyAsync(P->sc_timing, P->sc, sizeof(KScal),
                                             cudaMemcpyDeviceToDevice, st),
                        "timing scalars");
      if (!rc)
        rc = check_cuda(ctx, cudaMemsetAsync(&P->sc_timing->done, 0, sizeof(int), st), "timing");
      if (!rc)
        rc = check_cuda(ctx, cudaMemsetAsync(&P->sc_timing->stage_err, 0, sizeof(int), st),
                        "timing");
      if (rc) return rc;
      cudaEventRecord(P->ev[0], st);
      for (int r = 0; r < kReps; ++r)
        spmv_pc(std::integral_constant<int, 0>{}, st, zbuf<TV>(pc, 0), T.v[0], RH.v[0],
                P->sc_timing, nullptr);
      cudaEventRecord(P->ev[1], st);
      float ms = 0.f;
      if (cudaEventSynchronize(P->ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]) == cudaSuccess) {
        P->spmv_batch_ms += ms;
        P->spmv_batch_launches += kReps;
      }
      P->launches += kReps;
      rc = check_cuda(ctx, cudaGetLastError(), "SpMV timing");
      if (rc) return rc;
    }
  }
  if constexpr (NRHS == 2 && !RANK1) {
    if (time_spmv) {
      // The viscous SpMV (both right sides) the same way: 20 launches back to
      // back on this solve's operator and vectors, output into a work vector
      constexpr int kReps = 20;
      int rc = 0;
      if (!P->sc_timing) rc = palloc(ctx, P, &P->sc_timing, 1);
      if (!rc)
        rc = check_cuda(ctx, cudaMemcpyAsync(P->sc_timing, P->sc, sizeof(KScal),
                                             cudaMemcpyDeviceToDevice, st),
                        "timing scalars");
      if (!rc)
        rc = check_cuda(ctx, cudaMemsetAsync(&P->sc_timing->done, 0, sizeof(int), st), "timing");
      if (!rc)
        rc = check_cuda(ctx, cudaMemsetAsync(&P->sc_timing->stage_err, 0, sizeof(int), st),
                        "timing");
      if (rc) return rc;
      cudaEventRecord(P->ev[0], st);
      for (int r = 0; r < kReps; ++r) {
        if (vdir)
          k_spmv_p<K, NRHS, RANK1, TW, TV, kVDirect><<<Gv, kThreads, 0, st>>>(
              op, PP, T, RH, P->sc_timing, P->gr, nullptr);
        else
          k_spmv_p<K, NRHS, RANK1><<<Gs, kThreads, smem, st>>>(op, PP, T, RH, P->sc_timing, P->gr,
                                                               nullptr);
      }
      cudaEventRecord(P->ev[1], st);
      float ms = 0.f;
      if (cudaEventSynchronize(P->ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]) == cudaSuccess) {
        P->vspmv_batch_ms += ms;
        P->vspmv_batch_launches += kReps;
      }
      P->launches += kReps;
      rc = check_cuda(ctx, cudaGetLastError(), "SpMV timing");
      if (rc) return rc;
    }
  }
  return RBFFD_OK;
}

// FP64 iterative refinement: the residual uses the FP64 operator; each
// correction solves the FP32 copy of the operator in FP32 (FP32 weights,
// vectors and recurrences; the pressure solves with the FP32 V-cycle) to a
// loose relative tolerance, from the normalised residual.  A correction that
// does not lower the FP64 residual is undone and the inner solve repeated with
// another shadow residual.
template <int K, int NRHS, bool RANK1>
int refine(rbffd_ctx* ctx, StepPlan* P, const KOp<double, double>& op64,
           const KOp<float, float>& op32, double* const* x, const double* const* b, double tol,
           double inner_tol, int maxit, SolveResult* res, int* sweeps, cudaStream_t st,
           bool prof = false) {
  Vecs<double, NRHS> X, B, R;
  Vecs<float, NRHS> R32, E32;
  for (int q = 0; q < NRHS; ++q) {
    X.v[q] = x[q];
    B.v[q] = (double*)b[q];
    R.v[q] = P->r64[q];
    R32.v[q] = P->r32[q];
    E32.v[q] = P->e32[q];
  }
  const int G = P->grid;
  int used = 0, failures = 0, retries = 0;
  double prev_rel = INFINITY, last_nrm[2] = {0, 0};
  bool resumable = false;  // the last inner solve's directions can carry over
  res->iters = 0;
  res->status = 0;
  *sweeps = 0;
  double* h = (double*)ctx->host_pinned + 64;
  for (int sweep = 0;; ++sweep) {
    if (RANK1) k_sum<double><<<G, kThreads, 0, st>>>(x[0], op64.n, P->gr, P->dscal, op64.rdot);
    k_residual64<K, NRHS, RANK1><<<G, kThreads, 0, st>>>(op64, X, B, R, P->dscal, P->dscal + 1,
                                                         P->gr);
    P->launches += RANK1 ? 2 : 1;
    int rc = check_cuda(ctx, cudaGetLastError(), "residual");
    if (rc) return rc;
    rc = check_cuda(ctx, cudaMemcpyAsync(h, P->dscal + 1, 4 * sizeof(double),
                                         cudaMemcpyDeviceToHost, st),
                    "residual copy");
    if (rc) return rc;
    rc = check_cuda(ctx, cudaStreamSynchronize(st), "residual sync");
    if (rc) return rc;
    double worst = 0.0, nrm[2] = {0, 0};
    bool conv = true, finite = true;
    for (int q = 0; q < NRHS; ++q) {
      const double rr = h[2 * q], bb = h[2 * q + 1];
      if (!std::isfinite(rr)) finite = false;
      nrm[q] = sqrt(rr);
      const double rel = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
      worst = fmax(worst, rel);
      if (!(rr <= tol * tol * bb)) conv = false;
    }
    if (sweep > 0 && (!finite || !(worst < prev_rel))) {
      // the last correction made things worse: undo it and solve again
      k_addcorr<NRHS><<<G, kThreads, 0, st>>>(op64.n, X, E32, -last_nrm[0],
                                              NRHS > 1 ? -last_nrm[NRHS - 1] : 0.0);
      P->launches += 1;
      rc = check_cuda(ctx, cudaGetLastError(), "undo correction");
      if (rc) return rc;
      ++retries;
      resumable = false;
      if (++failures > 6 || used >= maxit) {
        res->relres = prev_rel;
        res->converged = false;
        res->status = finite ? 5 : 2;
        return RBFFD_OK;
      }
      continue;  // recompute the residual of the restored iterate
    }
    if (trace_on())
      fprintf(stderr, "[rbffd] refine nrhs=%d sweep=%d relres=%.3e used=%d\n", NRHS, sweep, worst,
              used);
    failures = 0;
    prev_rel = worst;
    res->relres = worst;
    res->converged = conv;
    if (conv || used >= maxit || sweep >= 60) return RBFFD_OK;
    ++*sweeps;
    const double i0 = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
    const double i1 = NRHS > 1 && nrm[NRHS - 1] > 0 ? 1.0 / nrm[NRHS - 1] : 0.0;
    k_to32<NRHS><<<G, kThreads, 0, st>>>(op64.n, R, R32, E32, i0, i1);
    P->launches += 2;  // with the correction below
    // A preconditioned inner solve resumes the previous sweep's Krylov
    // directions on the new residual (k_resume) instead of starting afresh.
    // (Measured neutral on the 1M cavity, 33.3 against 31.7 iterations per
    // step: each sweep's FP64 residual is mostly new content.)
    const double resume =
        resumable && nrm[0] > 0.0 && last_nrm[0] > 0.0 ? last_nrm[0] / nrm[0] : 0.0;
    SolveResult inner;
    rc = bicgstab<K, NRHS, RANK1, float, float>(ctx, P, op32, E32.v, R32.v, P->kw32, inner_tol,
                                                maxit - used, &inner, st, prof, retries,
                                                RANK1 ? P->amg : nullptr, true, resume);
    if (rc) return rc;
    resumable = inner.resumable;
    used += inner.iters > 0 ? inner.iters : 1;
    res->iters += inner.iters;
    last_nrm[0] = nrm[0];
    last_nrm[1] = nrm[1];
    k_addcorr<NRHS><<<G, kThreads, 0, st>>>(op64.n, X, E32, nrm[0],
                                            NRHS > 1 ? nrm[NRHS - 1] : 0.0);
    rc = check_cuda(ctx, cudaGetLastError(), "correction");
    if (rc) return rc;
  }
}

template <int K, bool MIX>
int run_steps(rbffd_ctx* ctx, StepPlan* P, const rbffd_flow& f, rbffd_state* s, const double* gu,
              const double* gv, int32_t n_steps, rbffd_stats* stats, cudaStream_t st) {
  const int G = P->grid;
  const int k = P->k;
  const double a = f.dt / (2.0 * f.Re);
  const void* vdx = MIX ? (const void*)P->vv_dx32 : (const void*)f.vv_dx;
  const void* vdy = MIX ? (const void*)P->vv_dy32 : (const void*)f.vv_dy;
  const void* vlap = MIX ? (const void*)P->vv_lap32 : (const void*)f.vv_lap;
  const void* plap = MIX ? (const void*)P->pp_lap32 : (const void*)f.pp_lap;
  const void* gdx = MIX ? (const void*)P->vp_dx32 : (const void*)f.vp_dx;
  const void* gdy = MIX ? (const void*)P->vp_dy32 : (const void*)f.vp_dy;
  if (MIX) {
    k_split<<<G, kThreads, 0, st>>>(f.N, s->u, P->u2);
    k_split<<<G, kThreads, 0, st>>>(f.N, s->v, P->v2);
    k_split<<<G, kThreads, 0, st>>>(f.M, s->pt, P->pt2);
    P->launches += 3;
  }
  const int64_t launches0 = P->launches;
  P->spmv_ms = 0.0;
  P->spmv_launches = 0;
  P->spmv_batch_ms = 0.0;
  P->spmv_batch_launches = 0;
  P->vspmv_batch_ms = 0.0;
  P->vspmv_batch_launches = 0;
  if (f.profile && !P->ev[0]) {
    for (int i = 0; i < StepPlan::kEv; ++i) {
      int rc = check_cuda(ctx, cudaEventCreate(&P->ev[i]), "event create");
      if (rc) return rc;
    }
    int rc = palloc(ctx, P, &P->evwork, StepPlan::kEv / 2);
    if (!rc) rc = check_cuda(ctx, cudaMemset(P->evwork, 0, sizeof(int) * (StepPlan::kEv / 2)),
                             "flags");
    if (rc) return rc;
  }
  KOp<double, double> H64{f.vv_idx, P->Hw, f.ld_v, f.N, k, 1, nullptr};
  KOp<double, double> L64{P->Lidx, P->Lw, f.ld_p, f.M, P->kL, 0, P->es, nullptr, P->a1};
  KOp<float, float> H32{f.vv_idx, P->Hw32, f.ld_v, f.N, k, 1, nullptr, nullptr};
  KOp<float, float> L32{P->Lidx, P->Lw32, f.ld_p, f.M, P->kL, 0, P->es32, nullptr, P->a1_32};
  L32.diff = P->a1_32 ? 1 : 0;
  const bool proj = P->proj != 0;
  if (f.precond && !proj) (MIX ? L32.tiles : L64.tiles) = P->Lt;
  (MIX ? H32.tiles : H64.tiles) = P->Ht;
  // open flows: one viscous operator per component on the shared index array
  KOp<double, double> Hu64{P->Hidx, P->Hw, f.ld_v, f.N, k, 1, nullptr};
  KOp<double, double> Hv64{P->Hidx, P->Hw_v, f.ld_v, f.N, k, 1, nullptr};
  KOp<float, float> Hu32{P->Hidx, P->Hw32, f.ld_v, f.N, k, 1, nullptr, nullptr};
  KOp<float, float> Hv32{P->Hidx, P->Hw32_v, f.ld_v, f.N, k, 1, nullptr, nullptr};
  (MIX ? Hu32.tiles : Hu64.tiles) = P->Ht;
  (MIX ? Hv32.tiles : Hv64.tiles) = P->Ht_v;
  for (int32_t step = 0; step < n_steps; ++step) {
    ConvArgs ca{f.N,  f.ld_v,       k,  f.vv_idx, vdx, vdy,   s->u,  s->v,  P->u2,
                P->v2, s->cu_prev, s->cv_prev, P->us, P->vs, P->us2, P->vs2, f.dt,
                s->j == 0 ? 1 : 0};
    k_convect<K, MIX><<<G, kThreads, 0, st>>>(ca);
    HelmRhsArgs ha{f.N,    f.ld_v, k,      f.vv_idx, vlap,   P->us,  P->vs,  P->us2,
                   P->vs2, f.vp_idx, gdx,  gdy,      s->pt,  P->pt2, f.v_bc, f.v_nx,
                   f.v_ny, gu,     gv,     a,        f.dt,   f.km_mode, P->ru, P->rv,
                   P->uss, P->vss, s->u,   s->v,     P->u2,  P->v2, f.cn_form, P->proj,
                   f.v_bcu, f.v_bcv};
    // the viscous solves start from the extrapolation of the previous steps'
    // solutions when this plan made them (P->px_step == s->j), as the
    // pressure solve does
    if (P->px_step == s->j) {
      ha.vord = std::min(P->vhist, kMaxHist);
      double b = ha.vord + 1.0;  // C(vord + 1, q + 1) with alternating signs
      for (int q = 0; q <= ha.vord; ++q) {
        ha.vc[q] = (q & 1) ? -b : b;
        b = b * (ha.vord - q) / (q + 2.0);
      }
      for (int q = 0; q < kMaxHist; ++q) {
        ha.hu[q] = P->vhu[(P->vhead + q) % kMaxHist];
        ha.hv[q] = P->vhv[(P->vhead + q) % kMaxHist];
      }
      P->vhead = (P->vhead + kMaxHist - 1) % kMaxHist;
      P->vhist = std::min(P->vhist + 1, kMaxHist);
    } else {
      P->vhist = 0;
    }
    k_helm_rhs<K, MIX><<<G, kThreads, 0, st>>>(ha);
    P->launches += 2 + (MIX ? 2 : 0) + 4 + (MIX ? 1 : 0);  // stage kernels of this step
    int rc = check_cuda(ctx, cudaGetLastError(), "stage 1-2 kernels");
    if (rc) return rc;
    double* hx[2] = {P->uss, P->vss};
    const double* hb[2] = {P->ru, P->rv};
    SolveResult hr;
    int sweeps = 0;
    // The viscous operator is well conditioned: its FP32 inner solves go to the
    // square of the inner tolerance (each FP64 residual of the 3M-row, two-sided
    // solve costs more than a few extra FP32 iterations).
    // In the FP64 path of a closed flow the viscous solves go 1000 times below
    // the tolerance (not below 1e-13; tolerances under 1e-13 are kept): the
    // error of u** enters the pressure right side through the divergence, and
    // what the extrapolated pressure guess cannot predict costs pressure
    // iterations (on the 1M cavity 25.5 per step at the tolerance, 9.0 at 1e-4
    // of it, each viscous solve 2 iterations from its extrapolated guess).  In
    // MIXED precision a tighter viscous target measured no gain (33.7 pressure
    // iterations per step at 1e-12), so the tolerance stays.
    const double vtol = (MIX || P->open || f.tol < 1e-13) ? f.tol : std::max(f.tol * 1e-3, 1e-13);
    if (P->open) {
      // per-component operators: one solve each
      SolveResult h2[2];
      int sw[2] = {0, 0};
      for (int c = 0; c < 2 && !rc; ++c) {
        const KOp<double, double>& o64 = c ? Hv64 : Hu64;
        const KOp<float, float>& o32 = c ? Hv32 : Hu32;
        if (MIX)
          rc = refine<K, 1, false>(ctx, P, o64, o32, &hx[c], &hb[c], f.tol,
                                   f.inner_tol * f.inner_tol, f.max_iter, &h2[c], &sw[c], st);
        else
          rc = bicgstab<K, 1, false, double, double>(ctx, P, o64, &hx[c], &hb[c], P->kw64, f.tol,
                                                     f.max_iter, &h2[c], st);
      }
      hr = h2[0];
      hr.iters = h2[0].iters + h2[1].iters;
      hr.relres = std::max(h2[0].relres, h2[1].relres);
      hr.converged = h2[0].converged && h2[1].converged;
      if (!h2[1].converged || h2[1].status == 2) hr.status = h2[1].status;
      sweeps = sw[0] + sw[1];
    } else if (MIX) {
      rc = refine<K, 2, false>(ctx, P, H64, H32, hx, hb, vtol, f.inner_tol * f.inner_tol,
                               f.max_iter, &hr, &sweeps, st);
    } else {
      rc = bicgstab<K, 2, false, double, double>(ctx, P, H64, hx, hb, P->kw64, vtol, f.max_iter,
                                                 &hr, st, false, 0, nullptr, false, 0.0,
                                                 f.profile != 0);
    }
    if (rc) return rc;
    if (stats) {
      stats->helm_iters += hr.iters;
      stats->helm_relres = hr.relres;
      stats->refinements += sweeps;
    }
    if (hr.status == 2) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite viscous solve");
    // a solve short of the tighter target but within the tolerance is accepted
    if (!hr.converged && !(hr.relres <= f.tol))
      return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                       "viscous solve: relative residual %.3e after %d iterations (status %d)",
                       hr.relres, hr.iters, hr.status);
    if (MIX) {
      k_split<<<G, kThreads, 0, st>>>(f.N, P->uss, P->uss2);
      k_split<<<G, kThreads, 0, st>>>(f.N, P->vss, P->vss2);
    }
    // The divergence is the right side of the pressure solve and nearly zero:
    // FP32 weights would leave their rounding (relative to the terms, not to
    // their small sum) in p~, so both precisions take it with FP64 weights.
    DivArgs da{f.M,    f.ld_p,  k,      f.pv_idx, f.pv_dx,  f.pv_dy,      P->uss,
               P->vss, P->uss2, P->vss2, f.p_bc,  P->scale, 1.0 / f.dt, P->pb, P->proj};
    k_divergence<K, false><<<G, kThreads, 0, st>>>(da);
    // Initial guess: the extrapolation in time through the previous steps'
    // solutions (up to cubic), else the state's p~.  Any guess
    // leaves the converged solution the same; a better one saves iterations
    // (p~ changes smoothly from step to step).
    if (P->px_step != s->j) {
      // the exact projection solves for the increment of p~: start from zero
      rc = proj ? check_cuda(ctx, cudaMemsetAsync(P->px, 0, sizeof(double) * f.M, st), "zero start")
                : check_cuda(ctx, cudaMemcpyAsync(P->px, s->pt, sizeof(double) * f.M,
                                                  cudaMemcpyDeviceToDevice, st),
                             "warm start");
      if (rc) return rc;
      P->nhist = 0;
    } else {
      const int ord = std::min(P->nhist, kMaxHist);
      History H;
      for (int q = 0; q < kMaxHist; ++q) H.h[q] = P->pxh[(P->hhead + q) % kMaxHist];
      k_extrapolate<<<G, kThreads, 0, st>>>(f.M, ord, P->px, H);
      rc = check_cuda(ctx, cudaGetLastError(), "extrapolation");
      if (rc) return rc;
      P->hhead = (P->hhead + kMaxHist - 1) % kMaxHist;  // the recycled slot is the newest
      P->nhist = std::min(P->nhist + 1, kMaxHist);
    }
    double* px[1] = {P->px};
    const double* pbv[1] = {P->pb};
    SolveResult pr;
    const bool prof = f.profile != 0;
    if (proj) {  // the composed operator's rows are read directly (runtime width)
      if (MIX)
        rc = refine<0, 1, true>(ctx, P, L64, L32, px, pbv, f.tol, f.inner_tol, f.max_iter, &pr,
                                &sweeps, st, prof);
      else
        rc = bicgstab<0, 1, true, double, double>(ctx, P, L64, px, pbv, P->kw64, f.tol,
                                                  f.max_iter, &pr, st, prof, 0, P->amg);
    } else if (MIX) {
      rc = refine<K, 1, true>(ctx, P, L64, L32, px, pbv, f.tol, f.inner_tol, f.max_iter, &pr,
                              &sweeps, st, prof);
    } else {
      rc = bicgstab<K, 1, true, double, double>(ctx, P, L64, px, pbv, P->kw64, f.tol, f.max_iter,
                                                &pr, st, prof, 0, P->amg);
    }
    if (rc) return rc;
    if (stats) {
      stats->poisson_iters += pr.iters;
      stats->poisson_relres = pr.relres;
      stats->refinements += MIX ? sweeps : 0;
    }
    if (pr.status == 2) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite pressure solve");
    if (!pr.converged)
      return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                       "pressure solve: relative residual %.3e after %d iterations (status %d)",
                       pr.relres, pr.iters, pr.status);
    k_sum<double><<<G, kThreads, 0, st>>>(P->px, f.M, P->gr, P->dscal);
    if (MIX) k_split<<<G, kThreads, 0, st>>>(f.M, P->px, P->px2);
    PresArgs pa{f.M,   f.ld_p, k,    f.pp_idx, plap,   P->px,  P->px2,
                P->dscal, a,   s->pt, s->p, P->pt2,   P->proj, P->pdir > 0 ? 1 : 0};
    k_pressure<K, MIX><<<G, kThreads, 0, st>>>(pa);
    // The exact projection corrects with G0 x (x = phi + const) and the wall
    // flux, with FP64 weights in both precisions (like the divergence), so
    // that D^(P,V) u_{j+1} vanishes to the solve's accuracy.
    CorrArgs ka{f.N,      f.ld_v, k,        f.vp_idx,       proj ? f.vp_dx : gdx,
                proj ? f.vp_dy : gdy,       proj ? P->px : s->pt,   proj ? P->px2 : P->pt2,
                P->uss,   P->vss, f.v_bc,   gu,             gv,   f.dt,
                f.overwrite_bc,   s->u,     s->v,           P->u2, P->v2,
                P->proj,  P->dscal, P->esn, f.v_nx,         f.v_ny,
                f.v_bcu,  f.v_bcv};
    if (proj && MIX) {
      k_correct<K, false><<<G, kThreads, 0, st>>>(ka);
      k_split<<<G, kThreads, 0, st>>>(f.N, s->u, P->u2);
      k_split<<<G, kThreads, 0, st>>>(f.N, s->v, P->v2);
    } else {
      k_correct<K, MIX><<<G, kThreads, 0, st>>>(ka);
    }
    rc = check_cuda(ctx, cudaGetLastError(), "stage 3 kernels");
    if (rc) return rc;
    s->j += 1;
    P->px_step = s->j;
    if (stats) stats->steps += 1;
  }
  int rc = check_cuda(ctx, cudaStreamSynchronize(st), "step sync");
  if (stats && proj && n_steps > 0 && !rc) {
    double sx = 0.0;
    rc = check_cuda(ctx, cudaMemcpy(&sx, P->dscal, sizeof(double), cudaMemcpyDeviceToHost),
                    "wall flux");
    stats->wall_flux = -f.dt * sx / P->esn_h;
  }
  if (stats) {
    stats->launches = P->launches - launches0;
    stats->spmv_launches = P->spmv_launches;
    stats->spmv_ms = P->spmv_ms;
    stats->spmv_batch_launches = P->spmv_batch_launches;
    stats->spmv_batch_ms = P->spmv_batch_ms;
    stats->vspmv_batch_launches = P->vspmv_batch_launches;
    stats->vspmv_batch_ms = P->vspmv_batch_ms;
  }
  return rc;
}

}  // namespace

int step_set_wait_limit(rbffd_ctx* ctx, long long polls) {
  const long long v = polls < 0 ? kSpinLimit : (polls > kSpinLimit ? kSpinLimit : polls);
  return check_cuda(ctx, cudaMemcpyToSymbol(g_wait_polls, &v, sizeof(v)), "wait limit");
}

int step_run(rbffd_ctx* ctx, const rbffd_flow* f, rbffd_state* s, const double* gu,
             const double* gv, int32_t n_steps, rbffd_stats* stats, cudaStream_t st) {
  const rbffd_flow key = plan_key(*f);
  if (ctx->plan && memcmp(&ctx->plan->key, &key, sizeof(rbffd_flow)) != 0) {
    cudaStreamSynchronize(st);
    step_plan_free(ctx->plan);
    ctx->plan = nullptr;
  }
  if (!ctx->plan) {
    int rc = build_plan(ctx, *f, &ctx->plan, st);
    if (rc) return rc;
  }
  StepPlan* P = ctx->plan;
  const bool mix = f->precision == RBFFD_PREC_MIXED;
  if (P->k == 28)
    return mix ? run_steps<28, true>(ctx, P, *f, s, gu, gv, n_steps, stats, st)
               : run_steps<28, false>(ctx, P, *f, s, gu, gv, n_steps, stats, st);
  return mix ? run_steps<0, true>(ctx, P, *f, s, gu, gv, n_steps, stats, st)
             : run_steps<0, false>(ctx, P, *f, s, gu, gv, n_steps, stats, st);
}

}  // namespace rbffd

// ===================================================================== adjoint
//
// Reverse-mode derivative of one fractional step (rbffd_adjoint_step).  Every
// transposed operator is stored as an ELL matrix of its own (built once per
// plan): the entries of each column of the forward operator are gathered into
// one row, ordered by forward row so the result does not depend on the order
// in which the build's atomics ran.  Transposed products are then plain
// gathers, like the forward ones.  The transposed pressure solve uses
// K = L^T - gamma 1 e^T: its solution z satisfies e^T z = 0 and L^T z = l - mean(l),
// which is the first block of the transposed bordered system
// [L^T 1; e^T 0] [z; z0] = [l; 0].
namespace rbffd {

struct TEll {
  int32_t* idx = nullptr;   // transposed column = forward row
  int32_t* slot = nullptr;  // forward slot of each entry, -1 for padding
  int* counts = nullptr;
  int width = 0;
  int64_t ld = 0, n = 0;
};

struct AdjointPlan {
  std::vector<void*> allocs;
  TEll tvv, tpv, tvp, tl;
  double *DxT = nullptr, *DyT = nullptr, *LapT = nullptr, *HwT = nullptr;
  double *PxT = nullptr, *PyT = nullptr, *GxT = nullptr, *GyT = nullptr, *LT = nullptr;
  double *e = nullptr, *es_t = nullptr;
  double *luss, *lvss, *lru, *lrv, *t1, *t2, *t3, *t4, *lus, *lvs, *lcu, *lcv;
  double *lpt, *z, *rhs;
};

void adjoint_plan_free(AdjointPlan* a) {
  if (!a) return;
  for (void* p : a->allocs) cudaFree(p);
  delete a;
}

namespace {

__global__ void k_t_count(int64_t n_rows, int64_t ld, int k, const int32_t* __restrict__ idx,
                          int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int s = 0; s < k; ++s) atomicAdd(&counts[idx[s * ld + i]], 1);
}

__global__ void k_t_max(int64_t n, const int* __restrict__ counts, int* __restrict__ mx) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, counts[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

__global__ void k_t_fill(int64_t n_rows, int64_t ld, int k, const int32_t* __restrict__ idx,
                         int* __restrict__ cursor, int64_t ldt, int32_t* __restrict__ tidx,
                         int32_t* __restrict__ tslot) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int s = 0; s < k; ++s) {
      const int32_t c = idx[s * ld + i];
      const int pos = atomicAdd(&cursor[c], 1);
      tidx[pos * ldt + c] = (int32_t)i;
      tslot[pos * ldt + c] = s;
    }
}

// order each transposed row by forward row; pad with (self, -1)
__global__ void k_t_sort_pad(int64_t n_cols, int64_t ldt, int width, const int* __restrict__ counts,
                             int32_t* __restrict__ tidx, int32_t* __restrict__ tslot) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cols;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int m = counts[c];
    for (int a = 1; a < m; ++a) {
      const int32_t r = tidx[a * ldt + c], q = tslot[a * ldt + c];
      int b = a;
      while (b > 0 && tidx[(b - 1) * ldt + c] > r) {
        tidx[b * ldt + c] = tidx[(b - 1) * ldt + c];
        tslot[b * ldt + c] = tslot[(b - 1) * ldt + c];
        --b;
      }
      tidx[b * ldt + c] = r;
      tslot[b * ldt + c] = q;
    }
    for (int a = m; a < width; ++a) {
      tidx[a * ldt + c] = (int32_t)c;
      tslot[a * ldt + c] = -1;
    }
  }
}

// tw[a][c] = alpha * w[slot][row] * rowmul[row] * colmul[c]  (multipliers optional)
__global__ void k_t_weights(int64_t n_cols, int64_t ldt, int width, const int32_t* __restrict__ tidx,
                            const int32_t* __restrict__ tslot, const double* __restrict__ w,
                            int64_t ld, const double* __restrict__ rowmul,
                            const double* __restrict__ colmul, double alpha,
                            double* __restrict__ tw) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cols;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double cm = colmul ? colmul[c] : 1.0;
    for (int a = 0; a < width; ++a) {
      const int32_t q = tslot[a * ldt + c];
      double v = 0.0;
      if (q >= 0) {
        const int32_t r = tidx[a * ldt + c];
        v = alpha * w[q * ld + r] * (rowmul ? rowmul[r] : 1.0) * cm;
      }
      tw[a * ldt + c] = v;
    }
  }
}

__global__ void k_adj_setup_vec(int64_t M, const uint8_t* __restrict__ p_bc,
                                const double* __restrict__ scale, double* __restrict__ e,
                                double* __restrict__ inv_scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    e[i] = p_bc[i] ? 1.0 : 0.0;  // the bordering vector: boundary rows
    inv_scale[i] = 1.0 / scale[i];
  }
}

__global__ void k_adj_es(int64_t M, const double* __restrict__ scale, const double* sum,
                         double* __restrict__ es_t) {
  const double g = *sum != 0.0 ? 1.0 / fabs(*sum) : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x)
    es_t[i] = -scale[i] * g;
}

__device__ __forceinline__ double tgather(const int32_t* __restrict__ idx,
                                          const double* __restrict__ w, int64_t ld, int width,
                                          int64_t i, const double* __restrict__ x) {
  double acc = 0.0;
  for (int s = 0; s < width; ++s) acc += w[s * ld + i] * x[idx[s * ld + i]];
  return acc;
}

// wall rows of the correction: the overwrite sends their adjoint to the wall data
__global__ void k_adj_mask(int64_t N, const double* __restrict__ lun, const double* __restrict__ lvn,
                           const uint8_t* __restrict__ v_bc, int overwrite, double* __restrict__ gu,
                           double* __restrict__ gv, double* __restrict__ luss,
                           double* __restrict__ lvss) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a = lun[i], b = lvn[i];
    if (overwrite && v_bc[i]) {
      gu[i] += a;
      gv[i] += b;
      a = 0.0;
      b = 0.0;
    }
    luss[i] = a;
    lvss[i] = b;
  }
}

// l~_j = l_pt_out,j - dt (G_x^T l_u** + G_y^T l_v**)_j
__global__ void k_adj_pt(int64_t M, TEll t, const double* __restrict__ GxT,
                         const double* __restrict__ GyT, const double* __restrict__ luss,
                         const double* __restrict__ lvss, const double* __restrict__ lpt_out,
                         double dt, double* __restrict__ lpt) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * blockDim.x)
    lpt[j] = lpt_out[j] - dt * (tgather(t.idx, GxT, t.ld, t.width, j, luss) +
                                tgather(t.idx, GyT, t.ld, t.width, j, lvss));
}

__global__ void k_adj_prhs(int64_t M, const double* __restrict__ lpt, const double* sum,
                           const double* __restrict__ scale, double* __restrict__ rhs,
                           double* __restrict__ z0) {
  const double mean = *sum / (double)M;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * blockDim.x) {
    rhs[j] = scale[j] * (lpt[j] - mean);
    z0[j] = 0.0;
  }
}

// l_u** += D^(P,V)_x^T (e o z / dt), likewise v
__global__ void k_adj_div(int64_t N, TEll t, const double* __restrict__ PxT,
                          const double* __restrict__ PyT, const double* __restrict__ ze,
                          double* __restrict__ luss, double* __restrict__ lvss) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    luss[i] += tgather(t.idx, PxT, t.ld, t.width, i, ze);
    lvss[i] += tgather(t.idx, PyT, t.ld, t.width, i, ze);
  }
}

// adjoint of b = F/dt on the interior rows (the Neumann rows' right side is 0)
__global__ void k_adj_ze(int64_t M, const double* __restrict__ z, const uint8_t* __restrict__ p_bc,
                         double inv_dt, double* __restrict__ ze) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * blockDim.x)
    ze[j] = p_bc[j] ? 0.0 : z[j] * inv_dt;
}

// wall rows of the viscous right side: wall data and the Kim & Moin term
__global__ void k_adj_wall(int64_t N, const double* __restrict__ lru, const double* __restrict__ lrv,
                           const uint8_t* __restrict__ v_bc, const double* __restrict__ nx,
                           const double* __restrict__ ny, int km, double dt,
                           double* __restrict__ gu, double* __restrict__ gv,
                           double* __restrict__ t1, double* __restrict__ t2,
                           double* __restrict__ t3, double* __restrict__ t4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = lru[i], b = lrv[i];
    if (v_bc[i]) {
      gu[i] += a;
      gv[i] += b;
      t1[i] = 0.0;
      t2[i] = 0.0;
      if (km == 1) {
        const double tx = -ny[i], ty = nx[i];
        const double mu = dt * (tx * a + ty * b);
        t3[i] = tx * mu;
        t4[i] = ty * mu;
      } else if (km == 2) {
        t3[i] = dt * a;
        t4[i] = dt * b;
      } else {
        t3[i] = 0.0;
        t4[i] = 0.0;
      }
    } else {
      t1[i] = a;
      t2[i] = b;
      t3[i] = 0.0;
      t4[i] = 0.0;
    }
  }
}

__global__ void k_adj_ptin(int64_t M, TEll t, const double* __restrict__ GxT,
                           const double* __restrict__ GyT, const double* __restrict__ t3,
                           const double* __restrict__ t4, double* __restrict__ lpt_in) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * blockDim.x)
    lpt_in[j] = tgather(t.idx, GxT, t.ld, t.width, j, t3) + tgather(t.idx, GyT, t.ld, t.width, j, t4);
}

// l_u* = l_r + a Lap^T l_r (interior rows of the viscous right side)
__global__ void k_adj_us(int64_t N, TEll t, const double* __restrict__ LapT,
                         const double* __restrict__ t1, const double* __restrict__ t2, double a,
                         double* __restrict__ lus, double* __restrict__ lvs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    lus[i] = t1[i] + a * tgather(t.idx, LapT, t.ld, t.width, i, t1);
    lvs[i] = t2[i] + a * tgather(t.idx, LapT, t.ld, t.width, i, t2);
  }
}

// Adams-Bashforth: adjoints of C_j and of the input C_{j-1}; products for the convection adjoint
__global__ void k_adj_ab2(int64_t N, const double* __restrict__ lus, const double* __restrict__ lvs,
                          double* __restrict__ lcu_io, double* __restrict__ lcv_io, int first,
                          double dt, const double* __restrict__ u, const double* __restrict__ v,
                          double* __restrict__ lcu, double* __restrict__ lcv,
                          double* __restrict__ t1, double* __restrict__ t2,
                          double* __restrict__ t3, double* __restrict__ t4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = lus[i], b = lvs[i];
    double cu = 1.5 * dt * a + lcu_io[i];
    double cv = 1.5 * dt * b + lcv_io[i];
    if (first) {
      cu += -0.5 * dt * a;
      cv += -0.5 * dt * b;
      lcu_io[i] = 0.0;
      lcv_io[i] = 0.0;
    } else {
      lcu_io[i] = -0.5 * dt * a;
      lcv_io[i] = -0.5 * dt * b;
    }
    lcu[i] = cu;
    lcv[i] = cv;
    t1[i] = u[i] * cu;
    t2[i] = v[i] * cu;
    t3[i] = u[i] * cv;
    t4[i] = v[i] * cv;
  }
}

// convection C(q) = -[u o D_x q + v o D_y q] (adjoint with respect to u, v)
__global__ void k_adj_conv(int64_t N, int64_t ld, int k, const int32_t* __restrict__ idx,
                           const double* __restrict__ Dx, const double* __restrict__ Dy, TEll t,
                           const double* __restrict__ DxT, const double* __restrict__ DyT,
                           const double* __restrict__ u, const double* __restrict__ v,
                           const double* __restrict__ lus, const double* __restrict__ lvs,
                           const double* __restrict__ lcu, const double* __restrict__ lcv,
                           const double* __restrict__ t1, const double* __restrict__ t2,
                           const double* __restrict__ t3, const double* __restrict__ t4,
                           double* __restrict__ lu, double* __restrict__ lv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double dxu = 0, dyu = 0, dxv = 0, dyv = 0;
    for (int s = 0; s < k; ++s) {
      const int32_t j = idx[s * ld + i];
      const double wx = Dx[s * ld + i], wy = Dy[s * ld + i];
      dxu += wx * u[j];
      dyu += wy * u[j];
      dxv += wx * v[j];
      dyv += wy * v[j];
    }
    const double ci = lcu[i], cj = lcv[i];
    lu[i] = lus[i] - dxu * ci - tgather(t.idx, DxT, t.ld, t.width, i, t1) -
            tgather(t.idx, DyT, t.ld, t.width, i, t2) - dxv * cj;
    lv[i] = lvs[i] - dyu * ci - dyv * cj - tgather(t.idx, DxT, t.ld, t.width, i, t3) -
            tgather(t.idx, DyT, t.ld, t.width, i, t4);
  }
}

int palloc_a(rbffd_ctx* ctx, AdjointPlan* a, void** out, size_t bytes) {
  void* ptr = nullptr;
  int rc = check_cuda(ctx, cudaMalloc(&ptr, bytes > 0 ? bytes : 1), "adjoint alloc");
  if (rc) return rc;
  a->allocs.push_back(ptr);
  *out = ptr;
  return RBFFD_OK;
}

// transposed structure of an ELL operator with n_rows rows into n_cols columns
int build_transpose(rbffd_ctx* ctx, AdjointPlan* a, const int32_t* idx, int64_t n_rows, int64_t ld,
                    int k, int64_t n_cols, int grid, TEll* t, cudaStream_t st) {
  int rc = palloc_a(ctx, a, (void**)&t->counts, sizeof(int) * (n_cols + 1));
  if (rc) return rc;
  int* mx = t->counts + n_cols;
  rc = check_cuda(ctx, cudaMemsetAsync(t->counts, 0, sizeof(int) * (n_cols + 1), st), "memset");
  if (rc) return rc;
  k_t_count<<<grid, 256, 0, st>>>(n_rows, ld, k, idx, t->counts);
  k_t_max<<<grid, 256, 0, st>>>(n_cols, t->counts, mx);
  int hmax = 0;
  rc = check_cuda(ctx, cudaMemcpyAsync(&hmax, mx, sizeof(int), cudaMemcpyDeviceToHost, st), "max");
  if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "transpose sync");
  if (rc) return rc;
  t->width = hmax > 0 ? hmax : 1;
  t->ld = round_up(n_cols, 32);
  t->n = n_cols;
  rc = palloc_a(ctx, a, (void**)&t->idx, sizeof(int32_t) * t->width * t->ld);
  if (!rc) rc = palloc_a(ctx, a, (void**)&t->slot, sizeof(int32_t) * t->width * t->ld);
  int* cursor = nullptr;
  if (!rc) rc = palloc_a(ctx, a, (void**)&cursor, sizeof(int) * n_cols);
  if (rc) return rc;
  rc = check_cuda(ctx, cudaMemsetAsync(cursor, 0, sizeof(int) * n_cols, st), "memset");
  if (rc) return rc;
  k_t_fill<<<grid, 256, 0, st>>>(n_rows, ld, k, idx, cursor, t->ld, t->idx, t->slot);
  k_t_sort_pad<<<grid, 256, 0, st>>>(n_cols, t->ld, t->width, t->counts, t->idx, t->slot);
  return check_cuda(ctx, cudaGetLastError(), "transpose kernels");
}

int t_weights(rbffd_ctx* ctx, AdjointPlan* a, const TEll& t, const double* w, int64_t ld,
              const double* rowmul, const double* colmul, double alpha, double** out, int grid,
              cudaStream_t st) {
  int rc = palloc_a(ctx, a, (void**)out, sizeof(double) * t.width * t.ld);
  if (rc) return rc;
  k_t_weights<<<grid, 256, 0, st>>>(t.n, t.ld, t.width, t.idx, t.slot, w, ld, rowmul, colmul,
                                    alpha, *out);
  return check_cuda(ctx, cudaGetLastError(), "transpose weights");
}

int build_adjoint_plan(rbffd_ctx* ctx, StepPlan* P, const rbffd_flow& f, cudaStream_t st) {
  AdjointPlan* a = new AdjointPlan();
  const int G = P->grid, k = P->k;
  int rc = 0;
#define TRYA(x)                \
  do {                         \
    rc = (x);                  \
    if (rc) {                  \
      adjoint_plan_free(a);    \
      return rc;               \
    }                          \
  } while (0)
  TRYA(build_transpose(ctx, a, f.vv_idx, f.N, f.ld_v, k, f.N, G, &a->tvv, st));
  TRYA(build_transpose(ctx, a, f.pv_idx, f.M, f.ld_p, k, f.N, G, &a->tpv, st));
  TRYA(build_transpose(ctx, a, f.vp_idx, f.N, f.ld_v, k, f.M, G, &a->tvp, st));
  TRYA(build_transpose(ctx, a, P->Lidx, f.M, f.ld_p, k, f.M, G, &a->tl, st));
  double* inv_scale = nullptr;
  TRYA(palloc_a(ctx, a, (void**)&a->e, sizeof(double) * f.M));
  TRYA(palloc_a(ctx, a, (void**)&inv_scale, sizeof(double) * f.M));
  TRYA(palloc_a(ctx, a, (void**)&a->es_t, sizeof(double) * f.M));
  k_adj_setup_vec<<<G, 256, 0, st>>>(f.M, f.p_bc, P->scale, a->e, inv_scale);
  TRYA(t_weights(ctx, a, a->tvv, f.vv_dx, f.ld_v, nullptr, nullptr, 1.0, &a->DxT, G, st));
  TRYA(t_weights(ctx, a, a->tvv, f.vv_dy, f.ld_v, nullptr, nullptr, 1.0, &a->DyT, G, st));
  TRYA(t_weights(ctx, a, a->tvv, f.vv_lap, f.ld_v, nullptr, nullptr, 1.0, &a->LapT, G, st));
  TRYA(t_weights(ctx, a, a->tvv, P->Hw, f.ld_v, nullptr, nullptr, 1.0, &a->HwT, G, st));
  TRYA(t_weights(ctx, a, a->tpv, f.pv_dx, f.ld_p, nullptr, nullptr, 1.0, &a->PxT, G, st));
  TRYA(t_weights(ctx, a, a->tpv, f.pv_dy, f.ld_p, nullptr, nullptr, 1.0, &a->PyT, G, st));
  TRYA(t_weights(ctx, a, a->tvp, f.vp_dx, f.ld_v, nullptr, nullptr, 1.0, &a->GxT, G, st));
  TRYA(t_weights(ctx, a, a->tvp, f.vp_dy, f.ld_v, nullptr, nullptr, 1.0, &a->GyT, G, st));
  // S L^T: unscale the forward rows (1/s_row), scale the transposed rows (s_col)
  TRYA(t_weights(ctx, a, a->tl, P->Lw, f.ld_p, inv_scale, P->scale, 1.0, &a->LT, G, st));
  // rank-one column -gamma S 1 with gamma = 1/|sum over boundary rows of s|
  k_sum<double><<<G, kThreads, 0, st>>>(P->scale, f.M, P->gr, P->dscal, a->e);
  k_adj_es<<<G, 256, 0, st>>>(f.M, P->scale, P->dscal, a->es_t);
  TRYA(check_cuda(ctx, cudaGetLastError(), "adjoint set-up"));
  double** vecN[] = {&a->luss, &a->lvss, &a->lru, &a->lrv, &a->t1,  &a->t2,
                     &a->t3,   &a->t4,   &a->lus, &a->lvs, &a->lcu, &a->lcv};
  for (double** v : vecN) TRYA(palloc_a(ctx, a, (void**)v, sizeof(double) * f.N));
  TRYA(palloc_a(ctx, a, (void**)&a->lpt, sizeof(double) * f.M));
  TRYA(palloc_a(ctx, a, (void**)&a->z, sizeof(double) * f.M));
  TRYA(palloc_a(ctx, a, (void**)&a->rhs, sizeof(double) * f.M));
#undef TRYA
  P->adj = a;
  return RBFFD_OK;
}

}  // namespace

int adjoint_run(rbffd_ctx* ctx, const rbffd_flow* fp, const rbffd_state* s, rbffd_adjoint* lam,
                double* grad_gu, double* grad_gv, rbffd_stats* stats, cudaStream_t st) {
  const rbffd_flow& f = *fp;
  const rbffd_flow key = plan_key(f);
  if (ctx->plan && memcmp(&ctx->plan->key, &key, sizeof(rbffd_flow)) != 0) {
    cudaStreamSynchronize(st);
    step_plan_free(ctx->plan);
    ctx->plan = nullptr;
  }
  if (!ctx->plan) {
    int rc = build_plan(ctx, f, &ctx->plan, st);
    if (rc) return rc;
  }
  StepPlan* P = ctx->plan;
  if (P->pdir)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "the adjoint exists for the bordered pressure system only (no Dirichlet rows)");
  if (!P->adj) {
    int rc = build_adjoint_plan(ctx, P, f, st);
    if (rc) return rc;
  }
  AdjointPlan* A = P->adj;
  const int G = P->grid;
  const double a = f.dt / (2.0 * f.Re);
  // correction and its wall overwrite
  k_adj_mask<<<G, kThreads, 0, st>>>(f.N, lam->u, lam->v, f.v_bc, f.overwrite_bc, grad_gu,
                                     grad_gv, A->luss, A->lvss);
  k_adj_pt<<<G, kThreads, 0, st>>>(f.M, A->tvp, A->GxT, A->GyT, A->luss, A->lvss, lam->pt, f.dt,
                                   A->lpt);
  // transposed pressure solve
  k_sum<double><<<G, kThreads, 0, st>>>(A->lpt, f.M, P->gr, P->dscal);
  k_adj_prhs<<<G, kThreads, 0, st>>>(f.M, A->lpt, P->dscal, P->scale, A->rhs, A->z);
  P->launches += 4;
  int rc = check_cuda(ctx, cudaGetLastError(), "adjoint kernels");
  if (rc) return rc;
  KOp<double, double> LT{A->tl.idx, A->LT, A->tl.ld, f.M, A->tl.width, 0, A->es_t, A->e};
  double* zx[1] = {A->z};
  const double* zb[1] = {A->rhs};
  SolveResult pr;
  rc = bicgstab<0, 1, true, double, double>(ctx, P, LT, zx, zb, P->kw64, f.tol, f.max_iter, &pr,
                                            st);
  if (rc) return rc;
  if (stats) {
    stats->poisson_iters += pr.iters;
    stats->poisson_relres = pr.relres;
  }
  if (pr.status == 2) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite adjoint pressure solve");
  if (!pr.converged)
    return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                     "adjoint pressure solve: relative residual %.3e after %d iterations",
                     pr.relres, pr.iters);
  k_adj_ze<<<G, kThreads, 0, st>>>(f.M, A->z, f.p_bc, 1.0 / f.dt, A->rhs);
  k_adj_div<<<G, kThreads, 0, st>>>(f.N, A->tpv, A->PxT, A->PyT, A->rhs, A->luss, A->lvss);
  // transposed viscous solves, two right sides; start from the right sides
  rc = check_cuda(ctx, cudaMemcpyAsync(A->lru, A->luss, sizeof(double) * f.N,
                                       cudaMemcpyDeviceToDevice, st), "copy");
  if (!rc) rc = check_cuda(ctx, cudaMemcpyAsync(A->lrv, A->lvss, sizeof(double) * f.N,
                                                cudaMemcpyDeviceToDevice, st), "copy");
  if (rc) return rc;
  KOp<double, double> HT{A->tvv.idx, A->HwT, A->tvv.ld, f.N, A->tvv.width, 1, nullptr, nullptr};
  double* hx[2] = {A->lru, A->lrv};
  const double* hb[2] = {A->luss, A->lvss};
  SolveResult hr;
  rc = bicgstab<0, 2, false, double, double>(ctx, P, HT, hx, hb, P->kw64, f.tol, f.max_iter, &hr,
                                             st);
  if (rc) return rc;
  if (stats) {
    stats->helm_iters += hr.iters;
    stats->helm_relres = hr.relres;
  }
  if (hr.status == 2) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite adjoint viscous solve");
  if (!hr.converged)
    return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                     "adjoint viscous solve: relative residual %.3e after %d iterations",
                     hr.relres, hr.iters);
  k_adj_wall<<<G, kThreads, 0, st>>>(f.N, A->lru, A->lrv, f.v_bc, f.v_nx, f.v_ny, f.km_mode, f.dt,
                                     grad_gu, grad_gv, A->t1, A->t2, A->t3, A->t4);
  k_adj_ptin<<<G, kThreads, 0, st>>>(f.M, A->tvp, A->GxT, A->GyT, A->t3, A->t4, lam->pt);
  k_adj_us<<<G, kThreads, 0, st>>>(f.N, A->tvv, A->LapT, A->t1, A->t2, a, A->lus, A->lvs);
  k_adj_ab2<<<G, kThreads, 0, st>>>(f.N, A->lus, A->lvs, lam->cu_prev, lam->cv_prev,
                                    s->j == 0 ? 1 : 0, f.dt, s->u, s->v, A->lcu, A->lcv, A->t1,
                                    A->t2, A->t3, A->t4);
  k_adj_conv<<<G, kThreads, 0, st>>>(f.N, f.ld_v, P->k, f.vv_idx, f.vv_dx, f.vv_dy, A->tvv, A->DxT,
                                     A->DyT, s->u, s->v, A->lus, A->lvs, A->lcu, A->lcv, A->t1,
                                     A->t2, A->t3, A->t4, lam->u, lam->v);
  P->launches += 7;
  rc = check_cuda(ctx, cudaGetLastError(), "adjoint kernels");
  if (rc) return rc;
  rc = check_cuda(ctx, cudaStreamSynchronize(st), "adjoint sync");
  if (stats) {
    stats->steps += 1;
  }
  return rc;
}

}  // namespace rbffd
