// Ensembles of independent flows on one staggered node set (rbffd_ensemble_step).
//
// E members (a power of two, at most 64) share every operator of Section 3's
// step and differ in their Reynolds number and wall data.  All vectors are
// member-contiguous: entry (i, e) of a field lives at [i * E + e] (the
// viscous work vectors hold u and v of every member, C = 2E columns, at
// [i * C + c]).  A thread owns one (row, column) pair and keeps its column
// under grid striding (the stride is a multiple of 256 and C divides 256), so
// every stencil weight and index is read once per row and broadcast to the
// row's columns, and every gather of a neighbour's values is one contiguous
// run of C entries: the operator stream is shared by all members.
//
// The step follows the MIXED design of step.cu: explicit stages with FP32
// weights gathering split (hi, lo) FP32 copies of the FP64 fields (reading R9),
// the divergence with FP64 weights, and the two implicit solves as FP64
// iterative refinement (FP64 residuals with FP64 weights) around FP32 BiCGSTAB
// solves with per-column scalars.  The pressure solves are right-
// preconditioned by a batched V-cycle on the multigrid hierarchy of step.cu
// (amg.cuh), with the same rank-one completion of the constant mode per
// column.  Per-column reductions are summed in a fixed order.
#include <cmath>
#include <cstring>
#include <vector>

#include "amg.cuh"
#include "common.cuh"

namespace rbffd {
namespace {

constexpr int kT = 256;        // threads per block
constexpr int kCMax = 128;     // columns of a batched solve (2 x 64 members)
constexpr int kRV = 3;         // values reduced per column
constexpr int kInnerRestart = 50;  // iterations of one inner solve, at most

__device__ __forceinline__ float2 split2e(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// Per-column solve scalars (one batched BiCGSTAB).
struct EScal {
  double rho[kCMax], alpha[kCMax], omega[kCMax], rr[kCMax], bb[kCMax];
  double cp[kCMax], cs[kCMax], kap[2][kCMax], sum_p[kCMax], sum_s[kCMax];
  double tol2;
  int active[kCMax];
  int status[kCMax];  // 0 ok, 1/3 breakdown, 2 non-finite
  int iters, maxit, done, C;
};

struct EReduce {
  double* partials;  // [grid][kRV][C]
  unsigned int* counter;
};

// Per-column reduction of NV values (column = thread index mod C, fixed under
// the loops; thread t is in group g = t / C of the kT / C groups).  In a block,
// the groups are summed by a fixed tree into group 0, which stores the block
// partials; the last block then has every thread sum the partials of blocks
// g, g + G, ... for its column in block order, reduces the groups by the same
// tree and runs fin(column, totals) for every column.  The order of every sum
// is fixed, so the result does not depend on timing.
template <int NV, typename Fin>
__device__ __forceinline__ void col_reduce(double (&v)[NV], int C, EReduce rd, Fin fin) {
  __shared__ double sh[NV][kT];
  __shared__ bool last;
  const int t = threadIdx.x, G = kT / C, g = t / C;
  auto tree = [&]() {  // sh[j][c] = sum over the groups of sh[j][g C + c]
    for (int h = G / 2; h >= 1; h /= 2) {
      if (g < h) {
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[j][t] += sh[j][t + h * C];
      }
      __syncthreads();
    }
  };
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j][t] = v[j];
  __syncthreads();
  tree();
  if (t < C) {
#pragma unroll
    for (int j = 0; j < NV; ++j) rd.partials[((size_t)blockIdx.x * kRV + j) * C + t] = sh[j][t];
  }
  __syncthreads();
  if (t == 0) {
    __threadfence();
    last = atomicAdd(rd.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int c = t % C;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double a = 0.0;
    for (int b = g; b < (int)gridDim.x; b += G)
      a += ((volatile double*)rd.partials)[((size_t)b * kRV + j) * C + c];
    sh[j][t] = a;
  }
  __syncthreads();
  tree();
  if (t < C) {
    double tot[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = sh[j][t];
    fin(t, tot);
  }
  if (t == 0) *rd.counter = 0u;
}

// Items f = i C + c (row i, column c) of a contiguous share of the rows per
// block: thread t takes the items r0 C + t + q kT, so its column is t mod C
// (C divides kT) for the whole loop, and the block walks its rows in order,
// so the gathers of nearby (Morton-ordered) rows find their lines in L1.
#define EFOR(n, C, I)                                                                     \
  const int64_t ef_share = ((int64_t)(n) + gridDim.x - 1) / gridDim.x;                   \
  const int64_t ef_r1 = min((int64_t)(n), ef_share * (blockIdx.x + 1));                  \
  const int ef_c = (int)threadIdx.x % (C), ef_step = kT / (C);                           \
  for (int64_t I = min((int64_t)(n), ef_share * blockIdx.x) + (int)threadIdx.x / (C),     \
               f = I * (C) + ef_c;                                                       \
       I < ef_r1; I += ef_step, f += kT)

// The same items for the gathering kernels, in another row order: row group
// g = t / C of the kT / C groups walks its own contiguous part of the block's
// rows one after the other, so a warp's consecutive rows are neighbours in
// the (Morton) node order and find most of their stencil's operand lines
// still in L1 from the row before.  The column is t mod C, as in EFOR.
#define EFOR_SEQ(n, C, I)                                                                 \
  const int64_t es_share = ((int64_t)(n) + gridDim.x - 1) / gridDim.x;                   \
  const int64_t es_r0 = min((int64_t)(n), es_share * blockIdx.x);                        \
  const int64_t es_r1 = min((int64_t)(n), es_share * (blockIdx.x + 1));                  \
  const int es_groups = kT / (C);                                                        \
  const int64_t es_sub = (es_share + es_groups - 1) / es_groups;                         \
  const int ef_c = (int)threadIdx.x % (C);                                               \
  const int64_t es_a = min(es_r1, es_r0 + es_sub * ((int)threadIdx.x / (C)));             \
  const int64_t es_b = min(es_r1, es_a + es_sub);                                        \
  for (int64_t I = es_a, f = es_a * (C) + ef_c; I < es_b; ++I, f += (C))

// ------------------------------------------------------------ explicit stages
// sum_s w[s][i] (x2[j][c] - x2[ref][c]) over split FP32 copies
// (K > 0: the stencil size at compile time, every gather issued at once)
template <int K>
__device__ __forceinline__ float gsplit(const int32_t* idx, const float* w, int64_t ld, int k,
                                        int64_t i, const float2* x2, int C, int c) {
  const float2 ref = x2[(int64_t)idx[i] * C + c];
  float acc = 0.f;
  const int kk = K > 0 ? K : k;
#pragma unroll(K > 0 ? K : 1)
  for (int s = 0; s < kk; ++s) {
    const float2 xj = x2[(int64_t)idx[s * ld + i] * C + c];
    acc += w[s * ld + i] * ((xj.x - ref.x) + (xj.y - ref.y));
  }
  return acc;
}

// Stage 1 (AB2 convection) for every member.
template <int K>
__global__ void __launch_bounds__(kT)
    e_convect(int64_t N, int64_t ld, int k, int E, const int32_t* __restrict__ idx,
              const float* __restrict__ wdx, const float* __restrict__ wdy,
              const double* __restrict__ u, const double* __restrict__ v,
              const float2* __restrict__ u2, const float2* __restrict__ v2,
              double* __restrict__ cu_prev, double* __restrict__ cv_prev, double* __restrict__ us,
              double* __restrict__ vs, float2* __restrict__ us2, float2* __restrict__ vs2,
              double dt, int first) {
  EFOR(N, E, i) {
    const int c = ef_c;
    const double ux = gsplit<K>(idx, wdx, ld, k, i, u2, E, c), uy = gsplit<K>(idx, wdy, ld, k, i, u2, E, c);
    const double vx = gsplit<K>(idx, wdx, ld, k, i, v2, E, c), vy = gsplit<K>(idx, wdy, ld, k, i, v2, E, c);
    const double ui = u[f], vi = v[f];
    const double cu = -(ui * ux + vi * uy), cv = -(ui * vx + vi * vy);
    const double cup = first ? cu : cu_prev[f], cvp = first ? cv : cv_prev[f];
    const double a = ui + dt * (1.5 * cu - 0.5 * cup), b = vi + dt * (1.5 * cv - 0.5 * cvp);
    us[f] = a;
    vs[f] = b;
    us2[f] = split2e(a);
    vs2[f] = split2e(b);
    cu_prev[f] = cu;
    cv_prev[f] = cv;
  }
}

// Stage 2 right side into the viscous layout (column e: u of member e, E + e:
// v): inside u* + a_e D_Lap (u* or u_j); walls: wall data (+ Kim & Moin term).
template <int K>
__global__ void __launch_bounds__(kT, 2)
    e_helm_rhs(int64_t N, int64_t ldv, int k, int E, const int32_t* __restrict__ vv_idx,
               const float* __restrict__ lap, const double* __restrict__ us,
               const double* __restrict__ vs, const float2* __restrict__ q2u,
               const float2* __restrict__ q2v, const int32_t* __restrict__ vp_idx,
               const float* __restrict__ gdx, const float* __restrict__ gdy,
               const float2* __restrict__ pt2, const uint8_t* __restrict__ v_bc,
               const double* __restrict__ v_nx, const double* __restrict__ v_ny,
               const double* __restrict__ gu, const double* __restrict__ gv,
               const double* __restrict__ a_col, double dt, int km,
               double* __restrict__ rhs, double* __restrict__ x0) {
  const int C = 2 * E;
  EFOR(N, E, i) {
    const int e = ef_c;
    double bu, bv;
    if (!v_bc[i]) {
      const double a = a_col[e];
      bu = us[f] + a * gsplit<K>(vv_idx, lap, ldv, k, i, q2u, E, e);
      bv = vs[f] + a * gsplit<K>(vv_idx, lap, ldv, k, i, q2v, E, e);
    } else {
      bu = gu[f];
      bv = gv[f];
      if (km) {
        const double gx = gsplit<K>(vp_idx, gdx, ldv, k, i, pt2, E, e);
        const double gy = gsplit<K>(vp_idx, gdy, ldv, k, i, pt2, E, e);
        if (km == 1) {
          const double tx = -v_ny[i], ty = v_nx[i], gt = tx * gx + ty * gy;
          bu += dt * gt * tx;
          bv += dt * gt * ty;
        } else {
          bu += dt * gx;
          bv += dt * gy;
        }
      }
    }
    rhs[i * C + e] = bu;
    rhs[i * C + E + e] = bv;
    x0[i * C + e] = bu;
    x0[i * C + E + e] = bv;
  }
}

// Stage 3a: F = D^(P,V) u** (FP64 weights), scaled right side of the pressure
// solve (0 on the Neumann rows)
template <int K>
__global__ void __launch_bounds__(kT)
    e_divergence(int64_t M, int64_t ldp, int k, int E, const int32_t* __restrict__ idx,
                 const double* __restrict__ wdx, const double* __restrict__ wdy,
                 const double* __restrict__ xv, const uint8_t* __restrict__ p_bc,
                 const double* __restrict__ scale, double inv_dt, double* __restrict__ b) {
  const int C = 2 * E;
  EFOR(M, E, i) {
    const int e = ef_c;
    double acc = 0.0;
    const int kk = K > 0 ? K : k;
#pragma unroll(K > 0 ? K : 1)
    for (int s = 0; s < kk; ++s) {
      const int64_t j = idx[s * ldp + i];
      acc += wdx[s * ldp + i] * xv[j * C + e] + wdy[s * ldp + i] * xv[j * C + E + e];
    }
    b[f] = p_bc[i] ? 0.0 : scale[i] * acc * inv_dt;
  }
}

// Stage 3c: p~ = x - mean(x) per member; p = p~ - a_e D^(P,P)_Lap p~
template <int K>
__global__ void __launch_bounds__(kT)
    e_pressure(int64_t M, int64_t ldp, int k, int E, const int32_t* __restrict__ idx,
               const float* __restrict__ lap, const double* __restrict__ x,
               const float2* __restrict__ x2, const double* __restrict__ mean,
               const double* __restrict__ a_col, double* __restrict__ pt, double* __restrict__ p,
               float2* __restrict__ pt2) {
  EFOR(M, E, i) {
    const int e = ef_c;
    const double v = x[f] - mean[e];
    pt[f] = v;
    p[f] = v - a_col[e] * gsplit<K>(idx, lap, ldp, k, i, x2, E, e);
    pt2[f] = split2e(v);
  }
}

// Stage 3d: u = u** - dt D^(V,P) p~; wall nodes set to the wall data
template <int K>
__global__ void __launch_bounds__(kT)
    e_correct(int64_t N, int64_t ldv, int k, int E, const int32_t* __restrict__ idx,
              const float* __restrict__ gdx, const float* __restrict__ gdy,
              const float2* __restrict__ pt2, const double* __restrict__ xv,
              const uint8_t* __restrict__ v_bc, const double* __restrict__ gu,
              const double* __restrict__ gv, double dt, int overwrite, double* __restrict__ u,
              double* __restrict__ v, float2* __restrict__ u2, float2* __restrict__ v2) {
  const int C = 2 * E;
  EFOR(N, E, i) {
    const int e = ef_c;
    double un = xv[i * C + e] - dt * gsplit<K>(idx, gdx, ldv, k, i, pt2, E, e);
    double vn = xv[i * C + E + e] - dt * gsplit<K>(idx, gdy, ldv, k, i, pt2, E, e);
    if (overwrite && v_bc[i]) {
      un = gu[f];
      vn = gv[f];
    }
    u[f] = un;
    v[f] = vn;
    u2[f] = split2e(un);
    v2[f] = split2e(vn);
  }
}

// Initial guess of a solve by extrapolation in time from a ring of earlier
// solutions h[0] (the previous step's), h[1], ... (newest first):
// x = sum_k (-1)^k C(ord + 1, k + 1) h[k], the polynomial of degree ord through
// the last ord + 1 solutions at the next step.  Rows with skip[i / per] set
// (Dirichlet rows) keep the value the caller wrote (their data).
constexpr int kEHist = 4;  // the previous solution and three older ones: cubic
struct EHist {
  const double* h[kEHist];
};
__global__ void e_extrapolate(int64_t n, int ord, EHist H, const uint8_t* __restrict__ skip,
                              int per, double* __restrict__ x) {
  double c[kEHist];
  double b = ord + 1.0;  // C(ord + 1, k + 1) with alternating signs
  for (int k = 0; k <= ord; ++k) {
    c[k] = (k & 1) ? -b : b;
    b = b * (ord - k) / (k + 2.0);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (skip && skip[i / per]) continue;
    double y = 0.0;
    for (int k = 0; k <= ord; ++k) y += c[k] * H.h[k][i];
    x[i] = y;
  }
}

__global__ void e_split(int64_t n, const double* __restrict__ x, float2* __restrict__ x2) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    x2[i] = split2e(x[i]);
}

// per-column sum of x (n rows, C columns) into out[c] / n (the mean)
__global__ void __launch_bounds__(kT)
    e_colmean(int64_t n, int C, const double* __restrict__ x, EReduce rd, double* out) {
  double v[1] = {0.0};
  EFOR(n, C, row) v[0] += x[f];
  col_reduce<1>(v, C, rd, [&](int c, double* t) { out[c] = t[0] / (double)n; });
}

// ---------------------------------------------------------- batched operators
// Viscous columns: y_c = x_c - a_c (Lz x_c) (Lz: the Laplacian with zero wall
// rows).  Pressure columns: y_c = S L z_c + kap_c (S L 1) + es mu_c.
struct EOp {
  const int32_t* idx;
  int64_t ld, n;
  int k;
  int visc;             // 1: viscous, 0: pressure
  const float* a;       // viscous: a per column
  const float* es;      // pressure: rank-one column
  const float* a1;      // pressure: row sums
};

template <int K>
__device__ __forceinline__ float erow32(const EOp& op, const float* w, int64_t i, const float* x,
                                      int C, int c) {
  float acc = 0.f;
  const int kk = K > 0 ? K : op.k;
#pragma unroll(K > 0 ? K : 1)
  for (int s = 0; s < kk; ++s) acc += w[s * op.ld + i] * x[(int64_t)op.idx[s * op.ld + i] * C + c];
  return acc;
}

// ---------------------------------------------------------- batched BiCGSTAB
// r = b (x0 = 0); rh = r; p = r; rho = (rh, r); rr; bb; (c . p) for the pressure
__global__ void __launch_bounds__(kT)
    e_init(int64_t n, int C, const float* __restrict__ b, float* __restrict__ r,
           float* __restrict__ rh, float* __restrict__ p, float* __restrict__ x,
           const float* __restrict__ cnode, EScal* sc, EReduce rd, double tol2, int maxit) {
  double v[3] = {0.0, 0.0, 0.0};
  EFOR(n, C, i) {
    const float bi = b[f];
    r[f] = bi;
    rh[f] = bi;
    p[f] = bi;
    x[f] = 0.f;
    v[0] += (double)bi * bi;
    v[1] += cnode ? (double)cnode[i] * bi : 0.0;
  }
  col_reduce<3>(v, C, rd, [&](int c, double* t) {
    sc->rr[c] = t[0];
    sc->bb[c] = t[0];
    sc->rho[c] = t[0];
    sc->cp[c] = t[1];
    sc->alpha[c] = 1.0;
    sc->omega[c] = 1.0;
    sc->status[c] = isfinite(t[0]) ? 0 : 2;
    sc->active[c] = (isfinite(t[0]) && t[0] > 0.0) ? 1 : 0;
    if (c == 0) {
      sc->tol2 = tol2;
      sc->maxit = maxit;
      sc->iters = 0;
      sc->done = 0;
      sc->C = C;
    }
  });
}

// v = A zp (+ rank-one terms); reduce (rh, v) -> alpha
template <int K>
__global__ void __launch_bounds__(kT)
    e_spmv_v(EOp op, const float* __restrict__ w, const float* __restrict__ zp,
             float* __restrict__ v, const float* __restrict__ rh, EScal* sc, EReduce rd) {
  if (sc->done) return;
  const int C = sc->C;
  // this thread's column is fixed: its scalars are read once
  const int c0 = (int)threadIdx.x % C;
  const bool act = sc->active[c0] != 0;
  const float ac = op.visc ? op.a[c0] : 0.f;
  const float kap = op.visc ? 0.f : (float)sc->kap[0][c0];
  const float sig = op.visc ? 0.f : (float)sc->sum_p[c0];
  double acc[1] = {0.0};
  if (act) {
    EFOR_SEQ(op.n, C, i) {
      float y = erow32<K>(op, w, i, zp, C, ef_c);
      if (op.visc)
        y = zp[f] - ac * y;
      else
        y += kap * op.a1[i] + op.es[i] * sig;
      v[f] = y;
      acc[0] += (double)rh[f] * y;
    }
  }
  col_reduce<1>(acc, C, rd, [&](int c, double* t) {
    if (!sc->active[c]) return;
    if (t[0] == 0.0 || !isfinite(t[0])) {
      sc->active[c] = 0;
      sc->status[c] = isfinite(t[0]) ? 1 : 2;
      return;
    }
    sc->alpha[c] = sc->rho[c] / t[0];
  });
}

// s = r - alpha v; reduce (c . s) for the pressure
__global__ void __launch_bounds__(kT)
    e_update_s(int64_t n, const float* __restrict__ r, const float* __restrict__ v,
               float* __restrict__ s, const float* __restrict__ cnode, EScal* sc, EReduce rd) {
  if (sc->done) return;
  const int C = sc->C;
  const int c0 = (int)threadIdx.x % C;
  const bool act = sc->active[c0] != 0;
  const float al = (float)sc->alpha[c0];
  double acc[1] = {0.0};
  if (act) {
    EFOR(n, C, i) {
      const float si = r[f] - al * v[f];
      s[f] = si;
      if (cnode) acc[0] += (double)cnode[i] * si;
    }
  }
  col_reduce<1>(acc, C, rd, [&](int c, double* t) { sc->cs[c] = t[0]; });
}

// t = A zs; reduce (t, s), (t, t) -> omega
template <int K>
__global__ void __launch_bounds__(kT)
    e_spmv_t(EOp op, const float* __restrict__ w, const float* __restrict__ zs,
             float* __restrict__ tv, const float* __restrict__ s, EScal* sc, EReduce rd) {
  if (sc->done) return;
  const int C = sc->C;
  const int c0 = (int)threadIdx.x % C;
  const bool act = sc->active[c0] != 0;
  const float ac = op.visc ? op.a[c0] : 0.f;
  const float kap = op.visc ? 0.f : (float)sc->kap[1][c0];
  const float sig = op.visc ? 0.f : (float)sc->sum_s[c0];
  double acc[2] = {0.0, 0.0};
  if (act) {
    EFOR_SEQ(op.n, C, i) {
      float y = erow32<K>(op, w, i, zs, C, ef_c);
      if (op.visc)
        y = zs[f] - ac * y;
      else
        y += kap * op.a1[i] + op.es[i] * sig;
      tv[f] = y;
      acc[0] += (double)y * s[f];
      acc[1] += (double)y * y;
    }
  }
  col_reduce<2>(acc, C, rd, [&](int c, double* t) {
    if (!sc->active[c]) return;
    if (!(t[1] > 0.0) || !isfinite(t[0])) {
      sc->active[c] = 0;
      sc->status[c] = isfinite(t[1]) ? 3 : 2;
      return;
    }
    sc->omega[c] = t[0] / t[1];
  });
}

// x += alpha zp + omega zs; r = s - omega t; reduce (rh, r), (r, r); beta
__global__ void __launch_bounds__(kT)
    e_update_xr(int64_t n, float* __restrict__ x, float* __restrict__ r,
                const float* __restrict__ rh, const float* __restrict__ zp,
                const float* __restrict__ zs, const float* __restrict__ s,
                const float* __restrict__ tv, int pc, EScal* sc, EReduce rd) {
  if (sc->done) return;
  const int C = sc->C;
  const int c0 = (int)threadIdx.x % C;
  const bool act = sc->active[c0] != 0;
  const float al = (float)sc->alpha[c0], om = (float)sc->omega[c0];
  const float kp = pc ? (float)sc->kap[0][c0] : 0.f, ks = pc ? (float)sc->kap[1][c0] : 0.f;
  double acc[2] = {0.0, 0.0};
  if (act) {
    EFOR(n, C, i) {
      x[f] += al * (zp[f] + kp) + om * (zs[f] + ks);
      const float ri = s[f] - om * tv[f];
      r[f] = ri;
      acc[0] += (double)rh[f] * ri;
      acc[1] += (double)ri * ri;
    }
  }
  col_reduce<2>(acc, C, rd, [&](int c, double* t) {
    if (sc->active[c]) {
      sc->rr[c] = t[1];
      const double rho_new = t[0];
      if (!isfinite(t[1])) {
        sc->active[c] = 0;
        sc->status[c] = 2;
      } else if (t[1] <= sc->tol2 * sc->bb[c]) {
        sc->active[c] = 0;
      } else if (rho_new == 0.0 || sc->omega[c] == 0.0) {
        sc->active[c] = 0;
        sc->status[c] = 1;
      } else {
        sc->alpha[c] = (rho_new / sc->rho[c]) * (sc->alpha[c] / sc->omega[c]);  // beta
        sc->rho[c] = rho_new;
      }
    }
    if (c == 0) ++sc->iters;
  });
}

// p = r + beta (p - omega v); reduce (c . p) for the pressure; done flag
__global__ void __launch_bounds__(kT)
    e_update_p(int64_t n, float* __restrict__ p, const float* __restrict__ r,
               const float* __restrict__ v, const float* __restrict__ cnode, EScal* sc,
               EReduce rd) {
  if (sc->done) return;
  const int C = sc->C;
  const int c0 = (int)threadIdx.x % C;
  const bool act = sc->active[c0] != 0;
  const float be = (float)sc->alpha[c0], om = (float)sc->omega[c0];
  double acc[1] = {0.0};
  if (act) {
    EFOR(n, C, i) {
      const float pi = r[f] + be * (p[f] - om * v[f]);
      p[f] = pi;
      if (cnode) acc[0] += (double)cnode[i] * pi;
    }
  }
  col_reduce<1>(acc, C, rd, [&](int c, double* t) {
    if (sc->active[c]) sc->cp[c] = t[0];
    if (c == sc->C - 1) {
      int any = 0;
      for (int q = 0; q < sc->C; ++q) any |= sc->active[q];
      if (!any || sc->iters >= sc->maxit) sc->done = 1;
    }
  });
}

// ------------------------------------------------------------ batched V-cycle
// r0[p][c] = c_p v[perm0[p]][c] - mu_c ce_p,  mu_c = (c . v)_c / (c . es)
__global__ void __launch_bounds__(kT)
    e_pc_in(int64_t M, int C, const float* __restrict__ v, const float* __restrict__ cl,
            const float* __restrict__ ce, const int32_t* __restrict__ perm0, int which,
            double inv_ces, const EScal* sc, float* __restrict__ r0) {
  if (sc->done) return;
  const int c0 = (int)threadIdx.x % C;
  const float mu = (float)((which ? sc->cs[c0] : sc->cp[c0]) * inv_ces);
  EFOR(M, C, p) r0[f] = cl[p] * v[(int64_t)perm0[p] * C + ef_c] - mu * ce[p];
}

// Pre-smoothing from zero (x = omega D^-1 r) and restriction of its residual
// to the aggregates: thread (aggregate I, column c) takes I's rows in order.
template <int W>
__global__ void __launch_bounds__(kT)
    e_pc_restrict(AmgLevel F, int64_t nagg, int C, const float* __restrict__ r,
                  float* __restrict__ x, float* __restrict__ rc, const EScal* sc) {
  if (sc->done) return;
  EFOR_SEQ(nagg, C, I) {
    const int c = ef_c;
    float acc = 0.f;
    for (int32_t i = F.cptr[I]; i < F.cptr[I + 1]; ++i) {
      const float ri = r[(int64_t)i * C + c];
      const float xi = F.wd[i] * ri;
      x[(int64_t)i * C + c] = xi;
      float ax = F.diag[i] * xi;
      if constexpr (W > 0) {  // every load of the row in flight at once
#pragma unroll
        for (int s = 0; s < W; ++s) {
          if (s < F.width) {
            const int32_t j = F.idx[s * F.ld + i];
            ax += F.val[s * F.ld + i] * (F.wd[j] * r[(int64_t)j * C + c]);
          }
        }
      } else {
        for (int s = 0; s < F.width; ++s) {
          const int32_t j = F.idx[s * F.ld + i];
          ax += F.val[s * F.ld + i] * (F.wd[j] * r[(int64_t)j * C + c]);
        }
      }
      acc += ri - ax;
    }
    rc[f] = acc;
  }
}

// Coarsest level: z = X r for the C columns (X: nc x nc, the dense inverse)
// as a tiled product.  A block takes TR rows of z and every column; thread t
// keeps column t mod C and the rows g, g + G, ... of the tile (G = kT / C
// groups).  X and r move through shared memory in slabs of kcj columns of X
// (rows of r); the next slab's loads are issued into registers before the
// current slab's products, so the loads overlap the arithmetic.  Every output
// sums its products in j order, as the plain dot product does.  Then the
// correction of the next finer level's rows of aggregate `row` (has_fine), or
// z itself.
constexpr int kCJ = 32;
constexpr int kCoarseRows = 16;  // TR for C >= 16 (fewer columns: one row per thread)
constexpr int kPre = 8;          // slab values a thread prefetches, per operand

__global__ void __launch_bounds__(kT)
    e_pc_coarse(int64_t nc, int C, const float* __restrict__ X, const float* __restrict__ r,
                float* __restrict__ z, AmgLevel Fine, float* __restrict__ xfine, int has_fine,
                const EScal* sc) {
  if (sc->done) return;
  __shared__ float xs[kT * kPre + kT];  // TR x kcj slab of X, rows padded by one
  __shared__ float rs[kCJ * 64];        // kcj x C slab of r (C <= 64)
  const int G = kT / C;
  const int TR = G > kCoarseRows ? G : kCoarseRows;
  const int kcj = kT * kPre / TR < kCJ ? kT * kPre / TR : kCJ;  // TR kcj <= kT kPre
  const int RPT = TR / G;  // rows per thread, <= kCoarseRows / 4
  const int t = (int)threadIdx.x, c = t % C, g = t / C;
  const int64_t row0 = (int64_t)blockIdx.x * TR;
  float acc[kCoarseRows / 4] = {};
  float px[kPre], pr[kPre];
  auto load = [&](int64_t j0) {
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int e = t + k * kT;
      if (e < TR * kcj) {
        const int rr = e / kcj, jj = e % kcj;
        px[k] = (row0 + rr < nc && j0 + jj < nc) ? X[(row0 + rr) * nc + j0 + jj] : 0.f;
      }
      if (e < kcj * C) {
        const int jj = e / C, cc = e % C;
        pr[k] = (j0 + jj < nc) ? r[(j0 + jj) * C + cc] : 0.f;
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int e = t + k * kT;
      if (e < TR * kcj) xs[(e / kcj) * (kcj + 1) + e % kcj] = px[k];
      if (e < kcj * C) rs[e] = pr[k];
    }
  };
  load(0);
  for (int64_t j0 = 0; j0 < nc; j0 += kcj) {
    store();
    __syncthreads();
    if (j0 + kcj < nc) load(j0 + kcj);
    const int jn = (int)(nc - j0 < kcj ? nc - j0 : kcj);
    for (int jj = 0; jj < jn; ++jj) {
      const float rv = rs[jj * C + c];
#pragma unroll
      for (int q = 0; q < kCoarseRows / 4; ++q)
        if (q < RPT) acc[q] += xs[(g + q * G) * (kcj + 1) + jj] * rv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kCoarseRows / 4; ++q) {
    const int64_t row = row0 + g + q * G;
    if (q >= RPT || row >= nc) continue;
    if (has_fine) {
      const float v = kAmgCoarseScale * acc[q];
      for (int32_t i = Fine.cptr[row]; i < Fine.cptr[row + 1]; ++i) xfine[(int64_t)i * C + c] += v;
    } else {
      z[row * C + c] = acc[q];
    }
  }
}

// Post-smoothing z = x + omega D^-1 (r - G x) on a level whose x holds the
// coarse correction; above level 0 it corrects the finer level's rows of each
// aggregate (x_fine += scale z), on level 0 it writes z in P-node order and
// reduces its per-column sum (for B v = z - mean(z) + mu / M)
template <int W>
__global__ void __launch_bounds__(kT)
    e_pc_up(AmgLevel F, int C, const float* __restrict__ r, const float* __restrict__ x,
            AmgLevel Fine, float* __restrict__ xfine, int level0,
            const int32_t* __restrict__ perm0, float* __restrict__ zout, int which,
            double inv_ces, double inv_R, EScal* sc, EReduce rd) {
  if (sc->done) return;
  double acc[1] = {0.0};
  EFOR_SEQ(F.n, C, i) {
    const int c = ef_c;
    const float xi = x[f];
    float ax = F.diag[i] * xi;
    if constexpr (W > 0) {
#pragma unroll
      for (int s = 0; s < W; ++s) {
        if (s < F.width) {
          const int32_t j = F.idx[s * F.ld + i];
          ax += F.val[s * F.ld + i] * x[(int64_t)j * C + c];
        }
      }
    } else {
      for (int s = 0; s < F.width; ++s) {
        const int32_t j = F.idx[s * F.ld + i];
        ax += F.val[s * F.ld + i] * x[(int64_t)j * C + c];
      }
    }
    const float zi = xi + F.wd[i] * (r[f] - ax);
    if (level0) {
      zout[(int64_t)perm0[i] * C + c] = zi;
      acc[0] += zi;
    } else {
      const float v = kAmgCoarseScale * zi;
      for (int32_t q = Fine.cptr[i]; q < Fine.cptr[i + 1]; ++q) xfine[(int64_t)q * C + c] += v;
    }
  }
  if (!level0) return;
  col_reduce<1>(acc, C, rd, [&](int c, double* t) {
    const double mu = (which ? sc->cs[c] : sc->cp[c]) * inv_ces;
    sc->kap[which][c] = (mu - t[0]) * inv_R;
    if (which)
      sc->sum_s[c] = mu;
    else
      sc->sum_p[c] = mu;
  });
}

// Without levels below the coarsest one, its result z (level-0 order) is
// mapped to P-node order and completed like e_pc_up's level 0
__global__ void __launch_bounds__(kT)
    e_pc_fin(int64_t M, int C, const float* __restrict__ z0, const int32_t* __restrict__ perm0,
             float* __restrict__ zout, int which, double inv_ces, double inv_R, EScal* sc,
             EReduce rd) {
  if (sc->done) return;
  double acc[1] = {0.0};
  EFOR(M, C, q) {
    const int c = ef_c;
    zout[(int64_t)perm0[q] * C + c] = z0[f];
    acc[0] += z0[f];
  }
  col_reduce<1>(acc, C, rd, [&](int c, double* t) {
    const double mu = (which ? sc->cs[c] : sc->cp[c]) * inv_ces;
    sc->kap[which][c] = (mu - t[0]) * inv_R;
    if (which)
      sc->sum_s[c] = mu;
    else
      sc->sum_p[c] = mu;
  });
}

// ------------------------------------------------------------- refinement
// r = b - A x in FP64 (FP64 weights); per-column (r, r), (b, b)
template <int K>
__global__ void __launch_bounds__(kT)
    e_residual64(EOp op, const double* __restrict__ w, const double* __restrict__ ad,
                 const double* __restrict__ esd, const double* __restrict__ x,
                 const double* __restrict__ b, double* __restrict__ r,
                 const double* __restrict__ xsum, int C, EReduce rd, double* out) {
  double acc[2] = {0.0, 0.0};
  EFOR_SEQ(op.n, C, i) {
    const int c = ef_c;
    double y = 0.0;
    const int kk = K > 0 ? K : op.k;
#pragma unroll(K > 0 ? K : 1)
    for (int s = 0; s < kk; ++s) y += w[s * op.ld + i] * x[(int64_t)op.idx[s * op.ld + i] * C + c];
    if (op.visc)
      y = x[f] - ad[c] * y;
    else
      y += esd[i] * xsum[c];
    const double ri = b[f] - y;
    r[f] = ri;
    acc[0] += ri * ri;
    acc[1] += b[f] * b[f];
  }
  col_reduce<2>(acc, C, rd, [&](int c, double* t) {
    out[2 * c] = t[0];
    out[2 * c + 1] = t[1];
  });
}

// per-column sum of x (the rank-one term of the scaled pressure operator)
__global__ void __launch_bounds__(kT)
    e_colsum(int64_t n, int C, const double* __restrict__ x, EReduce rd, double* out) {
  double v[1] = {0.0};
  EFOR(n, C, row) v[0] += x[f];
  col_reduce<1>(v, C, rd, [&](int c, double* t) { out[c] = t[0]; });
}

__global__ void e_to32(int64_t n, int C, const double* __restrict__ r, const double* __restrict__ sc,
                       float* __restrict__ r32) {
  EFOR(n, C, row) {
    const int c = ef_c;
    r32[f] = (float)(r[f] * sc[c]);
  }
}

__global__ void e_addcorr(int64_t n, int C, double* __restrict__ x, const float* __restrict__ e32,
                          const double* __restrict__ nrm) {
  EFOR(n, C, row) {
    const int c = ef_c;
    x[f] += nrm[c] * (double)e32[f];
  }
}

__global__ void e_scale_rows(int64_t n, int64_t ld, int k, const uint8_t* __restrict__ v_bc,
                             const double* __restrict__ lap, double* __restrict__ lz) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    for (int s = 0; s < k; ++s) lz[s * ld + i] = v_bc[i] ? 0.0 : lap[s * ld + i];
}

__global__ void e_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    y[i] = (float)x[i];
}

}  // namespace

// ------------------------------------------------------------------ the plan
struct EnsPlan {
  rbffd_flow key;
  int E = 0, k = 0, grid = 0;
  int64_t N = 0, M = 0;
  std::vector<void*> allocs;
  Amg* amg = nullptr;
  // shared operators
  int32_t* Lidx = nullptr;
  double *Lw = nullptr, *es = nullptr, *scale = nullptr, *lz = nullptr;
  float *Lw32 = nullptr, *es32 = nullptr, *a1_32 = nullptr, *lz32 = nullptr;
  float *vv_dx32 = nullptr, *vv_dy32 = nullptr, *vv_lap32 = nullptr, *pp_lap32 = nullptr,
        *vp_dx32 = nullptr, *vp_dy32 = nullptr;
  // member-contiguous work
  double *us = nullptr, *vs = nullptr, *rhs = nullptr, *xv = nullptr, *pb = nullptr, *px = nullptr;
  float2 *u2 = nullptr, *v2 = nullptr, *us2 = nullptr, *vs2 = nullptr, *pt2 = nullptr, *px2 = nullptr;
  double *r64 = nullptr, *aV = nullptr, *aE = nullptr, *nrm = nullptr, *isc = nullptr,
         *xsum = nullptr, *h2 = nullptr, *mean = nullptr;
  float *aV32 = nullptr;
  float* kw[9] = {};  // x r rh p v s t zp zs (FP32, C columns)
  float *r32 = nullptr;
  // batched V-cycle work per level (r, x) and the coarse r, z
  float* lr[kAmgMaxLevels + 1] = {};
  float* lx[kAmgMaxLevels + 1] = {};
  // rings of earlier solutions for the initial guesses (newest at index
  // head): viscous (C columns) and pressure (E columns); n*: how many hold
  // solutions of consecutive steps ending at the state's previous step
  double* vh[kEHist] = {};
  double* ph[kEHist] = {};
  int nvh = 0, nph = 0, hv = 0, hp = 0;
  int64_t last_j = -1;  // the state's step index after this plan's last step
  EScal* sc = nullptr;
  EScal* sc_t = nullptr;  // scalars of the timed SpMV launches (profile)
  EReduce rd{};
  int64_t launches = 0;
};

void ens_plan_free(EnsPlan* p) {
  if (!p) return;
  amg_free(p->amg);
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

namespace {

template <typename T>
int ealloc(rbffd_ctx* ctx, EnsPlan* p, T** out, size_t count) {
  void* ptr = nullptr;
  int rc = check_cuda(ctx, cudaMalloc(&ptr, sizeof(T) * (count ? count : 1)), "ensemble alloc");
  if (rc) return rc;
  p->allocs.push_back(ptr);
  *out = (T*)ptr;
  return RBFFD_OK;
}

// kern<28> when the stencil size k is 28 (every gather of a row unrolled and
// issued at once), kern<0> (runtime size) otherwise
#define EK(kern, grid, ...)                                      \
  do {                                                           \
    if (k == 28)                                                 \
      kern<28><<<grid, kT, 0, st>>>(__VA_ARGS__);                \
    else                                                         \
      kern<0><<<grid, kT, 0, st>>>(__VA_ARGS__);                 \
  } while (0)

// kern<8> / kern<16> for graph rows of at most that width (slots unrolled
// and predicated), kern<0> (plain loop) for wider ones
#define EW(kern, width, ...)                                     \
  do {                                                           \
    if ((width) <= 8)                                            \
      kern<8><<<G, kT, 0, st>>>(__VA_ARGS__);                    \
    else if ((width) <= 16)                                      \
      kern<16><<<G, kT, 0, st>>>(__VA_ARGS__);                   \
    else                                                         \
      kern<0><<<G, kT, 0, st>>>(__VA_ARGS__);                    \
  } while (0)

int ens_to32(rbffd_ctx* ctx, EnsPlan* p, const double* src, int64_t n, float** dst,
             cudaStream_t st) {
  int rc = ealloc(ctx, p, dst, n);
  if (rc) return rc;
  e_f32<<<p->grid, kT, 0, st>>>(n, src, *dst);
  return check_cuda(ctx, cudaGetLastError(), "ensemble to_f32");
}

// The scaled pressure operator of step.cu (same rows, same scaling, same
// rank-one column), built from the flow's FP64 operators.
__global__ void e_build_poisson(int64_t M, int64_t ld, int k, const int32_t* __restrict__ idx,
                                const double* __restrict__ lap, const uint8_t* __restrict__ p_bc,
                                const int32_t* __restrict__ bmap, int64_t ld_b,
                                const int32_t* __restrict__ pn_idx,
                                const double* __restrict__ pn_dx, const double* __restrict__ pn_dy,
                                const double* __restrict__ nx, const double* __restrict__ ny,
                                int32_t* __restrict__ Lidx, double* __restrict__ Lw,
                                double* __restrict__ es, double* __restrict__ scale,
                                int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < M; i += (int64_t)gridDim.x * kT) {
    const bool bnd = p_bc[i] != 0;
    const int32_t b = bnd ? bmap[i] : -1;
    if (bnd && b < 0) {
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
    es[i] = bnd ? -sc : 0.0;
    scale[i] = sc;
  }
}

__global__ void e_scatter_rows(int64_t nb, int64_t M, const int32_t* __restrict__ rows,
                               int32_t* __restrict__ bmap, int* __restrict__ err) {
  for (int64_t b = blockIdx.x * (int64_t)kT + threadIdx.x; b < nb; b += (int64_t)gridDim.x * kT) {
    const int32_t r = rows[b];
    if (r < 0 || r >= M || atomicCAS(&bmap[r], -1, (int32_t)b) != -1) atomicOr(err, 1);
  }
}

__global__ void e_rowsum(int64_t n, int64_t ld, int k, const double* __restrict__ w,
                         float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    double a = 0.0;
    for (int s = 0; s < k; ++s) a += w[s * ld + i];
    out[i] = (float)a;
  }
}

__global__ void e_diag(int64_t M, int64_t ld, int k, const int32_t* __restrict__ idx,
                       const double* __restrict__ w, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < M; i += (int64_t)gridDim.x * kT) {
    double s = 0.0;
    for (int q = 0; q < k; ++q)
      if (idx[q * ld + i] == (int32_t)i) s += w[q * ld + i];
    d[i] = s;
  }
}

__global__ void e_sum_scale(int64_t n, double* __restrict__ x, double* __restrict__ tmp) {
  // one block: deterministic sum, then x /= |sum|
  __shared__ double sh[kT];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kT) a += x[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kT; ++q) t += sh[q];
    *tmp = t;
  }
  __syncthreads();
  const double g = *tmp != 0.0 ? 1.0 / fabs(*tmp) : 1.0;
  for (int64_t i = threadIdx.x; i < n; i += kT) x[i] *= g;
}

rbffd_flow ens_key(const rbffd_flow& f) {
  rbffd_flow k = f;
  k.tol = k.inner_tol = 0.0;
  k.max_iter = k.km_mode = k.overwrite_bc = k.profile = k.cn_form = 0;
  k.Re = 0.0;
  return k;
}

int ens_build(rbffd_ctx* ctx, const rbffd_flow& f, int E, EnsPlan** out, cudaStream_t st) {
  EnsPlan* p = new EnsPlan();
  p->key = ens_key(f);
  p->E = E;
  p->k = ctx->prm.n;
  p->N = f.N;
  p->M = f.M;
  p->grid = sm_count() * 4;  // 4 blocks of 256 per SM (8 measured slower: 230 against 212 ms per step at 100k x 64)
  const int C = 2 * E, k = p->k;
  const int64_t nv = f.ld_v * k, np = f.ld_p * k;
  int rc = 0;
#define TRY(x)              \
  do {                      \
    rc = (x);               \
    if (rc) {               \
      ens_plan_free(p);     \
      return rc;            \
    }                       \
  } while (0)
  int32_t* bmap = nullptr;
  int* err = nullptr;
  TRY(ealloc(ctx, p, &p->Lidx, np));
  TRY(ealloc(ctx, p, &p->Lw, np));
  TRY(ealloc(ctx, p, &p->es, f.M));
  TRY(ealloc(ctx, p, &p->scale, f.M));
  TRY(ealloc(ctx, p, &bmap, f.M));
  TRY(ealloc(ctx, p, &err, 1));
  TRY(ealloc(ctx, p, &p->lz, nv));
  TRY(ealloc(ctx, p, &p->h2, 2 * kCMax));
  TRY(check_cuda(ctx, cudaMemsetAsync(err, 0, sizeof(int), st), "memset"));
  TRY(check_cuda(ctx, cudaMemsetAsync(bmap, 0xff, sizeof(int32_t) * f.M, st), "memset"));
  e_scatter_rows<<<p->grid, kT, 0, st>>>(f.nb_p, f.M, f.pn_rows, bmap, err);
  e_build_poisson<<<p->grid, kT, 0, st>>>(f.M, f.ld_p, k, f.pp_idx, f.pp_lap, f.p_bc, bmap,
                                          f.ld_b, f.pn_idx, f.pn_dx, f.pn_dy, f.p_nx, f.p_ny,
                                          p->Lidx, p->Lw, p->es, p->scale, err);
  e_sum_scale<<<1, kT, 0, st>>>(f.M, p->es, p->h2);
  e_scale_rows<<<p->grid, kT, 0, st>>>(f.N, f.ld_v, k, f.v_bc, f.vv_lap, p->lz);
  TRY(check_cuda(ctx, cudaGetLastError(), "ensemble plan kernels"));
  int herr = 0;
  TRY(check_cuda(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st),
                 "status"));
  TRY(check_cuda(ctx, cudaStreamSynchronize(st), "ensemble plan sync"));
  if (herr) {
    ens_plan_free(p);
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "Neumann rows (pn_rows) must list every boundary P-node once");
  }
  // multigrid hierarchy of the P-node edge graph (as step.cu builds it)
  if (f.precond) {
    std::vector<double> hd(f.M), hes(f.M);
    double* dd = nullptr;
    TRY(ealloc(ctx, p, &dd, f.M));
    e_diag<<<p->grid, kT, 0, st>>>(f.M, f.ld_p, k, p->Lidx, p->Lw, dd);
    TRY(check_cuda(ctx, cudaMemcpyAsync(hd.data(), dd, sizeof(double) * f.M,
                                        cudaMemcpyDeviceToHost, st), "diag copy"));
    TRY(check_cuda(ctx, cudaMemcpyAsync(hes.data(), p->es, sizeof(double) * f.M,
                                        cudaMemcpyDeviceToHost, st), "es copy"));
    TRY(check_cuda(ctx, cudaStreamSynchronize(st), "diag sync"));
    TRY(amg_build(ctx, f, hd.data(), hes.data(), &p->amg, st));
  }
  TRY(ens_to32(ctx, p, p->Lw, np, &p->Lw32, st));
  TRY(ens_to32(ctx, p, p->es, f.M, &p->es32, st));
  TRY(ealloc(ctx, p, &p->a1_32, f.M));
  e_rowsum<<<p->grid, kT, 0, st>>>(f.M, f.ld_p, k, p->Lw, p->a1_32);
  TRY(ens_to32(ctx, p, p->lz, nv, &p->lz32, st));
  TRY(ens_to32(ctx, p, f.vv_dx, nv, &p->vv_dx32, st));
  TRY(ens_to32(ctx, p, f.vv_dy, nv, &p->vv_dy32, st));
  TRY(ens_to32(ctx, p, f.vv_lap, nv, &p->vv_lap32, st));
  TRY(ens_to32(ctx, p, f.pp_lap, np, &p->pp_lap32, st));
  TRY(ens_to32(ctx, p, f.vp_dx, nv, &p->vp_dx32, st));
  TRY(ens_to32(ctx, p, f.vp_dy, nv, &p->vp_dy32, st));
  const int64_t nV = f.N * E, nP = f.M * E, nW = f.N * C;
  TRY(ealloc(ctx, p, &p->us, nV));
  TRY(ealloc(ctx, p, &p->vs, nV));
  TRY(ealloc(ctx, p, &p->rhs, nW));
  TRY(ealloc(ctx, p, &p->xv, nW));
  TRY(ealloc(ctx, p, &p->pb, nP));
  TRY(ealloc(ctx, p, &p->px, nP));
  for (int q = 0; q < kEHist; ++q) {
    TRY(ealloc(ctx, p, &p->vh[q], nW));
    TRY(ealloc(ctx, p, &p->ph[q], nP));
  }
  TRY(ealloc(ctx, p, &p->u2, nV));
  TRY(ealloc(ctx, p, &p->v2, nV));
  TRY(ealloc(ctx, p, &p->us2, nV));
  TRY(ealloc(ctx, p, &p->vs2, nV));
  TRY(ealloc(ctx, p, &p->pt2, nP));
  TRY(ealloc(ctx, p, &p->px2, nP));
  TRY(ealloc(ctx, p, &p->r64, nW));
  TRY(ealloc(ctx, p, &p->r32, nW));
  for (int q = 0; q < 9; ++q) TRY(ealloc(ctx, p, &p->kw[q], nW));
  TRY(ealloc(ctx, p, &p->aV, C));
  TRY(ealloc(ctx, p, &p->aV32, C));
  TRY(ealloc(ctx, p, &p->aE, E));
  TRY(ealloc(ctx, p, &p->nrm, kCMax));
  TRY(ealloc(ctx, p, &p->isc, kCMax));
  TRY(ealloc(ctx, p, &p->xsum, kCMax));
  TRY(ealloc(ctx, p, &p->mean, kCMax));
  TRY(ealloc(ctx, p, &p->sc, 1));
  TRY(ealloc(ctx, p, &p->sc_t, 1));
  TRY(ealloc(ctx, p, &p->rd.partials, (size_t)p->grid * kRV * kCMax));
  TRY(ealloc(ctx, p, &p->rd.counter, 1));
  TRY(check_cuda(ctx, cudaMemsetAsync(p->rd.counter, 0, sizeof(unsigned int), st), "memset"));
  if (const Amg* a = p->amg) {
    // level l (0 <= l < nlev; the coarsest is lev[nlev - 1], nc rows)
    for (int l = 0; l < a->nlev; ++l) {
      TRY(ealloc(ctx, p, &p->lr[l], a->lev[l].n * E));
      TRY(ealloc(ctx, p, &p->lx[l], a->lev[l].n * E));
    }
  }
  TRY(check_cuda(ctx, cudaStreamSynchronize(st), "ensemble plan"));
#undef TRY
  *out = p;
  return RBFFD_OK;
}

// B v for the C pressure columns of v (v: kw[3] = p or kw[5] = s): batched V-cycle
void ens_vcycle(EnsPlan* P, const float* v, int which, float* zout, cudaStream_t st) {
  // The hierarchy's nlev levels include the coarsest, lev[nlev - 1] (nc rows,
  // dense inverse Xc); only the levels above it restrict (their cptr maps the
  // next level's rows to their own).
  const Amg* a = P->amg;
  const int C = P->E, G = P->grid, L = a->nlev;
  e_pc_in<<<G, kT, 0, st>>>(P->M, C, v, a->c, a->ce, a->perm0, which, a->inv_ces, P->sc,
                            P->lr[0]);
  for (int l = 0; l + 1 < L; ++l)
    EW(e_pc_restrict, a->lev[l].width, a->lev[l], a->lev[l + 1].n, C, P->lr[l], P->lx[l],
       P->lr[l + 1], P->sc);
  const AmgLevel none{};
  const bool fine = L >= 2;
  const int TRc = kT / C > kCoarseRows ? kT / C : kCoarseRows;
  const int Gc = (int)((a->nc + TRc - 1) / TRc);
  e_pc_coarse<<<Gc, kT, 0, st>>>(a->nc, C, a->Xc, P->lr[L - 1], fine ? nullptr : P->lx[0],
                                fine ? a->lev[L - 2] : none, fine ? P->lx[L - 2] : nullptr,
                                fine ? 1 : 0, P->sc);
  if (!fine)  // the coarsest level is level 0: its z (in lx[0]) is the result
    e_pc_fin<<<G, kT, 0, st>>>(P->M, C, P->lx[0], a->perm0, zout, which, a->inv_ces, a->inv_R,
                               P->sc, P->rd);
  for (int l = L - 2; l >= 0; --l)
    EW(e_pc_up, a->lev[l].width, a->lev[l], C, P->lr[l], P->lx[l], l ? a->lev[l - 1] : none,
       l ? P->lx[l - 1] : nullptr, l == 0 ? 1 : 0, a->perm0, zout, which, a->inv_ces,
       a->inv_R, P->sc, P->rd);
  P->launches += 2 + 2 * (L - 1) + (fine ? 0 : 1);
}

struct ESolve {
  int iters = 0;
  int sweeps = 0;  // refinement sweeps (inner solves)
  bool converged = true;
  bool nonfinite = false;
  double relres = 0.0;
};

// One batched FP32 BiCGSTAB on C columns: op32 e = r32 (x0 = 0) to inner_tol.
int ens_bicgstab(rbffd_ctx* ctx, EnsPlan* P, const EOp& op, const float* w32, int C, bool pc,
                 double inner_tol, int maxit, ESolve* res, cudaStream_t st) {
  const int G = P->grid, k = op.k;
  float *x = P->kw[0], *r = P->kw[1], *rh = P->kw[2], *pp = P->kw[3], *v = P->kw[4],
        *s = P->kw[5], *t = P->kw[6], *zp = P->kw[7], *zs = P->kw[8];
  const float* cnode = pc ? P->amg->cnode : nullptr;
  const int64_t n = op.n;
  e_init<<<G, kT, 0, st>>>(n, C, P->r32, r, rh, pp, x, cnode, P->sc, P->rd,
                           inner_tol * inner_tol, maxit);
  EScal* h = (EScal*)ctx->host_pinned;
  int issued = 0;
  for (;;) {
    const int chunk = 4;
    for (int it = 0; it < chunk; ++it) {
      const float* zpp = pp;
      const float* zss = s;
      if (pc) {
        ens_vcycle(P, pp, 0, zp, st);
        zpp = zp;
      }
      EK(e_spmv_v, G, op, w32, zpp, v, rh, P->sc, P->rd);
      e_update_s<<<G, kT, 0, st>>>(n, r, v, s, cnode, P->sc, P->rd);
      if (pc) {
        ens_vcycle(P, s, 1, zs, st);
        zss = zs;
      }
      EK(e_spmv_t, G, op, w32, zss, t, s, P->sc, P->rd);
      e_update_xr<<<G, kT, 0, st>>>(n, x, r, rh, zpp, zss, s, t, pc ? 1 : 0, P->sc, P->rd);
      e_update_p<<<G, kT, 0, st>>>(n, pp, r, v, cnode, P->sc, P->rd);
      P->launches += 5;
    }
    issued += chunk;
    int rc = check_cuda(ctx, cudaGetLastError(), "ensemble bicgstab");
    if (rc) return rc;
    rc = check_cuda(ctx, cudaMemcpyAsync(h, P->sc, sizeof(EScal), cudaMemcpyDeviceToHost, st),
                    "ensemble scalars");
    if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "ensemble sync");
    if (rc) return rc;
    if (h->done || issued >= maxit) break;
  }
  res->iters = h->iters;
  for (int c = 0; c < C; ++c)
    if (h->status[c] == 2) res->nonfinite = true;
  return RBFFD_OK;
}

// FP64 refinement around ens_bicgstab: x (FP64, C columns) solves the FP64
// operator to tol per column.
int ens_refine(rbffd_ctx* ctx, EnsPlan* P, const EOp& op, const double* w64, const float* w32,
               int C, bool pc, double* x, const double* b, double tol, double inner_tol,
               int maxit, ESolve* res, cudaStream_t st) {
  const int G = P->grid, k = op.k;
  // [2C] norms, staged after the EScal that the inner solves copy to offset 0
  double* h = (double*)ctx->host_pinned + 4096;
  double hn[kCMax], hi[kCMax];
  res->iters = 0;
  res->converged = false;
  int used = 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (!op.visc) e_colsum<<<G, kT, 0, st>>>(op.n, C, x, P->rd, P->xsum);
    EK(e_residual64, G, op, w64, P->aV, P->es, x, b, P->r64, P->xsum, C, P->rd, P->h2);
    P->launches += op.visc ? 1 : 2;
    int rc = check_cuda(ctx, cudaGetLastError(), "ensemble residual");
    if (!rc)
      rc = check_cuda(ctx, cudaMemcpyAsync(h, P->h2, sizeof(double) * 2 * C,
                                           cudaMemcpyDeviceToHost, st), "residual copy");
    if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "residual sync");
    if (rc) return rc;
    bool conv = true;
    double worst = 0.0;
    for (int c = 0; c < C; ++c) {
      const double rr = h[2 * c], bb = h[2 * c + 1];
      if (!std::isfinite(rr)) {
        res->nonfinite = true;
        return RBFFD_OK;
      }
      worst = fmax(worst, bb > 0 ? sqrt(rr / bb) : sqrt(rr));
      if (!(rr <= tol * tol * bb)) conv = false;
      hn[c] = sqrt(rr);
      hi[c] = hn[c] > 0 ? 1.0 / hn[c] : 0.0;
    }
    res->relres = worst;
    if (conv) {
      res->converged = true;
      return RBFFD_OK;
    }
    if (used >= maxit) return RBFFD_OK;
    rc = check_cuda(ctx, cudaMemcpyAsync(P->nrm, hn, sizeof(double) * C, cudaMemcpyHostToDevice, st),
                    "norms");
    if (!rc)
      rc = check_cuda(ctx, cudaMemcpyAsync(P->isc, hi, sizeof(double) * C, cudaMemcpyHostToDevice,
                                           st), "scales");
    if (rc) return rc;
    e_to32<<<G, kT, 0, st>>>(op.n, C, P->r64, P->isc, P->r32);
    ESolve inner;
    // at most kInnerRestart iterations per inner solve: a column whose
    // recurrences stagnate restarts from its true residual in the next sweep
    rc = ens_bicgstab(ctx, P, op, w32, C, pc, inner_tol,
                      maxit - used < kInnerRestart ? maxit - used : kInnerRestart, &inner, st);
    if (rc) return rc;
    used += inner.iters > 0 ? inner.iters : 1;
    res->iters += inner.iters;
    res->sweeps += 1;
    e_addcorr<<<G, kT, 0, st>>>(op.n, C, x, P->kw[0], P->nrm);
    P->launches += 2;
  }
  return RBFFD_OK;
}

}  // namespace

int ensemble_run(rbffd_ctx* ctx, const rbffd_flow* fp, int E, const double* Re, rbffd_state* s,
                 const double* gu, const double* gv, int32_t n_steps, rbffd_stats* stats,
                 cudaStream_t st) {
  const rbffd_flow& f = *fp;
  const rbffd_flow key = ens_key(f);
  if (ctx->ens && (ctx->ens->E != E || memcmp(&ctx->ens->key, &key, sizeof(rbffd_flow)) != 0)) {
    cudaStreamSynchronize(st);
    ens_plan_free(ctx->ens);
    ctx->ens = nullptr;
  }
  if (!ctx->ens) {
    int rc = ens_build(ctx, f, E, &ctx->ens, st);
    if (rc) return rc;
  }
  EnsPlan* P = ctx->ens;
  const int G = P->grid, k = P->k, C = 2 * E;
  // per-column a = dt / (2 Re) (viscous columns: u of member e, then v)
  double av[kCMax];
  float av32[kCMax];
  for (int e = 0; e < E; ++e) {
    av[e] = av[E + e] = f.dt / (2.0 * Re[e]);
    av32[e] = av32[E + e] = (float)av[e];
  }
  int rc = check_cuda(ctx, cudaMemcpyAsync(P->aV, av, sizeof(double) * C, cudaMemcpyHostToDevice, st),
                      "a");
  if (!rc) rc = check_cuda(ctx, cudaMemcpyAsync(P->aV32, av32, sizeof(float) * C,
                                                cudaMemcpyHostToDevice, st), "a32");
  if (!rc) rc = check_cuda(ctx, cudaMemcpyAsync(P->aE, av, sizeof(double) * E,
                                                cudaMemcpyHostToDevice, st), "aE");
  if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "a sync");
  if (rc) return rc;
  const int64_t nV = f.N * E, nP = f.M * E, nW = f.N * C;
  e_split<<<G, kT, 0, st>>>(nV, s->u, P->u2);
  e_split<<<G, kT, 0, st>>>(nV, s->v, P->v2);
  e_split<<<G, kT, 0, st>>>(nP, s->pt, P->pt2);
  const int64_t l0 = P->launches;
  EOp H{f.vv_idx, f.ld_v, f.N, k, 1, P->aV32, nullptr, nullptr};
  EOp L{P->Lidx, f.ld_p, f.M, k, 0, nullptr, P->es32, P->a1_32};
  // push x (a solve's solution of the state's previous step) into a ring of
  // earlier solutions; returns the order of the extrapolation the ring allows
  auto push = [&](double* const* ring, int* head, int* count, const double* x, int64_t n) {
    const int slot = (*head + kEHist - 1) % kEHist;
    int r = check_cuda(ctx, cudaMemcpyAsync(ring[slot], x, sizeof(double) * n,
                                            cudaMemcpyDeviceToDevice, st),
                       "solution history");
    *head = slot;
    *count = std::min(*count + 1, kEHist);
    return r;
  };
  auto ring_of = [&](double* const* ring, int head) {
    EHist H;
    for (int q = 0; q < kEHist; ++q) H.h[q] = ring[(head + q) % kEHist];
    return H;
  };
  for (int32_t step = 0; step < n_steps; ++step) {
    // the solves start from the extrapolation of their previous solutions
    // while this plan made the state's previous steps
    const bool hist = P->last_j == s->j;
    if (!hist) P->nvh = P->nph = 0;
    if (hist) {
      rc = push(P->vh, &P->hv, &P->nvh, P->xv, nW);
      if (rc) return rc;
    }
    EK(e_convect, G, f.N, f.ld_v, k, E, f.vv_idx, P->vv_dx32, P->vv_dy32, s->u, s->v,
                                P->u2, P->v2, s->cu_prev, s->cv_prev, P->us, P->vs, P->us2,
                                P->vs2, f.dt, s->j == 0 ? 1 : 0);
    EK(e_helm_rhs, G, f.N, f.ld_v, k, E, f.vv_idx, P->vv_lap32, P->us, P->vs,
                                 f.cn_form ? P->u2 : P->us2, f.cn_form ? P->v2 : P->vs2,
                                 f.vp_idx, P->vp_dx32, P->vp_dy32, P->pt2, f.v_bc, f.v_nx,
                                 f.v_ny, gu, gv, P->aE, f.dt, f.km_mode, P->rhs, P->xv);
    P->launches += 2;
    if (P->nvh > 0) {
      e_extrapolate<<<G, kT, 0, st>>>(nW, P->nvh - 1, ring_of(P->vh, P->hv), f.v_bc, C, P->xv);
      P->launches += 1;
    }
    rc = check_cuda(ctx, cudaGetLastError(), "ensemble stages 1-2");
    if (rc) return rc;
    ESolve hr;
    rc = ens_refine(ctx, P, H, P->lz, P->lz32, C, false, P->xv, P->rhs, f.tol,
                    f.inner_tol * f.inner_tol, f.max_iter, &hr, st);
    if (rc) return rc;
    if (stats) {
      stats->helm_iters += hr.iters;
      stats->helm_relres = hr.relres;
    }
    if (hr.nonfinite) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite ensemble viscous solve");
    if (!hr.converged)
      return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                       "ensemble viscous solve: relative residual %.3e", hr.relres);
    EK(e_divergence, G, f.M, f.ld_p, k, E, f.pv_idx, f.pv_dx, f.pv_dy, P->xv, f.p_bc,
                                   P->scale, 1.0 / f.dt, P->pb);
    if (hist) {
      rc = push(P->ph, &P->hp, &P->nph, P->px, nP);
      if (rc) return rc;
      e_extrapolate<<<G, kT, 0, st>>>(nP, P->nph - 1, ring_of(P->ph, P->hp), nullptr, 1, P->px);
      P->launches += 1;
    } else {
      rc = check_cuda(ctx, cudaMemcpyAsync(P->px, s->pt, sizeof(double) * nP,
                                           cudaMemcpyDeviceToDevice, st), "warm start");
      if (rc) return rc;
    }
    ESolve pr;
    rc = ens_refine(ctx, P, L, P->Lw, P->Lw32, E, P->amg != nullptr, P->px, P->pb, f.tol,
                    f.inner_tol, f.max_iter, &pr, st);
    if (rc) return rc;
    if (stats) {
      stats->poisson_iters += pr.iters;
      stats->refinements += pr.sweeps;
      stats->poisson_relres = pr.relres;
    }
    if (pr.nonfinite) return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite ensemble pressure solve");
    if (!pr.converged)
      return set_error(ctx, RBFFD_ERR_NOT_CONVERGED,
                       "ensemble pressure solve: relative residual %.3e", pr.relres);
    e_colmean<<<G, kT, 0, st>>>(f.M, E, P->px, P->rd, P->mean);
    e_split<<<G, kT, 0, st>>>(nP, P->px, P->px2);
    EK(e_pressure, G, f.M, f.ld_p, k, E, f.pp_idx, P->pp_lap32, P->px, P->px2, P->mean,
                                 P->aE, s->pt, s->p, P->pt2);
    EK(e_correct, G, f.N, f.ld_v, k, E, f.vp_idx, P->vp_dx32, P->vp_dy32, P->pt2, P->xv,
                                f.v_bc, gu, gv, f.dt, f.overwrite_bc, s->u, s->v, P->u2, P->v2);
    P->launches += 6;
    rc = check_cuda(ctx, cudaGetLastError(), "ensemble stage 3");
    if (rc) return rc;
    s->j += 1;
    P->last_j = s->j;
    if (stats) stats->steps += 1;
  }
  rc = check_cuda(ctx, cudaStreamSynchronize(st), "ensemble sync");
  if (stats) stats->launches = P->launches - l0;
  if (!rc && stats && f.profile) {
    // the batched pressure SpMV timed alone: 20 back-to-back launches on this
    // plan's operator and work vectors (every column active), CUDA events on
    // the caller's stream
    EScal* hs = (EScal*)ctx->host_pinned;
    memset(hs, 0, sizeof(EScal));
    hs->C = E;
    for (int c = 0; c < E; ++c) hs->active[c] = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = check_cuda(ctx, cudaMemcpyAsync(P->sc_t, hs, sizeof(EScal), cudaMemcpyHostToDevice, st),
                    "timing scalars");
    if (!rc) rc = check_cuda(ctx, cudaEventCreate(&e0), "event");
    if (!rc) rc = check_cuda(ctx, cudaEventCreate(&e1), "event");
    if (!rc) {
      constexpr int kReps = 20;
      cudaEventRecord(e0, st);
      for (int r = 0; r < kReps; ++r)
        EK(e_spmv_v, G, L, P->Lw32, P->kw[7], P->kw[4], P->kw[2], P->sc_t, P->rd);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      rc = check_cuda(ctx, cudaEventSynchronize(e1), "timing sync");
      if (!rc && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        stats->spmv_batch_ms += ms;
        stats->spmv_batch_launches += kReps;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  return rc;
}

}  // namespace rbffd
