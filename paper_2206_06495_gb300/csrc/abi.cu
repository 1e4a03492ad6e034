// C ABI: context lifetime, error reporting, argument validation.
#include <cstring>
#include <new>
#include <vector>

#include <cmath>

#include "common.cuh"

namespace rbffd {

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

int set_error(rbffd_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int check_cuda(rbffd_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RBFFD_OK;
  if (e == cudaErrorMemoryAllocation)
    return set_error(ctx, RBFFD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(ctx, RBFFD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ctx_scratch(rbffd_ctx* ctx, size_t bytes, void** out) {
  if (bytes > ctx->scratch_bytes) {
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    size_t want = bytes + bytes / 4;
    int rc = check_cuda(ctx, cudaMalloc(&ctx->scratch, want), "scratch allocation");
    if (rc) return rc;
    ctx->scratch_bytes = want;
  }
  *out = ctx->scratch;
  return RBFFD_OK;
}

static int n_monomials(int q) { return q < 0 ? 0 : (q + 1) * (q + 2) / 2; }

}  // namespace rbffd

using namespace rbffd;

extern "C" {

int rbffd_version(void) { return 100; }

int rbffd_create(rbffd_ctx** ctx, const rbffd_params* p) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  *ctx = nullptr;
  rbffd_params prm{28, 7, 3};
  if (p) prm = *p;
  if (prm.n < 1 || prm.n > kMaxStencil || prm.m < 3 || prm.m > 13 || (prm.m % 2) == 0 ||
      prm.q < -1 || prm.q > 5 || prm.n < n_monomials(prm.q) ||
      prm.n + n_monomials(prm.q) > kMaxSystem)
    return RBFFD_ERR_INVALID_ARG;
  rbffd_ctx* c = new (std::nothrow) rbffd_ctx();
  if (!c) return RBFFD_ERR_OOM;
  c->prm = prm;
  if (cudaMallocHost(&c->host_pinned, kHostPinnedBytes) != cudaSuccess) {
    delete c;
    return RBFFD_ERR_CUDA;
  }
  *ctx = c;
  return RBFFD_OK;
}

int rbffd_destroy(rbffd_ctx* ctx) {
  if (!ctx) return RBFFD_OK;
  if (ctx->plan) step_plan_free(ctx->plan);
  if (ctx->ens) ens_plan_free(ctx->ens);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  delete ctx;
  return RBFFD_OK;
}

const char* rbffd_last_error(const rbffd_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

static int build_weights_impl(rbffd_ctx* ctx, const double* ax, const double* ay,
                              int64_t n_alpha, const double* bx, const double* by, int64_t n_beta,
                              const uint8_t* beta_mask, const int32_t* alpha_self,
                              uint32_t op_mask, int32_t* idx, double* w, int64_t ld,
                              int64_t* bad_node, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (bad_node) *bad_node = -1;
  const int k = ctx->prm.n;
  if (n_alpha < 0 || n_beta < 0)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "negative node count");
  if ((op_mask & 15u) == 0 || (op_mask & ~15u))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "op_mask must be a nonzero OR of RBFFD_OP_*");
  if (n_alpha == 0) return RBFFD_OK;
  if (n_beta < k)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "stencil size %d exceeds %lld beta-nodes", k,
                     (long long)n_beta);
  if (n_alpha > INT32_MAX || n_beta > INT32_MAX)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "node counts must fit int32");
  if (!ax || !ay || !bx || !by || !idx || !w)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null array pointer");
  if (ld < n_alpha || ld % 32)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "ld must be >= n_alpha and a multiple of 32");
  if (beta_mask || alpha_self) {
    // both tables are small set-up inputs: check them on the host before any kernel reads them
    if (beta_mask) {
      std::vector<uint8_t> m((size_t)n_beta);
      int rc = check_cuda(ctx, cudaMemcpyAsync(m.data(), beta_mask, (size_t)n_beta,
                                               cudaMemcpyDeviceToHost, stream), "mask copy");
      if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(stream), "mask sync");
      if (rc) return rc;
      int64_t cnt = 0;
      for (uint8_t v : m) cnt += v != 0;
      if (cnt < k - (alpha_self ? 1 : 0))
        return set_error(ctx, RBFFD_ERR_INVALID_ARG, "only %lld beta-nodes pass the mask",
                         (long long)cnt);
    }
    if (alpha_self) {
      std::vector<int32_t> a((size_t)n_alpha);
      int rc = check_cuda(ctx, cudaMemcpyAsync(a.data(), alpha_self, sizeof(int32_t) * n_alpha,
                                               cudaMemcpyDeviceToHost, stream), "self copy");
      if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(stream), "self sync");
      if (rc) return rc;
      for (int32_t v : a)
        if (v < 0 || v >= n_beta)
          return set_error(ctx, RBFFD_ERR_INVALID_ARG, "alpha_self entry %d out of range", v);
    }
  }
  int rc = knn_build(ctx, ax, ay, n_alpha, bx, by, n_beta, beta_mask, alpha_self, k, idx, ld,
                     stream);
  if (rc) return rc;
  return weights_build(ctx, ax, ay, n_alpha, bx, by, idx, ld, op_mask, w, bad_node, stream);
}

int rbffd_build_weights(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t n_alpha,
                        const double* bx, const double* by, int64_t n_beta, uint32_t op_mask,
                        int32_t* idx, double* w, int64_t ld, int64_t* bad_node,
                        cudaStream_t stream) {
  return build_weights_impl(ctx, ax, ay, n_alpha, bx, by, n_beta, nullptr, nullptr, op_mask, idx,
                            w, ld, bad_node, stream);
}

int rbffd_build_weights_masked(rbffd_ctx* ctx, const double* ax, const double* ay,
                               int64_t n_alpha, const double* bx, const double* by,
                               int64_t n_beta, const uint8_t* beta_mask,
                               const int32_t* alpha_self, uint32_t op_mask, int32_t* idx,
                               double* w, int64_t ld, int64_t* bad_node, cudaStream_t stream) {
  return build_weights_impl(ctx, ax, ay, n_alpha, bx, by, n_beta, beta_mask, alpha_self, op_mask,
                            idx, w, ld, bad_node, stream);
}

int rbffd_apply_op(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, void* y, double alpha,
                   double beta, int32_t xy_dtype, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!D) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  if (D->n_rows < 0 || D->n_cols < 1 || D->n < 1 || D->n > kMaxStencil || D->ld < D->n_rows ||
      D->ld % 32)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad operator shape");
  if ((D->w_dtype != RBFFD_F64 && D->w_dtype != RBFFD_F32) ||
      (xy_dtype != RBFFD_F64 && xy_dtype != RBFFD_F32))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad dtype");
  if (D->n_rows == 0) return RBFFD_OK;  // nothing to read or write
  if (!D->idx || !D->w || !x || !y) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  return spmv_apply(ctx, D, x, y, alpha, beta, xy_dtype, stream);
}

int rbffd_apply_op_shape(rbffd_ctx* ctx, const rbffd_ell* D, int32_t xy_dtype, int32_t* threads,
                         int32_t* blocks_per_sm) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!D || !threads || !blocks_per_sm) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  int t = 0, b = 0;
  const int rc = spmv_shape(ctx, D, xy_dtype, &t, &b);
  *threads = t;
  *blocks_per_sm = b;
  return rc;
}

static int check_flow(rbffd_ctx* ctx, const rbffd_flow* flow) {
  if (!flow) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null flow");
  const rbffd_flow& f = *flow;
  if (f.N < ctx->prm.n || f.M < ctx->prm.n || f.ld_v < f.N || f.ld_p < f.M || f.ld_v % 32 ||
      f.ld_p % 32 || f.N > INT32_MAX || f.M > INT32_MAX || f.nb_p < 0 || f.nb_p > f.M ||
      (f.nb_p > 0 && (f.ld_b < f.nb_p || f.ld_b % 32)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad node counts or leading dimensions");
  if (!f.vv_idx || !f.vv_dx || !f.vv_dy || !f.vv_lap || !f.pv_idx || !f.pv_dx || !f.pv_dy ||
      !f.pp_idx || !f.pp_dx || !f.pp_dy || !f.pp_lap || !f.vp_idx || !f.vp_dx || !f.vp_dy ||
      !f.v_bc || !f.v_nx || !f.v_ny || !f.p_bc || !f.p_nx || !f.p_ny ||
      (f.nb_p > 0 && (!f.pn_rows || !f.pn_idx || !f.pn_dx || !f.pn_dy)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null operator or boundary array");
  if (!(f.Re > 0) || !(f.dt > 0) || !(f.tol > 0) || f.max_iter < 1 ||
      (f.precision != RBFFD_PREC_FP64 && f.precision != RBFFD_PREC_MIXED) || f.km_mode < 0 ||
      f.km_mode > 2 || (f.precision == RBFFD_PREC_MIXED && !(f.inner_tol > 0 && f.inner_tol < 1)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad Re, dt, tolerances or modes");
  if (f.precond != 0 && f.precond != 1)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "precond must be 0 or 1");
  if ((f.projection != RBFFD_PROJ_PAPER && f.projection != RBFFD_PROJ_EXACT) ||
      (f.cn_form != RBFFD_CN_PRINTED && f.cn_form != RBFFD_CN_KIM_MOIN))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "projection and cn_form must be 0 or 1");
  if (f.precond && (!f.p_edges || f.n_edges < 1 || f.n_edges > INT32_MAX || !f.p_x || !f.p_y))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "precond = 1 needs p_edges, n_edges, p_x, p_y");
  // open flows: per-component velocity conditions with their Neumann rows
  if ((f.v_bcu == nullptr) != (f.v_bcv == nullptr))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "v_bcu and v_bcv are both set or both null");
  if (f.v_bcu) {
    if (f.nb_v < 0 || f.nb_v > f.N ||
        (f.nb_v > 0 && (f.ld_vb < f.nb_v || f.ld_vb % 32 || !f.vn_rows || !f.vn_idx ||
                        !f.vn_dx || !f.vn_dy)))
      return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad Neumann V-rows (nb_v, ld_vb, vn_*)");
    if (f.projection != RBFFD_PROJ_PAPER || (f.km_mode != 0 && f.km_mode != 2))
      return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                       "open flows run the paper's projection with km_mode 0 or 2");
  }
  return RBFFD_OK;
}

int rbffd_step(rbffd_ctx* ctx, const rbffd_flow* flow, rbffd_state* state, const double* gu,
               const double* gv, int32_t n_steps, rbffd_stats* stats, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!flow || !state || !gu || !gv)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  if (n_steps < 0) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "negative n_steps");
  int rc = check_flow(ctx, flow);
  if (rc) return rc;
  if (!state->u || !state->v || !state->cu_prev || !state->cv_prev || !state->pt || !state->p)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null state array");
  if (n_steps == 0) return RBFFD_OK;
  return step_run(ctx, flow, state, gu, gv, n_steps, stats, stream);
}

int rbffd_ensemble_step(rbffd_ctx* ctx, const rbffd_flow* flow, int32_t n_members,
                        const double* Re, rbffd_state* state, const double* gu, const double* gv,
                        int32_t n_steps, rbffd_stats* stats, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!flow || !state || !gu || !gv || !Re)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  if (n_members < 1 || n_members > 64 || (n_members & (n_members - 1)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "n_members must be a power of two, 1..64");
  for (int e = 0; e < n_members; ++e)
    if (!(Re[e] > 0.0) || !std::isfinite(Re[e]))
      return set_error(ctx, RBFFD_ERR_INVALID_ARG, "Re[%d] must be finite and positive", e);
  if (n_steps < 0) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "negative n_steps");
  int rc = check_flow(ctx, flow);
  if (rc) return rc;
  if (flow->projection != RBFFD_PROJ_PAPER)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "ensembles run the paper's projection only");
  if (flow->v_bcu)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "ensembles run the cavity's walls only");
  if (!state->u || !state->v || !state->cu_prev || !state->cv_prev || !state->pt || !state->p)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null state array");
  if (n_steps == 0) return RBFFD_OK;
  return ensemble_run(ctx, flow, n_members, Re, state, gu, gv, n_steps, stats, stream);
}

int rbffd_stencil_condition(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t n_alpha,
                            const double* bx, const double* by, int64_t n_beta,
                            const int32_t* idx, int64_t ld, double* cond, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (n_alpha < 0 || n_beta < ctx->prm.n || ld < n_alpha || ld % 32 || n_alpha > INT32_MAX)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad sizes");
  if (n_alpha == 0) return RBFFD_OK;
  if (!ax || !ay || !bx || !by || !idx || !cond)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  return cond_build(ctx, ax, ay, n_alpha, bx, by, idx, ld, cond, stream);
}

static bool ell_f64_ok(const rbffd_ell* D) {
  return D && D->n_rows >= 0 && D->n_cols >= 1 && D->n >= 1 && D->n <= kMaxStencil &&
         D->ld >= D->n_rows && D->ld % 32 == 0 && D->w_dtype == RBFFD_F64 &&
         (D->n_rows == 0 || (D->idx && D->w));
}

int rbffd_modified_wavenumber(rbffd_ctx* ctx, const rbffd_ell* Dx, const rbffd_ell* Dy,
                              const rbffd_ell* Dlap, const double* ax, const double* ay,
                              const double* bx, const double* by, double kx, double ky,
                              double* k1, double* k2, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ell_f64_ok(Dx) || !ell_f64_ok(Dy) || (Dlap && !ell_f64_ok(Dlap)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad operator (FP64 ELL expected)");
  if (Dy->n_rows != Dx->n_rows || Dy->n != Dx->n || Dy->ld != Dx->ld ||
      Dy->n_cols != Dx->n_cols || (Dlap && (Dlap->n_rows != Dx->n_rows ||
                                             Dlap->n_cols != Dx->n_cols)))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "operators of different shapes");
  if (!(kx * kx + ky * ky > 0.0) || !std::isfinite(kx) || !std::isfinite(ky))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "wave vector must be finite and nonzero");
  if (Dx->n_rows == 0) return RBFFD_OK;
  if (!ax || !ay || !bx || !by || !k1 || (Dlap && !k2))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  return analysis_mw(ctx, Dx, Dy, Dlap, ax, ay, bx, by, kx, ky, k1, k2, stream);
}

int rbffd_stencil_error(rbffd_ctx* ctx, const rbffd_ell* D, uint32_t op, const double* ax,
                        const double* ay, const double* bx, const double* by, const double* dr,
                        double* err, double* err_mean, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ell_f64_ok(D)) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad operator (FP64 ELL expected)");
  int opi = -1;
  if (op == RBFFD_OP_INTERP) opi = 0;
  else if (op == RBFFD_OP_DX) opi = 1;
  else if (op == RBFFD_OP_DY) opi = 2;
  else if (op == RBFFD_OP_LAP) opi = 3;
  if (opi < 0) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "op must be one RBFFD_OP_* bit");
  if (!dr && D->n < 7)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "dr from the stencil needs n >= 7");
  if (D->n_rows == 0) return RBFFD_OK;
  if (!ax || !ay || !bx || !by || !err) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  return analysis_error(ctx, D, opi, ax, ay, bx, by, dr, err, err_mean, stream);
}

int rbffd_debug_set_wait_limit(rbffd_ctx* ctx, int64_t polls) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  return step_set_wait_limit(ctx, (long long)polls);
}

int rbffd_adjoint_step(rbffd_ctx* ctx, const rbffd_flow* flow, const rbffd_state* fwd,
                       rbffd_adjoint* lam, double* grad_gu, double* grad_gv, rbffd_stats* stats,
                       cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!flow || !fwd || !lam || !grad_gu || !grad_gv)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  int rc = check_flow(ctx, flow);
  if (rc) return rc;
  if (!fwd->u || !fwd->v || fwd->j < 0)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "bad forward state");
  if (!lam->u || !lam->v || !lam->cu_prev || !lam->cv_prev || !lam->pt)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null adjoint array");
  if (flow->projection != RBFFD_PROJ_PAPER || flow->cn_form != RBFFD_CN_PRINTED)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "the adjoint exists for the paper's step only (projection 0, cn_form 0)");
  if (flow->v_bcu)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "the adjoint exists for the cavity's walls only");
  return adjoint_run(ctx, flow, fwd, lam, grad_gu, grad_gv, stats, stream);
}

}  // extern "C"

extern "C" int rbffd_cylinder_forces(rbffd_ctx* ctx, const rbffd_flow* flow, const double* u,
                                     const double* v, const double* p, const int32_t* rows,
                                     int32_t n_c, double cx, double cy, double radius, double Re,
                                     double* cd_cl, cudaStream_t stream) {
  if (!ctx) return RBFFD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!flow || !u || !v || !p || !rows || !cd_cl)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "null pointer");
  int rc = check_flow(ctx, flow);
  if (rc) return rc;
  if (!flow->p_x || !flow->p_y)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "forces need the P-node coordinates p_x, p_y");
  if (n_c < 4 || n_c % 2 || !(radius > 0.0) || !(Re > 0.0))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "n_c must be even and at least 4, radius and Re positive");
  std::vector<int32_t> h(n_c);
  rc = check_cuda(ctx, cudaMemcpyAsync(h.data(), rows, sizeof(int32_t) * n_c,
                                       cudaMemcpyDeviceToHost, stream), "rows copy");
  if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(stream), "rows sync");
  if (rc) return rc;
  for (int32_t q = 0; q < n_c; ++q)
    if (h[q] < 0 || h[q] >= flow->M)
      return set_error(ctx, RBFFD_ERR_INVALID_ARG, "surface row %d out of range", q);
  return analysis_forces(ctx, *flow, u, v, p, rows, n_c, cx, cy, radius, Re, cd_cl, stream);
}
