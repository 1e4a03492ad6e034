/*
 * rbffd.h - C ABI of the GB300 RBF-FD staggered-node Navier-Stokes hot path.
 *
 * The method is the semi-implicit fractional-step solver of Chu & Schmidt,
 * "RBF-FD discretization of the Navier-Stokes equations on scattered but
 * staggered nodes": polyharmonic-spline-plus-polynomial (PHS+poly) stencil
 * weights (Section 2), sparse differentiation matrices between a pressure
 * node set (P-grid) and a velocity node set (V-grid) (Section 2.2, Section 4),
 * and the three-stage time step of Section 3.
 *
 * Conventions shared by every entry point
 *  - Every call returns an int status: RBFFD_OK (0) or a negative RBFFD_ERR_*.
 *    No exception crosses the ABI and nothing calls exit/abort.
 *    rbffd_last_error(ctx) gives a message for the last failing call on ctx.
 *  - Array arguments are DEVICE pointers owned by the caller unless stated
 *    otherwise.  The library owns only the workspace inside the opaque
 *    rbffd_ctx, released by rbffd_destroy.
 *  - Work is issued on the caller's cudaStream_t.  Calls that report a
 *    device-side status (singular stencil, Krylov convergence) synchronise
 *    that stream before returning.
 *  - Sparse operators use a slot-major ELL layout: for an operator with n
 *    rows, stencil size k and leading dimension ld >= n (a multiple of 32),
 *    idx[s * ld + i] is the s-th stencil node of row i (int32, nearest first)
 *    and w[s * ld + i] its weight.  Operators built on the same node pair
 *    share one idx array.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RBFFD_OK 0
#define RBFFD_ERR_INVALID_ARG (-1)      /* null pointer, bad size, even m, k too small or too large */
#define RBFFD_ERR_SINGULAR_STENCIL (-2) /* an augmented system had a zero or non-finite pivot */
#define RBFFD_ERR_NOT_CONVERGED (-3)    /* a Krylov solve reached its iteration cap */
#define RBFFD_ERR_NONFINITE (-4)        /* a non-finite value appeared in a solve */
#define RBFFD_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define RBFFD_ERR_OOM (-6)              /* workspace allocation failed */

/* operator selection bits for rbffd_build_weights (Section 2.1, Eq. Lf) */
#define RBFFD_OP_INTERP 1u /* L = identity: interpolation to the alpha-node  */
#define RBFFD_OP_DX 2u     /* L = d/dx                                        */
#define RBFFD_OP_DY 4u     /* L = d/dy                                        */
#define RBFFD_OP_LAP 8u    /* L = d2/dx2 + d2/dy2                             */

/* element types */
#define RBFFD_F64 0
#define RBFFD_F32 1

/* precision policy of rbffd_step */
#define RBFFD_PREC_FP64 0  /* everything in FP64 */
#define RBFFD_PREC_MIXED 1 /* FP32 SpMVs and inner Krylov, FP64 iterative refinement */

/* projection of rbffd_step (rbffd_flow.projection) */
#define RBFFD_PROJ_PAPER 0 /* Section 3: pressure Poisson with D^(P,P)_Lap */
#define RBFFD_PROJ_EXACT 1 /* composed D^(P,V) G0: discretely divergence-free velocity */

/* Crank-Nicolson right side of rbffd_step (rbffd_flow.cn_form) */
#define RBFFD_CN_PRINTED 0  /* Eq. u_ss: (I + a D_Lap) u*                    */
#define RBFFD_CN_KIM_MOIN 1 /* Kim & Moin: u* + a D_Lap u_j                   */

/* Boundary conditions of open flows (rbffd_flow.v_bcu, v_bcv, p_bc). */
#define RBFFD_BC_DIRICHLET 1 /* velocity: the wall data (Kim & Moin value for u**) */
#define RBFFD_BC_NEUMANN 2   /* velocity: n.grad = 0 on a one-sided stencil         */
#define RBFFD_PBC_DIRICHLET 2 /* p_bc value of a Dirichlet pressure row (p~ = 0)    */

typedef struct rbffd_ctx rbffd_ctx;

/* Stencil parameters (n, m, q) of Section 4; the paper selects (28, 7, 3). */
typedef struct rbffd_params {
  int32_t n; /* stencil size: nearest beta-nodes per alpha-node, 1..64        */
  int32_t m; /* PHS exponent of phi(r) = r^m; odd, 3..13                     */
  int32_t q; /* degree of the polynomial augmentation, -1 (none) .. 5;
                the system size (n + (q+1)(q+2)/2) must not exceed 96 and n
                must be at least the number of monomials                    */
} rbffd_params;

/* Create a context.  p may be NULL for (28, 7, 3). */
int rbffd_create(rbffd_ctx** ctx, const rbffd_params* p);
/* Release a context and its workspace (after the caller's streams are idle). */
int rbffd_destroy(rbffd_ctx* ctx);
/* Message of the last failing call on ctx; never NULL. */
const char* rbffd_last_error(const rbffd_ctx* ctx);
/* Library version as major*10000 + minor*100 + patch. */
int rbffd_version(void);

/*
 * rbffd_build_weights - stencils and PHS+poly weights of D_L^(alpha,beta).
 *
 * Section 2.2: row i of D_L^(alpha,beta) uses the n nearest beta-nodes of
 * alpha-node i; Section 2.1, Eq. rbf_poly_compact: the weights solve
 *   [A P; P^T 0] [w; c] = [L phi; L P]
 * with A_ij = |x_i - x_j|^m and P the monomials up to degree q.  Each system
 * is shifted to the alpha-node and scaled by the largest stencil radius before
 * the solve (LU with partial pivoting, FP64); the weights are unscaled after.
 *
 * ax, ay     alpha-node coordinates, double[n_alpha]
 * bx, by     beta-node coordinates, double[n_beta]
 * op_mask    OR of RBFFD_OP_* (at least one)
 * idx        out: int32[n * ld], nearest first, ties by lower index;
 *            distances are compared as dx*dx + dy*dy, each operation rounded
 * w          out: double[nops * n * ld]; the operators are stored in bit
 *            order INTERP, DX, DY, LAP, skipping those not requested
 * ld         leading dimension, >= n_alpha, a multiple of 32
 * bad_node   HOST out (may be NULL): lowest alpha index whose system was
 *            singular, or -1
 * Errors: INVALID_ARG (n > n_beta, sizes), SINGULAR_STENCIL (weights of
 * singular rows are set to 0; all other rows are valid), CUDA, OOM.
 * Synchronises `stream`.
 */
int rbffd_build_weights(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t n_alpha,
                        const double* bx, const double* by, int64_t n_beta, uint32_t op_mask,
                        int32_t* idx, double* w, int64_t ld, int64_t* bad_node,
                        cudaStream_t stream);

/*
 * rbffd_build_weights_masked - as rbffd_build_weights with two stencil rules
 * used for one-sided boundary operators (Section 2.2's nearest-n rule applied
 * to a subset of the beta-nodes):
 * beta_mask   device uint8[n_beta] or NULL: only beta-nodes with a nonzero
 *             entry are stencil candidates
 * alpha_self  device int32[n_alpha] or NULL: when given, slot 0 of row i is
 *             beta-node alpha_self[i] (normally the alpha-node itself, present
 *             in the beta set but masked out) and slots 1..n-1 are the n-1
 *             nearest candidates
 * Both tables are checked on the host (INVALID_ARG if fewer than the needed
 * candidates pass the mask or an alpha_self entry is out of range).
 * Used for the pressure rows of boundary P-nodes: the node itself followed by
 * its n-1 nearest interior P-nodes.  Synchronises `stream`.
 */
int rbffd_build_weights_masked(rbffd_ctx* ctx, const double* ax, const double* ay,
                               int64_t n_alpha, const double* bx, const double* by,
                               int64_t n_beta, const uint8_t* beta_mask,
                               const int32_t* alpha_self, uint32_t op_mask, int32_t* idx,
                               double* w, int64_t ld, int64_t* bad_node, cudaStream_t stream);

/*
 * rbffd_build_weights_noalloc - rbffd_build_weights for callers that cannot
 * allocate GPU memory (for instance code inside a host framework that owns the
 * whole device memory pool, or a loop with a fixed memory budget that cannot
 * pay for cudaMalloc/cudaFree).  The paper has no counterpart; this is a
 * deployment variant of the same computation and returns the same idx and w.
 * It takes no context and allocates nothing: its k-NN buckets and status
 * word live in a 2 MiB device array that every GPU loading the library holds
 * until the process exits.  The first call on each device looks up that
 * array's device address (make that first call before any stream capture).
 * p may be NULL for (28, 7, 3).  n_beta may not exceed 65,536 (INVALID_ARG
 * beyond).  Every call uses the same array and overwrites what the previous
 * call left there; calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  Errors are
 * returned as codes only (no message).  Synchronises `stream`.
 */
int rbffd_build_weights_noalloc(const rbffd_params* p, const double* ax, const double* ay,
                                int64_t n_alpha, const double* bx, const double* by,
                                int64_t n_beta, uint32_t op_mask, int32_t* idx, double* w,
                                int64_t ld, int64_t* bad_node, cudaStream_t stream);

/* One ELL operator (see the conventions above). */
typedef struct rbffd_ell {
  const int32_t* idx; /* int32[n * ld]                                       */
  const void* w;      /* double or float [n * ld], per w_dtype               */
  int64_t n_rows;     /* alpha-nodes                                          */
  int64_t n_cols;     /* beta-nodes (every idx entry is < n_cols)            */
  int64_t ld;         /* leading dimension, >= n_rows, a multiple of 32      */
  int32_t n;          /* stencil size                                         */
  int32_t w_dtype;    /* RBFFD_F64 or RBFFD_F32                               */
} rbffd_ell;

/*
 * rbffd_apply_op - y = alpha * D x + beta * y (Section 2.2: D f(x^beta)
 * approximates L f(x^alpha)).  x has n_cols entries and y n_rows, both of
 * xy_dtype (RBFFD_F64 or RBFFD_F32).  With beta == 0, y is not read.
 * Accumulation is in FP64 for FP64 weights and in FP32 for FP32 weights.
 * Asynchronous, except that the first call for an operator shape (rows
 * rounded to a power of two, stencil size, weight and vector types) in a
 * context autotunes the launch shape: it times each candidate block size and
 * grid on this operator into context scratch (synchronising `stream`; skipped
 * while the stream is being captured) and keeps the fastest.  Every shape
 * adds a row's terms in the same order, so results do not depend on the
 * choice.  An operator with n_rows == 0 is a no-op (its arrays, x and y may
 * then be null).  Errors: INVALID_ARG (null pointer, bad shape or dtype), CUDA.
 */
int rbffd_apply_op(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, void* y, double alpha,
                   double beta, int32_t xy_dtype, cudaStream_t stream);

/*
 * rbffd_apply_op_shape - the launch shape rbffd_apply_op uses for this
 * operator shape in this context (threads per block, blocks per SM): the
 * autotuner's choice once a call has tuned it, the default before.  HOST
 * outputs.  Errors: INVALID_ARG.
 */
int rbffd_apply_op_shape(rbffd_ctx* ctx, const rbffd_ell* D, int32_t xy_dtype, int32_t* threads,
                         int32_t* blocks_per_sm);

/*
 * Staggered flow problem (Section 3).  Every operator is FP64 ELL with the
 * stencil size of the context; idx arrays index the beta set named second:
 *   vv_*: V-grid -> V-grid (N rows, ld_v), pv_*: V-values -> P-nodes
 *   (D^(P,V), M rows, ld_p), pp_*: P -> P (M rows, ld_p), vp_*: P-values ->
 *   V-nodes (D^(V,P), N rows, ld_v).
 * Boundary description:
 *   v_bc[i] != 0   V-node i lies on a wall; u, v there are Dirichlet data
 *   v_nx, v_ny     outward wall normal at wall V-nodes (unit length)
 *   p_bc[i] != 0   P-node i is a boundary node: its pressure row is the
 *                  homogeneous Neumann row p_nx D_x + p_ny D_y built on the
 *                  one-sided stencil pn_* below
 *   p_nx, p_ny     outward normal at boundary P-nodes
 *   nb_p, ld_b     number of boundary P-nodes; leading dimension of pn_*
 *   pn_rows        int32[nb_p]: the P-node of each Neumann row (every P-node
 *                  with p_bc != 0 appears exactly once)
 *   pn_idx, pn_dx, pn_dy  one-sided P -> P stencils of those nodes (slot 0 =
 *                  the node, then its nearest interior P-nodes), as built by
 *                  rbffd_build_weights_masked
 * Re, dt          Reynolds number and time step; a = dt / (2 Re)
 * precision       RBFFD_PREC_FP64 or RBFFD_PREC_MIXED
 * tol             relative residual of both implicit solves (scaled systems)
 * inner_tol       MIXED only: relative tolerance of each FP32 inner solve
 * max_iter        cap on Krylov iterations per solve (inner iterations summed)
 * km_mode         boundary value of the intermediate velocity (Kim & Moin,
 *                 end of Section 3): 2 = wall data + dt * D^(V,P) p~_j, both
 *                 components as printed (the binding's default); 1 = wall
 *                 data + dt * the component of D^(V,P) p~_j along the wall
 *                 tangent; 0 = wall data only
 * overwrite_bc    1 = set wall V-nodes to the wall data after the correction
 * profile         1 = time every SpMV launch of the pressure solves with CUDA
 *                 events on `stream` (reported in rbffd_stats); 0 = off
 * precond         pressure-solve preconditioner (not in the paper, which does
 *                 not say how it solves): 0 = none, 1 = one multigrid V-cycle
 *                 on the weighted graph Laplacian of the P-node edges (right
 *                 preconditioning; the converged solution is unchanged).  The
 *                 hierarchy is built on the host once per flow description.
 * p_edges         int32[n_edges][2]: the two P-nodes of each edge of the
 *                 staggered node set (each V-node sits at an edge midpoint)
 * p_x, p_y        P-node coordinates, device double[M] (edge weights
 *                 1/|x_a - x_b|^2); all three are read only when precond = 1
 * projection      RBFFD_PROJ_PAPER (the step below, as in Section 3) or
 *                 RBFFD_PROJ_EXACT: the pressure operator is the composition
 *                 D^(P,V) G0 of the divergence with the gradient D^(V,P) whose
 *                 wall rows are zero (built once per flow description, at most
 *                 kMaxComposed = 128 entries per row), so the corrected velocity
 *                 is discretely divergence-free at every P-node.  The paper
 *                 replaces that composition by D^(P,P)_Lap (Section 3); this
 *                 variant has no counterpart there.  Its step:
 *                   u** = g on wall rows; inside, the right side (per cn_form)
 *                   minus dt G0 p~_j (pressure-increment form; km_mode and
 *                   overwrite_bc are not used);
 *                   D^(P,V) G0 phi + mu e = F / dt on every P-node, 1^T phi
 *                   = 0, e = D^(P,V) w with w the wall normal (v_nx, v_ny) at
 *                   wall V-nodes;
 *                   u_{j+1} = u** - dt G0 phi - mu dt w (the one divergence
 *                   component no gradient can remove leaves as a uniform
 *                   wall-normal velocity mu dt, reported as wall_flux);
 *                   p~_{j+1} = p~_j + phi; p_{j+1} = p~_{j+1} - a D^(P,P)_Lap phi
 * cn_form         RBFFD_CN_PRINTED (Eq. u_ss, the default) or RBFFD_CN_KIM_MOIN
 *                 (right side u* + a D^(V,V)_Lap u_j, Kim & Moin's
 *                 Crank-Nicolson form; the printed one adds an O(dt) term)
 *
 * Open flows (Section 5.2, flow past a cylinder).  With v_bcu and v_bcv null
 * every boundary V-node (v_bc != 0) is a Dirichlet node for both components
 * and every boundary P-node a Neumann node, as in the cavity.  Otherwise:
 * v_bcu, v_bcv    uint8 [N]: per V-node and component 0 (interior; exactly
 *                 where v_bc is 0), RBFFD_BC_DIRICHLET (row u** = g_{j+1} +
 *                 dt D^(V,P) p~_j per km_mode 2/0, overwritten by g_{j+1} after
 *                 the correction) or RBFFD_BC_NEUMANN (row n.grad u** = 0,
 *                 corrected like an interior node)
 * nb_v, ld_vb     number of Neumann V-rows and their leading dimension
 *                 (a multiple of 32, >= nb_v)
 * vn_rows         int32 [nb_v]: the V-nodes with a Neumann row (every V-node
 *                 with a Neumann component, each once)
 * vn_idx          int32 [n][ld_vb]: their one-sided stencils, the node itself in
 *                 slot 0, then n-1 interior V-nodes (rbffd_build_weights_masked)
 * vn_dx, vn_dy    float64 [n][ld_vb]: D_x, D_y weights of those stencils; the row
 *                 is v_nx D_x + v_ny D_y
 * p_bc            RBFFD_PBC_DIRICHLET marks a Dirichlet pressure row (p~ = 0);
 *                 with any such row the pressure system is nonsingular: no
 *                 bordering, and p~ is not shifted to mean zero.  Such nodes
 *                 need no Neumann row in pn_rows.
 * Open flows run the paper's projection (projection = RBFFD_PROJ_PAPER) with
 * km_mode 0 or 2; rbffd_adjoint_step and rbffd_ensemble_step refuse them.
 */
typedef struct rbffd_flow {
  int64_t N, M, ld_v, ld_p;
  const int32_t* vv_idx;
  const double *vv_dx, *vv_dy, *vv_lap;
  const int32_t* pv_idx;
  const double *pv_dx, *pv_dy;
  const int32_t* pp_idx;
  const double *pp_dx, *pp_dy, *pp_lap;
  const int32_t* vp_idx;
  const double *vp_dx, *vp_dy;
  const uint8_t* v_bc;
  const double *v_nx, *v_ny;
  const uint8_t* p_bc;
  const double *p_nx, *p_ny;
  int64_t nb_p, ld_b;
  const int32_t* pn_rows;
  const int32_t* pn_idx;
  const double *pn_dx, *pn_dy;
  double Re, dt;
  int32_t precision;
  int32_t precond;
  double tol, inner_tol;
  int32_t max_iter;
  int32_t km_mode;
  int32_t overwrite_bc;
  int32_t profile;
  const int32_t* p_edges;
  int64_t n_edges;
  const double *p_x, *p_y;
  int32_t projection;
  int32_t cn_form;
  const uint8_t *v_bcu, *v_bcv;
  int64_t nb_v, ld_vb;
  const int32_t* vn_rows;
  const int32_t* vn_idx;
  const double *vn_dx, *vn_dy;
} rbffd_flow;

/* Solver state at step j (all FP64 device arrays owned by the caller). */
typedef struct rbffd_state {
  double *u, *v;             /* velocity at V-nodes, [N]                     */
  double *cu_prev, *cv_prev; /* convective terms C_{j-1}(u), C_{j-1}(v), [N] */
  double *pt;                /* pressure correction p~_j (mean zero), [M]    */
  double *p;                 /* pressure p_j, [M]                            */
  int64_t j;                 /* step counter; j == 0 uses C_{-1} = C_0       */
} rbffd_state;

/* Per-call statistics (host struct, filled by rbffd_step). */
typedef struct rbffd_stats {
  int64_t steps;            /* steps taken                                    */
  int64_t helm_iters;       /* Krylov iterations of the viscous solves        */
  int64_t poisson_iters;    /* Krylov iterations of the pressure solves      */
  int64_t refinements;      /* FP64 refinement sweeps (MIXED)                 */
  double helm_relres;       /* last relative residual, viscous solve         */
  double poisson_relres;    /* last relative residual, pressure solve        */
  int64_t launches;         /* kernels launched by this call                  */
  int64_t spmv_launches;    /* profile: timed SpMV launches of the pressure solves */
  double spmv_ms;           /* profile: their summed durations, milliseconds  */
  int64_t spmv_batch_launches; /* profile: the same SpMV relaunched back to back after
                                  each pressure solve (20 per solve)            */
  double spmv_batch_ms;     /* profile: their summed durations, milliseconds  */
  double wall_flux;         /* RBFFD_PROJ_EXACT: wall-normal velocity mu dt of the
                               last step; 0 otherwise                          */
  int64_t vspmv_batch_launches; /* profile, FP64 closed flows: the viscous SpMV (two
                                   right sides) relaunched back to back after each
                                   viscous solve (20 per solve)                 */
  double vspmv_batch_ms;    /* profile: their summed durations, milliseconds  */
} rbffd_stats;

/*
 * rbffd_step - advance `n_steps` fractional steps (Section 3):
 *  1. C_j(q) = -[u o D^(V,V)_x q + v o D^(V,V)_y q]; u* = u_j + dt (3/2 C_j - 1/2 C_{j-1})
 *  2. (I - a D^(V,V)_Lap) u** = (I + a D^(V,V)_Lap) u* (Eq. u_ss), wall rows = identity
 *     with the Kim & Moin value (km_mode); likewise v**
 *  3. F = D^(P,V)_x u** + D^(P,V)_y v** (Eq. divergence); D^(P,P)_Lap p~ = F/dt
 *     (Eq. pressure_Poisson) at every interior P-node, homogeneous Neumann
 *     rows at boundary P-nodes; the constant null space is removed by the
 *     bordered system [L e; 1^T 0] with e = 1 on the boundary rows (the
 *     multiplier takes up the incompatibility there); p~ has zero mean
 *  4. p = p~ - a D^(P,P)_Lap p~;  u_{j+1} = u** - dt D^(V,P)_x p~, v likewise
 *     (Eq. velocity_next_timestep); wall nodes set to the wall data
 * gu, gv: device double[N], wall data g_{j+1} (used at wall V-nodes only),
 * held fixed over the n_steps of one call.  state is updated in place;
 * state->j advances by n_steps.  stats (HOST, may be NULL) is filled.
 * Errors: INVALID_ARG, NOT_CONVERGED (state holds the last iterate), NONFINITE,
 * CUDA, OOM.  Synchronises `stream`.
 */
int rbffd_step(rbffd_ctx* ctx, const rbffd_flow* flow, rbffd_state* state, const double* gu,
               const double* gv, int32_t n_steps, rbffd_stats* stats, cudaStream_t stream);

/*
 * rbffd_stencil_condition - condition numbers of the local systems.
 *
 * Section 4.2 (the histograms of cond(A_aug) used to choose q): for every
 * alpha-node, the 1-norm condition number ||A_aug||_1 ||A_aug^-1||_1 of the
 * augmented matrix [A P; P^T 0] of Eq. rbf_poly_compact that
 * rbffd_build_weights factors for that node, i.e. in local coordinates
 * (shifted to the alpha-node, scaled by the largest stencil radius), with
 * the context's (n, m, q).  The inverse is formed from the same LU with
 * partial pivoting (one solve per unit vector, FP64).
 * idx        int32[n * ld]: the stencils (as written by rbffd_build_weights)
 * cond       out: double[n_alpha]; +inf for a singular system
 * Errors: INVALID_ARG, CUDA, OOM.  Synchronises `stream`.
 */
int rbffd_stencil_condition(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t n_alpha,
                            const double* bx, const double* by, int64_t n_beta,
                            const int32_t* idx, int64_t ld, double* cond, cudaStream_t stream);

/*
 * rbffd_modified_wavenumber - Eq. 2d_mw at every alpha-node.
 *
 * Section 4.1: for the plane wave exp(i k.x) with k = (kx, ky) and
 * k~ = |k|, the radial derivative delta_r = (kx D_x + ky D_y) / k~ gives the
 * modified wavenumber k* = -i delta_r{exp(i k.x)} exp(-i k.x_0).  Output
 * k1[i] = k* / k~ (complex, interleaved re, im); when Dlap is given, also
 * k2[i] = -D_Lap{exp(i k.x)} exp(-i k.x_0) / k~^2 (the second-derivative
 * counterpart, 1 for an exact operator).  The phase of every stencil node is
 * taken relative to the alpha-node.  Dx, Dy: FP64 ELL operators of the same
 * shape (rows = alpha-nodes, columns = beta-nodes); Dlap may be NULL.
 * ax, ay  alpha-node coordinates; bx, by  beta-node coordinates.
 * k1, k2  out: double[2 * n_rows] (k2 ignored when Dlap is NULL).
 * Errors: INVALID_ARG (shapes, dtype, k = 0), CUDA.  Asynchronous.
 */
int rbffd_modified_wavenumber(rbffd_ctx* ctx, const rbffd_ell* Dx, const rbffd_ell* Dy,
                              const rbffd_ell* Dlap, const double* ax, const double* ay,
                              const double* bx, const double* by, double kx, double ky,
                              double* k1, double* k2, cudaStream_t stream);

/*
 * rbffd_stencil_error - per-node relative error of an operator (Section 4,
 * Eq. test and Eq. relative_error).
 *
 * For alpha-node i the test function is g_i(x, y) = cos(x / dr_i) cos(y / dr_i)
 * with dr_i the local spacing; the error is |(D g_i)_i - L g_i(x_i)| divided
 * by max |L g_i| (1 for RBFFD_OP_INTERP, 1/dr_i for RBFFD_OP_DX and _DY,
 * 2/dr_i^2 for RBFFD_OP_LAP).  The paper's E is the mean over the nodes.
 * D        FP64 ELL operator of the operation `op` (one RBFFD_OP_* bit)
 * dr       device double[n_rows] or NULL: NULL takes dr_i as the mean distance
 *          from the alpha-node to stencil slots 1..6, which for a collocated
 *          operator (slot 0 = the node itself) is the mean distance to its 6
 *          nearest nodes; needs n >= 7
 * err      out: double[n_rows]
 * err_mean out (device double, may be NULL): the mean of err, summed in a
 *          fixed order
 * Errors: INVALID_ARG, CUDA, OOM.  Asynchronous.
 */
int rbffd_stencil_error(rbffd_ctx* ctx, const rbffd_ell* D, uint32_t op, const double* ax,
                        const double* ay, const double* bx, const double* by, const double* dr,
                        double* err, double* err_mean, cudaStream_t stream);

/*
 * rbffd_debug_set_wait_limit - test hook (no counterpart in the paper): the
 * number of polls the step's kernels spend on their first wait for a tile or
 * record staged into shared memory before they give up.  polls = 0 makes
 * every such wait give up at once; polls < 0 restores the default (2^22).
 * A kernel that gives up still waits, up to the default limit, for the copies
 * it issued, sets the solve's error flag and returns; the step then fails
 * with RBFFD_ERR_CUDA ("... bounded wait") and the context stays usable.
 * The setting is per process and device (the current one), not per context.
 * Errors: INVALID_ARG (null ctx), CUDA.
 */
int rbffd_debug_set_wait_limit(rbffd_ctx* ctx, int64_t polls);

/*
 * rbffd_ensemble_step - advance an ensemble of independent flows that share
 * one node set and its operators (the batching of many flows at once; the
 * paper runs one flow at a time).  Member e is the step of rbffd_step
 * (Section 3, the paper's projection) with Reynolds number Re[e] and its own
 * wall data, in the MIXED design (FP32 explicit stages and inner Krylov
 * solves, FP64 refinement of both implicit solves to flow->tol).  Every
 * operator is read once per row for all members.
 * flow       the shared flow description (flow->Re and flow->precision are
 *            not used; projection must be RBFFD_PROJ_PAPER)
 * n_members  E, a power of two from 1 to 64
 * Re         HOST double[E]
 * state      member-contiguous device arrays: u, v, cu_prev, cv_prev hold
 *            double[N * E] with member e of V-node i at [i * E + e]; pt, p hold
 *            double[M * E]; j is shared by the members
 * gu, gv     device double[N * E], wall data of every member (same layout)
 * Errors: INVALID_ARG, NOT_CONVERGED, NONFINITE, CUDA, OOM.  Synchronises
 * `stream`; stats (HOST, may be NULL) sums the Krylov iterations over the
 * batched solves (one iteration advances every member).
 */
int rbffd_ensemble_step(rbffd_ctx* ctx, const rbffd_flow* flow, int32_t n_members,
                        const double* Re, rbffd_state* state, const double* gu, const double* gv,
                        int32_t n_steps, rbffd_stats* stats, cudaStream_t stream);

/*
 * rbffd_probe_fma - measured FMA throughput of the device (no counterpart in
 * the paper): 8 independent FMA chains per thread, 8 blocks of 256 threads
 * per SM, `iters` FMAs per chain, timed with CUDA events on `stream`.
 * dtype RBFFD_F64 or RBFFD_F32; *gflops (HOST) receives 2 * FMAs / s / 1e9.
 * Used as the arithmetic roofline of the FP64 weight solves.  Synchronises.
 */
int rbffd_probe_fma(rbffd_ctx* ctx, int32_t dtype, int32_t iters, double* gflops,
                    cudaStream_t stream);

/* Adjoint variables of a state (FP64 device arrays owned by the caller):
 * dJ/du, dJ/dv (N), dJ/dC_{j-1}(u), dJ/dC_{j-1}(v) (N), dJ/dp~ (M). */
typedef struct rbffd_adjoint {
  double *u, *v, *cu_prev, *cv_prev, *pt;
} rbffd_adjoint;

/*
 * rbffd_adjoint_step - reverse-mode derivative of one rbffd_step step (the
 * discrete adjoint of Section 3's three stages under the same readings: Kim &
 * Moin wall term per km_mode, wall overwrite, AB2 start, bordered pressure).
 * fwd    the forward state the step started from (step j; only u, v and j are
 *        read: the step is linear in everything else)
 * lam    in: adjoints of the step's outputs (state j+1); out: adjoints of its
 *        inputs (state j), in place
 * grad_gu, grad_gv  device double[N]: the adjoint of the step's wall data
 *        g_{j+1} is ADDED to them (wall entries only)
 * The operators of the step are transposed once per flow description (kept in
 * the context).  Transposed solves use the flow's tol and max_iter.  FP64.
 * Only the paper's step (projection = RBFFD_PROJ_PAPER, cn_form =
 * RBFFD_CN_PRINTED) has an adjoint; other flows give INVALID_ARG.
 * A training loop stores checkpoints of forward states and recomputes the
 * states between them before walking backwards.  Errors: as rbffd_step.
 * Synchronises `stream`; stats (HOST, may be NULL) receives the iteration
 * counts of the transposed solves.
 */
int rbffd_adjoint_step(rbffd_ctx* ctx, const rbffd_flow* flow, const rbffd_state* fwd,
                       rbffd_adjoint* lam, double* grad_gu, double* grad_gv, rbffd_stats* stats,
                       cudaStream_t stream);

/*
 * rbffd_cylinder_forces - drag and lift coefficients of a circular body
 * (Section 5.2): C = F / (1/2 rho U^2 D) with rho = U = 1 and D = 2 radius,
 * F the force of the fluid on the body, the integral over its surface of
 * (-p I + (grad U + grad U^T) / Re) n with n the unit normal from the body
 * into the fluid, by composite Simpson's rule in the angle.
 *   flow    the flow description (its D^(P,V) operators and P-node
 *           coordinates p_x, p_y are used; p_x, p_y must be set)
 *   u, v    velocity at the V-nodes, float64 [N], device
 *   p       pressure at the P-nodes, float64 [M], device
 *   rows    int32 [n_c], device: the body's surface P-nodes, equally spaced in
 *           angle about (cx, cy), in increasing angle; n_c even, at least 4
 *   radius  the body's radius; Re the Reynolds number of the viscous stress
 *   cd_cl   double[2], HOST: C_D (along +x) and C_L (along +y)
 * Synchronous.  Errors: INVALID_ARG (null pointers, odd or small n_c, a row
 * outside [0, M), missing coordinates), CUDA.
 */
int rbffd_cylinder_forces(rbffd_ctx* ctx, const rbffd_flow* flow, const double* u,
                          const double* v, const double* p, const int32_t* rows, int32_t n_c,
                          double cx, double cy, double radius, double Re, double* cd_cl,
                          cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RBFFD_H */
