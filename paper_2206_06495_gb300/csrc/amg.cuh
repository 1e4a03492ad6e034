// Multigrid preconditioner of the pressure solve.
//
// The paper solves its pressure Poisson system without saying how; an
// unpreconditioned Krylov method needs O(1/h) iterations on it.  Both the
// scaled RBF-FD Laplacian and the weighted graph Laplacian of the P-node
// edges (the edges whose midpoints are the V-nodes of the staggered node set,
// Section 3) approximate the same continuous operator, so the graph Laplacian
// G is spectrally close to it with bounds that do not depend on h.  G is a
// symmetric M-matrix with zero row sums: plain aggregation multigrid on it is
// robust, while a multigrid on the RBF-FD matrix itself is not (its Jacobi
// iteration grows transiently near the walls).  One V-cycle on G is the right
// preconditioner of BiCGSTAB; it changes the iteration count, not the
// solution, which is still the converged solve of the RBF-FD system.
//
// G: edge weight 1/|x_a - x_b|^2; an edge between two boundary P-nodes is left
// out (boundary rows of the pressure system are one-sided Neumann rows on
// interior nodes) unless one of its ends has no other edge to an interior node.
// Hierarchy: two passes of pairwise matching by strongest normalised coupling
// per level (aggregates of up to 4 nodes), Galerkin coarse matrices P^T G P
// with piecewise-constant P, down to at most kAmgCoarse nodes, where the dense
// inverse of (G_c + sigma 1 1^T) is applied.  Every level is renumbered so that
// each aggregate's rows are contiguous (level 0 through the permutation perm0).  Smoother: one damped Jacobi
// sweep before and after the coarse correction, which is scaled by
// kAmgCoarseScale (the usual over-correction of plain aggregation).
// The hierarchy is built once per flow description on the host (like a
// symbolic factorisation); every V-cycle operation runs in CUDA kernels, in
// FP32 (a preconditioner only has to be a fixed linear map).
#pragma once

#include <vector>

#include "common.cuh"

namespace rbffd {

constexpr int kAmgMaxLevels = 16;
constexpr int kAmgCoarse = 2048;  // coarsest level: at most this many rows, solved densely
constexpr float kAmgOmega = 0.8f;
constexpr float kAmgCoarseScale = 2.0f;

// One level of the hierarchy (device arrays).  Rows of level l + 1 are the
// aggregates of level l.  The coarsest level holds only r, z and the dense
// inverse.
struct AmgLevel {
  int64_t n = 0, ld = 0;   // rows; leading dimension of the slot-major arrays
  int width = 0;           // off-diagonal slots per row (padding: own index, weight 0)
  int32_t* idx = nullptr;  // [width][ld] off-diagonal columns
  float* val = nullptr;    // [width][ld] off-diagonal entries (<= 0)
  float* diag = nullptr;   // [n]
  float* wd = nullptr;     // [n] omega / diag
  int32_t* cptr = nullptr;  // [n(l+1) + 1]: rows cptr[I] .. cptr[I+1]-1 form aggregate I
                            // (row I of level l + 1); at most four rows each
  float* r = nullptr;      // right side at this level
  float* x = nullptr;      // pre-smoothed iterate
  float* z = nullptr;      // level result (after the post-smoothing sweep)
};

// Block records of a level.  The restriction of level l gives each block the
// kRecAggs consecutive aggregates 64 b .. 64 b + 63 of level l + 1, whose rows
// are the consecutive level-l rows f0 .. f0 + nrows - 1 (at most kRecRows).
// The record of block b holds what is static about those rows (graph row, its
// diagonal and Jacobi weight, and aux: on level 0 the P-node index of each
// row, above it the first row on level l - 1 of each row's aggregate, nrows + 1
// entries) in the layout one bulk copy stages into shared memory; the sweep
// of the level takes the same blocks.
constexpr int kRecAggs = 64;
constexpr int kRecRows = 256;

template <int W>
struct LevelRec {
  int32_t f0, nrows, nagg, pad;
  int32_t off[kRecAggs + 4];  // aggregate I = 64 b + t: rows f0 + off[t] .. f0 + off[t+1] - 1
  int32_t idx[W * kRecRows];  // slot s of row f0 + r at [s * kRecRows + r]
  float val[W * kRecRows];
  float diag[kRecRows];
  float wd[kRecRows];
  int32_t aux[kRecRows + 4];
};

struct Amg {
  int nlev = 0;
  AmgLevel lev[kAmgMaxLevels];
  float* Xc = nullptr;  // [nc][nc] dense inverse on the coarsest level
  int32_t* perm0 = nullptr;  // [M] level-0 row p is P-node perm0[p] (the nested order)
  int64_t nc = 0;
  // level-0 map of a residual v of the scaled pressure system: r0 = c v - mu ce,
  // mu = (c . v) / (c . es); the result is z + mu / M (see step.cu)
  float* c = nullptr;   // [M] diag(G) / diag(A), in the level-0 order
  float* cnode = nullptr;  // [M] the same in P-node order (for (c . v) of Krylov vectors)
  float* ce = nullptr;  // [M] c * es
  float *zp = nullptr, *zs = nullptr;     // [M] V-cycle results for p and s (B v = z + kap), FP32 solves
  double *zpd = nullptr, *zsd = nullptr;  // the same for FP64 solves
  double inv_ces = 0.0;
  double inv_R = 0.0;
  // block records of each level with a restriction (LevelRec<rec_w[l]>), or null
  unsigned char* rec[kAmgMaxLevels] = {};
  int rec_w[kAmgMaxLevels] = {};      // slot count: 8 or 16 (the level's width at most that)
  int64_t rec_n[kAmgMaxLevels] = {};  // number of records (blocks of kRecAggs aggregates)
  std::vector<int> sizes;  // rows per level (host copy, for reports)
  std::vector<void*> allocs;
};

// Build the hierarchy of the flow's P-node edge graph.  diag_a and es are
// HOST copies (M values) of the diagonal and the rank-one column of the scaled
// pressure operator.  Errors: INVALID_ARG (edges out of range, coincident
// endpoints, a P-node without edges, a graph that does not coarsen), CUDA, OOM.
int amg_build(rbffd_ctx* ctx, const rbffd_flow& f, const double* diag_a, const double* es,
              Amg** out, cudaStream_t st);
void amg_free(Amg* a);

}  // namespace rbffd
