// Shared device helpers and the context definition of the CUDA path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "rbffd.h"

namespace rbffd {

constexpr int kWarp = 32;
constexpr int kMaxStencil = 64;  // largest n accepted by the ABI
constexpr int kMaxSystem = 96;   // largest n + (q+1)(q+2)/2
constexpr size_t kHostPinnedBytes = 65536;  // per-context pinned status buffer

// Number of SMs on the current device; grid sizes are multiples of it.
int sm_count();

// -------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values per thread in a fixed order (deterministic for
// a fixed block size).  Result valid in thread 0.  `sh` holds at least
// NV * blockDim.x doubles.  The threads only store their values; warp 0 adds
// them (each lane a strided column, then one butterfly), so a block issues
// about (blockDim.x / 32 + 4) FP64 adds per value instead of five per value
// in every warp: FP64 instructions are scarce on this GPU.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j * nt + tid] = v[j];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double a = sh[j * nt + tid];
      for (int k = tid + 32; k < nt; k += 32) a += sh[j * nt + k];
      v[j] = warp_sum(a);
    }
  }
  __syncthreads();
}

// Grid-wide deterministic reduction via "last block finishes": every block
// writes its partial sums, the last block to arrive adds all partials in
// block order with a fixed tree and runs `fin` on the totals in thread 0.
// No block waits on another; the counter is reset by the last block.
struct GridReduce {
  double* partials;       // [gridDim.x * NV]
  unsigned int* counter;  // one word, zero between launches
};

template <int NV, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], GridReduce gr, double* sh, Fin fin) {
  block_sum<NV>(v, sh);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) gr.partials[blockIdx.x * NV + j] = v[j];
    __threadfence();
    unsigned int t = atomicAdd(gr.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] += ((volatile double*)gr.partials)[b * NV + j];
  }
  block_sum<NV>(acc, sh);
  if (threadIdx.x == 0) {
    fin(acc);
    *gr.counter = 0u;
  }
}

}  // namespace rbffd

// ------------------------------------------------------------------ context
namespace rbffd {
struct StepPlan;
struct EnsPlan;
}

struct rbffd_ctx {
  rbffd_params prm;
  std::string err;
  // scratch owned by the context (grown on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* host_pinned = nullptr;  // small pinned buffer for status words
  rbffd::StepPlan* plan = nullptr;
  rbffd::EnsPlan* ens = nullptr;  // ensemble step plan (rbffd_ensemble_step)
  // launch shapes the SpMV autotuner picked, per operator shape key
  std::vector<std::pair<uint64_t, int>> spmv_shapes;
};

namespace rbffd {

int set_error(rbffd_ctx* ctx, int code, const char* fmt, ...);
int check_cuda(rbffd_ctx* ctx, cudaError_t e, const char* what);
// grow-only device scratch of the context
int ctx_scratch(rbffd_ctx* ctx, size_t bytes, void** out);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// entry points implemented per translation unit
int knn_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
              const double* by, int64_t nb, const uint8_t* beta_mask,
              const int32_t* alpha_self, int k, int32_t* idx, int64_t ld, cudaStream_t st);
int weights_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
                  const double* by, const int32_t* idx, int64_t ld, uint32_t op_mask, double* w,
                  int64_t* bad_node, cudaStream_t st);
int spmv_apply(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, void* y, double alpha,
               double beta, int32_t xy_dtype, cudaStream_t st);
int spmv_shape(rbffd_ctx* ctx, const rbffd_ell* D, int32_t xy_dtype, int* threads,
               int* blocks_per_sm);
int step_run(rbffd_ctx* ctx, const rbffd_flow* f, rbffd_state* s, const double* gu,
             const double* gv, int32_t n_steps, rbffd_stats* stats, cudaStream_t st);
void step_plan_free(struct StepPlan* p);
int step_set_wait_limit(rbffd_ctx* ctx, long long polls);
int adjoint_run(rbffd_ctx* ctx, const rbffd_flow* f, const rbffd_state* s, rbffd_adjoint* lam,
                double* grad_gu, double* grad_gv, rbffd_stats* stats, cudaStream_t st);
int ensemble_run(rbffd_ctx* ctx, const rbffd_flow* f, int E, const double* Re, rbffd_state* s,
                 const double* gu, const double* gv, int32_t n_steps, rbffd_stats* stats,
                 cudaStream_t st);
void ens_plan_free(struct EnsPlan* p);
int cond_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
               const double* by, const int32_t* idx, int64_t ld, double* cond, cudaStream_t st);
int analysis_mw(rbffd_ctx* ctx, const rbffd_ell* Dx, const rbffd_ell* Dy, const rbffd_ell* Dl,
                const double* ax, const double* ay, const double* bx, const double* by,
                double kx, double ky, double* k1, double* k2, cudaStream_t st);
int analysis_forces(rbffd_ctx* ctx, const rbffd_flow& f, const double* u, const double* v,
                    const double* p, const int32_t* rows, int32_t n_c, double cx, double cy,
                    double radius, double Re, double* out_host, cudaStream_t st);
int analysis_error(rbffd_ctx* ctx, const rbffd_ell* D, int op, const double* ax,
                   const double* ay, const double* bx, const double* by, const double* dr,
                   double* err, double* mean, cudaStream_t st);
// allocation-free variants on caller-provided device scratch (status codes only)
size_t knn_scratch_bytes(int64_t nb, int64_t max_cells);
int knn_build_scratch(const double* ax, const double* ay, int64_t na, const double* bx,
                      const double* by, int64_t nb, int k, int32_t* idx, int64_t ld,
                      void* scratch, size_t scratch_bytes, int64_t max_cells, cudaStream_t st);
int weights_build_scratch(int n, int m, int q, const double* ax, const double* ay, int64_t na,
                          const double* bx, const double* by, const int32_t* idx, int64_t ld,
                          uint32_t op_mask, double* w, unsigned long long* d_bad,
                          int64_t* bad_node, cudaStream_t st);

}  // namespace rbffd
