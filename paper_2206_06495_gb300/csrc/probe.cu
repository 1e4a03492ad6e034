// Throughput probes of the FP64 and FP32 FMA pipes (used to report the weight
// build and the FP64 stages against a measured arithmetic peak).
#include "common.cuh"

namespace rbffd {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ out, int iters, T b, T c) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
    a4 = fma(a4, b, c);
    a5 = fma(a5, b, c);
    a6 = fma(a6, b, c);
    a7 = fma(a7, b, c);
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
double run_probe(rbffd_ctx* ctx, int iters, cudaStream_t st, int* rc) {
  const int blocks = sm_count() * 8, threads = 256;
  void* buf = nullptr;
  *rc = ctx_scratch(ctx, sizeof(T) * blocks * threads, &buf);
  if (*rc) return 0.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads, 0, st>>>((T*)buf, iters / 8, (T)0.999999, (T)1e-7);  // warm
  cudaEventRecord(e0, st);
  k_fma_chains<T><<<blocks, threads, 0, st>>>((T*)buf, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  *rc = check_cuda(ctx, cudaEventSynchronize(e1), "probe");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*rc || ms <= 0.f) return 0.0;
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return flops / (ms * 1e-3) / 1e9;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_probe_fma(rbffd_ctx* ctx, int32_t dtype, int32_t iters, double* gflops,
                               cudaStream_t stream) {
  if (!ctx || !gflops || iters < 8 || (dtype != RBFFD_F64 && dtype != RBFFD_F32))
    return RBFFD_ERR_INVALID_ARG;
  int rc = 0;
  *gflops = dtype == RBFFD_F64 ? run_probe<double>(ctx, iters, stream, &rc)
                               : run_probe<float>(ctx, iters, stream, &rc);
  return rc;
}
