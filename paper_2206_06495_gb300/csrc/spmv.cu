// Operator application y = alpha * D x + beta * y for slot-major ELL operators
// (Section 2.2).  One thread per row: for each stencil slot the warp reads 32
// consecutive idx and w entries (one coalesced line each) and gathers x from
// L2.  With the paper's n = 28 the slot loop is fully unrolled so every load of
// a row is in flight at once.
//
// Launch shape (block size and blocks per SM) is picked by a small autotuner:
// the first call for an operator shape (rows rounded to a power of two, stencil
// size, weight and vector types) times every candidate on the caller's own
// operator, writing into context scratch, and keeps the fastest for the
// context.  Every candidate adds each row's terms in the same order, so the
// choice never changes the result.
#include <algorithm>

#include "common.cuh"

namespace rbffd {
namespace {

template <typename T>
struct AccOf;
template <>
struct AccOf<double> {
  using type = double;
};
template <>
struct AccOf<float> {
  using type = float;
};

template <int K, typename TW, typename TX, int BS>
__global__ void __launch_bounds__(BS) ell_apply(const int32_t* __restrict__ idx,
                                                const TW* __restrict__ w, int64_t n_rows,
                                                int64_t ld, int k_rt, const TX* __restrict__ x,
                                                TX* __restrict__ y, double alpha, double beta) {
  using A = typename AccOf<TW>::type;
  const int k = K > 0 ? K : k_rt;
  for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * BS) {
    A acc = 0;
    if (K > 0) {
#pragma unroll
      for (int s = 0; s < K; ++s) acc += (A)w[s * ld + i] * (A)x[idx[s * ld + i]];
    } else {
      for (int s = 0; s < k; ++s) acc += (A)w[s * ld + i] * (A)x[idx[s * ld + i]];
    }
    A out = (A)alpha * acc;
    if (beta != 0.0) out += (A)beta * (A)y[i];
    y[i] = (TX)out;
  }
}

// candidate launch shapes: (threads per block, blocks per SM), at most 2048
// resident threads per SM
struct Shape {
  int bs, bps;
};
constexpr Shape kShapes[] = {{128, 4}, {128, 8}, {128, 16}, {256, 2}, {256, 4},
                             {256, 8}, {512, 2}, {512, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kDefaultShape = 5;  // 256 threads, 8 blocks per SM

template <int K, typename TW, typename TX>
void launch_k(const rbffd_ell* D, const void* x, void* y, double alpha, double beta, int shape,
              cudaStream_t st) {
  const Shape s = kShapes[shape];
  const int blocks =
      (int)std::max<int64_t>(1, std::min<int64_t>((D->n_rows + s.bs - 1) / s.bs,
                                                  (int64_t)sm_count() * s.bps));
  const TW* w = (const TW*)D->w;
  switch (s.bs) {
    case 128:
      ell_apply<K, TW, TX, 128><<<blocks, 128, 0, st>>>(D->idx, w, D->n_rows, D->ld, D->n,
                                                         (const TX*)x, (TX*)y, alpha, beta);
      break;
    case 512:
      ell_apply<K, TW, TX, 512><<<blocks, 512, 0, st>>>(D->idx, w, D->n_rows, D->ld, D->n,
                                                         (const TX*)x, (TX*)y, alpha, beta);
      break;
    default:
      ell_apply<K, TW, TX, 256><<<blocks, 256, 0, st>>>(D->idx, w, D->n_rows, D->ld, D->n,
                                                         (const TX*)x, (TX*)y, alpha, beta);
  }
}

template <typename TW, typename TX>
void launch(const rbffd_ell* D, const void* x, void* y, double alpha, double beta, int shape,
            cudaStream_t st) {
  if (D->n == 28)
    launch_k<28, TW, TX>(D, x, y, alpha, beta, shape, st);
  else
    launch_k<0, TW, TX>(D, x, y, alpha, beta, shape, st);
}

void launch_any(const rbffd_ell* D, const void* x, void* y, double alpha, double beta,
                int32_t xy_dtype, int shape, cudaStream_t st) {
  if (D->w_dtype == RBFFD_F64) {
    if (xy_dtype == RBFFD_F64)
      launch<double, double>(D, x, y, alpha, beta, shape, st);
    else
      launch<double, float>(D, x, y, alpha, beta, shape, st);
  } else {
    if (xy_dtype == RBFFD_F64)
      launch<float, double>(D, x, y, alpha, beta, shape, st);
    else
      launch<float, float>(D, x, y, alpha, beta, shape, st);
  }
}

uint64_t shape_key(const rbffd_ell* D, int32_t xy_dtype) {
  int lg = 0;
  while (lg < 62 && (int64_t(1) << lg) < D->n_rows) ++lg;
  return (uint64_t)lg | ((uint64_t)D->n << 8) | ((uint64_t)D->w_dtype << 24) |
         ((uint64_t)xy_dtype << 28);
}

// Time every candidate shape (one warm-up and three timed launches each) into
// scratch output; returns the fastest, or the default if anything fails.
int tune(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, int32_t xy_dtype, cudaStream_t st) {
  const size_t ybytes = (size_t)D->n_rows * (xy_dtype == RBFFD_F64 ? 8 : 4);
  void* scratch = nullptr;
  if (ctx_scratch(ctx, ybytes, &scratch) != RBFFD_OK) return kDefaultShape;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return kDefaultShape;
  }
  int best = kDefaultShape;
  float best_ms = 0.f;
  for (int s = 0; s < kNumShapes; ++s) {
    launch_any(D, x, scratch, 1.0, 0.0, xy_dtype, s, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) launch_any(D, x, scratch, 1.0, 0.0, xy_dtype, s, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      best = kDefaultShape;
      break;
    }
    if (s == 0 || ms < best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  return best;
}

}  // namespace

int spmv_apply(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, void* y, double alpha,
               double beta, int32_t xy_dtype, cudaStream_t st) {
  const uint64_t key = shape_key(D, xy_dtype);
  int shape = -1;
  for (const auto& kv : ctx->spmv_shapes)
    if (kv.first == key) shape = kv.second;
  if (shape < 0) {
    // tuning synchronises the stream: not while it is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      shape = tune(ctx, D, x, xy_dtype, st);
      ctx->spmv_shapes.emplace_back(key, shape);
    } else {
      cudaGetLastError();
      shape = kDefaultShape;
    }
  }
  launch_any(D, x, y, alpha, beta, xy_dtype, shape, st);
  return check_cuda(ctx, cudaGetLastError(), "ell_apply");
}

int spmv_shape(rbffd_ctx* ctx, const rbffd_ell* D, int32_t xy_dtype, int* threads,
               int* blocks_per_sm) {
  const uint64_t key = shape_key(D, xy_dtype);
  for (const auto& kv : ctx->spmv_shapes)
    if (kv.first == key) {
      *threads = kShapes[kv.second].bs;
      *blocks_per_sm = kShapes[kv.second].bps;
      return RBFFD_OK;
    }
  *threads = kShapes[kDefaultShape].bs;
  *blocks_per_sm = kShapes[kDefaultShape].bps;
  return RBFFD_OK;
}

}  // namespace rbffd
