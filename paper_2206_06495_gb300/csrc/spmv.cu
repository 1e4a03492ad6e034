// Operator application y = alpha * D x + beta * y for slot-major ELL operators
// (Section 2.2).  One thread per row: for each stencil slot the warp reads 32
// consecutive idx and w entries (one coalesced line each) and gathers x from
// L2.  With the paper's n = 28 the slot loop is fully unrolled so every load of
// a row is in flight at once.
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

template <int K, typename TW, typename TX>
__global__ void __launch_bounds__(256) ell_apply(const int32_t* __restrict__ idx,
                                                 const TW* __restrict__ w, int64_t n_rows,
                                                 int64_t ld, int k_rt, const TX* __restrict__ x,
                                                 TX* __restrict__ y, double alpha, double beta) {
  using A = typename AccOf<TW>::type;
  const int k = K > 0 ? K : k_rt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
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

template <typename TW, typename TX>
void launch(const rbffd_ell* D, const void* x, void* y, double alpha, double beta, int blocks,
            cudaStream_t st) {
  const TW* w = (const TW*)D->w;
  if (D->n == 28)
    ell_apply<28, TW, TX><<<blocks, 256, 0, st>>>(D->idx, w, D->n_rows, D->ld, D->n,
                                                   (const TX*)x, (TX*)y, alpha, beta);
  else
    ell_apply<0, TW, TX><<<blocks, 256, 0, st>>>(D->idx, w, D->n_rows, D->ld, D->n,
                                                  (const TX*)x, (TX*)y, alpha, beta);
}

}  // namespace

int spmv_apply(rbffd_ctx* ctx, const rbffd_ell* D, const void* x, void* y, double alpha,
               double beta, int32_t xy_dtype, cudaStream_t st) {
  const int sms = sm_count();
  const int blocks = (int)std::min<int64_t>((D->n_rows + 255) / 256, (int64_t)sms * 8);
  if (D->w_dtype == RBFFD_F64) {
    if (xy_dtype == RBFFD_F64)
      launch<double, double>(D, x, y, alpha, beta, blocks, st);
    else
      launch<double, float>(D, x, y, alpha, beta, blocks, st);
  } else {
    if (xy_dtype == RBFFD_F64)
      launch<float, double>(D, x, y, alpha, beta, blocks, st);
    else
      launch<float, float>(D, x, y, alpha, beta, blocks, st);
  }
  return check_cuda(ctx, cudaGetLastError(), "ell_apply");
}

}  // namespace rbffd
