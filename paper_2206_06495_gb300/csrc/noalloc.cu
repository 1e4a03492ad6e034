// rbffd_build_weights_noalloc: stencils and weights without any allocation.
//
// For callers that may not allocate GPU memory themselves or through this
// library: code running inside a host framework that owns the device memory
// pool and forbids other cudaMalloc calls, or a loop with a fixed memory
// budget that cannot afford cudaMalloc/cudaFree and the device-wide
// synchronisation they can imply.  The k-NN buckets and the status word live
// in one file-scope device array of fixed size, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
#include "common.cuh"

namespace rbffd {
namespace {

constexpr size_t kNoAllocScratchBytes = 2u << 20;  // 2 MiB per device
constexpr int64_t kNoAllocMaxBeta = 65536;          // largest n_beta accepted

// Device scratch shared by every call of the entry point below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch in the current context.  In host code the
// array's name is only a host-side stand-in, so the address is looked up on
// every call: the lookup allocates nothing and does not synchronise, and a
// cached address would outlive the context it belongs to (cudaDeviceReset
// destroys the context and the module; the next context loads the module
// afresh, possibly at another address).
int scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RBFFD_ERR_CUDA;
  *out = p;
  return RBFFD_OK;
}

}  // namespace
}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_build_weights_noalloc(const rbffd_params* p, const double* ax,
                                           const double* ay, int64_t n_alpha, const double* bx,
                                           const double* by, int64_t n_beta, uint32_t op_mask,
                                           int32_t* idx, double* w, int64_t ld,
                                           int64_t* bad_node, cudaStream_t stream) {
  if (bad_node) *bad_node = -1;
  const rbffd_params prm = p ? *p : rbffd_params{28, 7, 3};
  const int np = prm.q < 0 ? 0 : (prm.q + 1) * (prm.q + 2) / 2;
  if (prm.n < 1 || prm.n > kMaxStencil || prm.m < 3 || prm.m > 13 || (prm.m % 2) == 0 ||
      prm.q < -1 || prm.q > 5 || prm.n < np || prm.n + np > kMaxSystem)
    return RBFFD_ERR_INVALID_ARG;
  if (n_alpha < 0 || n_beta < 0 || (op_mask & 15u) == 0 || (op_mask & ~15u))
    return RBFFD_ERR_INVALID_ARG;
  if (n_alpha == 0) return RBFFD_OK;
  if (n_beta < prm.n || n_beta > kNoAllocMaxBeta || n_alpha > INT32_MAX) return RBFFD_ERR_INVALID_ARG;
  if (!ax || !ay || !bx || !by || !idx || !w || ld < n_alpha || ld % 32)
    return RBFFD_ERR_INVALID_ARG;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  // layout: [status word (256 B)] [k-NN buckets]
  unsigned long long* d_bad = (unsigned long long*)base;
  char* knn_scratch = (char*)base + 256;
  const size_t knn_bytes = kNoAllocScratchBytes - 256;
  const int64_t max_cells = n_beta + 16;  // about two beta-nodes per bucket or fewer buckets
  if (knn_scratch_bytes(n_beta, max_cells) > knn_bytes) return RBFFD_ERR_INVALID_ARG;
  rc = knn_build_scratch(ax, ay, n_alpha, bx, by, n_beta, prm.n, idx, ld, knn_scratch, knn_bytes,
                         max_cells, stream);
  if (rc) return rc;
  return weights_build_scratch(prm.n, prm.m, prm.q, ax, ay, n_alpha, bx, by, idx, ld, op_mask, w,
                               d_bad, bad_node, stream);
}
