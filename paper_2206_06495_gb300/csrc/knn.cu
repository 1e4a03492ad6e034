// Stencil search (Section 2.2: each alpha-node uses its n nearest beta-nodes).
//
// A uniform bucket grid over the bounding box of both node sets holds about
// two beta-nodes per cell.  Buckets are built with a counting sort (count,
// exclusive scan, scatter).  Each alpha-node (one thread) then scans rings of
// cells around its own cell, keeping the k best candidates ordered by
// (squared distance, index); it stops once no point outside the rings seen so
// far can beat the current k-th candidate.  Squared distances are formed as
// dx*dx + dy*dy with each operation rounded on its own, so the ordering
// (including ties) is reproducible on any IEEE machine.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace rbffd {
namespace {

constexpr int kScanBlock = 1024;

__global__ void bbox_partial(const double* __restrict__ ax, const double* __restrict__ ay,
                             int64_t na, const double* __restrict__ bx,
                             const double* __restrict__ by, int64_t nb, double* out) {
  double mnx = DBL_MAX, mny = DBL_MAX, mxx = -DBL_MAX, mxy = -DBL_MAX;
  const int64_t n = na + nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x = i < na ? ax[i] : bx[i - na];
    double y = i < na ? ay[i] : by[i - na];
    mnx = fmin(mnx, x);
    mny = fmin(mny, y);
    mxx = fmax(mxx, x);
    mxy = fmax(mxy, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mnx = fmin(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
    mny = fmin(mny, __shfl_xor_sync(0xffffffffu, mny, o));
    mxx = fmax(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
    mxy = fmax(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
  }
  __shared__ double sh[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sh[0][wid] = mnx;
    sh[1][wid] = mny;
    sh[2][wid] = mxx;
    sh[3][wid] = mxy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      mnx = fmin(mnx, sh[0][w]);
      mny = fmin(mny, sh[1][w]);
      mxx = fmax(mxx, sh[2][w]);
      mxy = fmax(mxy, sh[3][w]);
    }
    out[blockIdx.x * 4 + 0] = mnx;
    out[blockIdx.x * 4 + 1] = mny;
    out[blockIdx.x * 4 + 2] = mxx;
    out[blockIdx.x * 4 + 3] = mxy;
  }
}

struct Grid {
  double x0, y0, cell, inv_cell;
  int gx, gy;
};

__device__ __forceinline__ int cell_of(double v, double v0, double inv, int g) {
  int c = (int)floor((v - v0) * inv);
  return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__global__ void bucket_count(const double* __restrict__ bx, const double* __restrict__ by,
                             int64_t nb, const uint8_t* __restrict__ mask, Grid g,
                             int* __restrict__ cell_id, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask && !mask[i]) {
      cell_id[i] = -1;
      continue;
    }
    int cx = cell_of(bx[i], g.x0, g.inv_cell, g.gx);
    int cy = cell_of(by[i], g.y0, g.inv_cell, g.gy);
    int c = cy * g.gx + cx;
    cell_id[i] = c;
    atomicAdd(&counts[c], 1);
  }
}

// Exclusive scan, three phases: per-block scan, scan of block totals, add.
__global__ void scan_blocks(const int* __restrict__ in, int* __restrict__ out, int n,
                            int* __restrict__ block_tot) {
  __shared__ int sh[kScanBlock];
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == kScanBlock - 1) block_tot[blockIdx.x] = sh[threadIdx.x];
}

__global__ void scan_totals(int* block_tot, int nblocks) {
  // one block; sequential chunks keep it simple and exact
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += kScanBlock) {
    __shared__ int sh[kScanBlock];
    int i = base + threadIdx.x;
    int v = i < nblocks ? block_tot[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
      int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblocks) block_tot[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
}

__global__ void scan_add(int* __restrict__ out, int n, const int* __restrict__ block_off,
                         int* __restrict__ cursor, const int* __restrict__ counts) {
  int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) {
    int v = out[i] + block_off[blockIdx.x];
    out[i] = v;
    cursor[i] = v;
    // sentinel: end of the last cell = number of bucketed (unmasked) points
    if (i == n - 1) out[n] = v + counts[i];
  }
}

__global__ void bucket_scatter(int64_t nb, const int* __restrict__ cell_id,
                               int* __restrict__ cursor, int* __restrict__ cell_pts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell_id[i];
    if (c < 0) continue;
    int pos = atomicAdd(&cursor[c], 1);
    cell_pts[pos] = (int)i;
  }
}

__device__ __forceinline__ bool better(double d, int j, double bd, int bj) {
  return d < bd || (d == bd && j < bj);
}

// Optional forms: beta_mask excludes beta-nodes whose mask is 0 (they were
// never bucketed); alpha_self puts a given beta index in slot 0 and searches
// the remaining k-1 slots.
template <int KMAX>
__global__ void __launch_bounds__(128) knn_query(
    const double* __restrict__ ax, const double* __restrict__ ay, int64_t na,
    const double* __restrict__ bx, const double* __restrict__ by,
    const int* __restrict__ cell_start, const int* __restrict__ cell_pts, Grid g, int k_all,
    const int32_t* __restrict__ alpha_self, int32_t* __restrict__ idx, int64_t ld) {
  const int off = alpha_self ? 1 : 0;
  const int k = k_all - off;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (alpha_self) idx[i] = alpha_self[i];
    if (k == 0) continue;
    const double qx = ax[i], qy = ay[i];
    const int cx = cell_of(qx, g.x0, g.inv_cell, g.gx);
    const int cy = cell_of(qy, g.y0, g.inv_cell, g.gy);
    // distance from the query to the sides of its own cell (0 if clamped)
    double ex = fmin(qx - (g.x0 + cx * g.cell), (g.x0 + (cx + 1) * g.cell) - qx);
    double ey = fmin(qy - (g.y0 + cy * g.cell), (g.y0 + (cy + 1) * g.cell) - qy);
    const double edge = fmax(0.0, fmin(ex, ey));
    double bd[KMAX];
    int bi[KMAX];
    int cnt = 0;
    for (int r = 0;; ++r) {
      const int x_lo = cx - r, x_hi = cx + r, y_lo = cy - r, y_hi = cy + r;
      for (int yy = y_lo; yy <= y_hi; ++yy) {
        if (yy < 0 || yy >= g.gy) continue;
        const bool full_row = (yy == y_lo || yy == y_hi);
        const int step = full_row ? 1 : (x_hi - x_lo);
        for (int xx = x_lo; xx <= x_hi; xx += (step > 0 ? step : 1)) {
          if (xx < 0 || xx >= g.gx) continue;
          const int c = yy * g.gx + xx;
          const int p1 = cell_start[c + 1];
          for (int p = cell_start[c]; p < p1; ++p) {
            const int j = cell_pts[p];
            const double dx = __dsub_rn(bx[j], qx);
            const double dy = __dsub_rn(by[j], qy);
            const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            if (cnt < k) {
              int s = cnt++;
              while (s > 0 && better(d2, j, bd[s - 1], bi[s - 1])) {
                bd[s] = bd[s - 1];
                bi[s] = bi[s - 1];
                --s;
              }
              bd[s] = d2;
              bi[s] = j;
            } else if (better(d2, j, bd[k - 1], bi[k - 1])) {
              int s = k - 1;
              while (s > 0 && better(d2, j, bd[s - 1], bi[s - 1])) {
                bd[s] = bd[s - 1];
                bi[s] = bi[s - 1];
                --s;
              }
              bd[s] = d2;
              bi[s] = j;
            }
          }
        }
      }
      const bool covered = x_lo <= 0 && y_lo <= 0 && x_hi >= g.gx - 1 && y_hi >= g.gy - 1;
      if (covered) break;
      if (cnt == k) {
        // every point outside the (2r+1)^2 block is at least this far away
        const double lb = r * g.cell + edge;
        if (bd[k - 1] < lb * lb * (1.0 - 1e-12)) break;
      }
    }
    for (int s = 0; s < k; ++s) idx[(s + off) * ld + i] = bi[s];
  }
}

}  // namespace

int knn_build(rbffd_ctx* ctx, const double* ax, const double* ay, int64_t na, const double* bx,
              const double* by, int64_t nb, const uint8_t* beta_mask,
              const int32_t* alpha_self, int k, int32_t* idx, int64_t ld, cudaStream_t st) {
  const int sms = sm_count();
  // --- bounding box
  const int bb_blocks = 64;  // partials fit the pinned status buffer
  // scratch layout: [bbox partials][cell_id nb][counts cells+1][cursor cells][cell_pts nb][block_tot]
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_bb = carve(sizeof(double) * 4 * bb_blocks);
  void* base = nullptr;
  int rc = ctx_scratch(ctx, off, &base);
  if (rc) return rc;
  double* d_bb = (double*)((char*)base + o_bb);
  bbox_partial<<<bb_blocks, 256, 0, st>>>(ax, ay, na, bx, by, nb, d_bb);
  rc = check_cuda(ctx, cudaGetLastError(), "bbox kernel");
  if (rc) return rc;
  double* h_bb = (double*)ctx->host_pinned;
  rc = check_cuda(ctx, cudaMemcpyAsync(h_bb, d_bb, sizeof(double) * 4 * bb_blocks,
                                       cudaMemcpyDeviceToHost, st),
                  "bbox copy");
  if (rc) return rc;
  rc = check_cuda(ctx, cudaStreamSynchronize(st), "bbox sync");
  if (rc) return rc;
  double x0 = DBL_MAX, y0 = DBL_MAX, x1 = -DBL_MAX, y1 = -DBL_MAX;
  for (int b = 0; b < bb_blocks; ++b) {
    x0 = fmin(x0, h_bb[4 * b + 0]);
    y0 = fmin(y0, h_bb[4 * b + 1]);
    x1 = fmax(x1, h_bb[4 * b + 2]);
    y1 = fmax(y1, h_bb[4 * b + 3]);
  }
  if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(x1) || !std::isfinite(y1))
    return set_error(ctx, RBFFD_ERR_NONFINITE, "non-finite node coordinates");
  double w = x1 - x0, h = y1 - y0;
  double span = fmax(fmax(w, h), 1e-300);
  if (w < 1e-9 * span) w = 1e-9 * span;
  if (h < 1e-9 * span) h = 1e-9 * span;
  double cell = sqrt(w * h * 2.0 / (double)nb);
  Grid g;
  for (;;) {
    double gx = ceil(w / cell), gy = ceil(h / cell);
    if (gx * gy <= 4.0 * (double)nb + 16.0 && gx < 1e8 && gy < 1e8) {
      g.gx = (int)fmax(gx, 1.0);
      g.gy = (int)fmax(gy, 1.0);
      break;
    }
    cell *= 1.5;
  }
  g.x0 = x0;
  g.y0 = y0;
  g.cell = cell;
  g.inv_cell = 1.0 / cell;
  const int cells = g.gx * g.gy;
  const int scan_blocks_n = (cells + kScanBlock - 1) / kScanBlock;
  off = 0;
  carve(sizeof(double) * 4 * bb_blocks);
  const size_t o_cid = carve(sizeof(int) * nb);
  const size_t o_cnt = carve(sizeof(int) * (cells + 1));
  const size_t o_start = carve(sizeof(int) * (cells + 1));
  const size_t o_cur = carve(sizeof(int) * cells);
  const size_t o_pts = carve(sizeof(int) * nb);
  const size_t o_tot = carve(sizeof(int) * (scan_blocks_n + 1));
  rc = ctx_scratch(ctx, off, &base);
  if (rc) return rc;
  char* b = (char*)base;
  int* d_cid = (int*)(b + o_cid);
  int* d_cnt = (int*)(b + o_cnt);
  int* d_start = (int*)(b + o_start);
  int* d_cur = (int*)(b + o_cur);
  int* d_pts = (int*)(b + o_pts);
  int* d_tot = (int*)(b + o_tot);
  rc = check_cuda(ctx, cudaMemsetAsync(d_cnt, 0, sizeof(int) * (cells + 1), st), "memset");
  if (rc) return rc;
  const int gblocks = 4 * sms;
  bucket_count<<<gblocks, 256, 0, st>>>(bx, by, nb, beta_mask, g, d_cid, d_cnt);
  scan_blocks<<<scan_blocks_n, kScanBlock, 0, st>>>(d_cnt, d_start, cells, d_tot);
  scan_totals<<<1, kScanBlock, 0, st>>>(d_tot, scan_blocks_n);
  scan_add<<<scan_blocks_n, kScanBlock, 0, st>>>(d_start, cells, d_tot, d_cur, d_cnt);
  bucket_scatter<<<gblocks, 256, 0, st>>>(nb, d_cid, d_cur, d_pts);
  const int qblocks = (int)std::min<int64_t>((na + 127) / 128, (int64_t)sms * 32);
  if (k <= 32)
    knn_query<32><<<qblocks, 128, 0, st>>>(ax, ay, na, bx, by, d_start, d_pts, g, k, alpha_self,
                                           idx, ld);
  else
    knn_query<64><<<qblocks, 128, 0, st>>>(ax, ay, na, bx, by, d_start, d_pts, g, k, alpha_self,
                                           idx, ld);
  return check_cuda(ctx, cudaGetLastError(), "knn kernels");
}

}  // namespace rbffd

namespace rbffd {

// Scratch bytes the search below needs for n_beta beta-nodes when the bucket
// grid is limited to max_cells cells.
size_t knn_scratch_bytes(int64_t nb, int64_t max_cells) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const int64_t scan_blocks_n = (max_cells + kScanBlock - 1) / kScanBlock;
  return up(sizeof(double) * 4 * 64) + up(sizeof(int) * nb) + 2 * up(sizeof(int) * (max_cells + 1)) +
         up(sizeof(int) * max_cells) + up(sizeof(int) * nb) + up(sizeof(int) * (scan_blocks_n + 1));
}

// The stencil search of knn_build on caller-provided device scratch: no
// allocation, no context.  The bucket grid is coarsened until it has at most
// max_cells cells (the result does not depend on the grid).  Returns an
// RBFFD status code.
int knn_build_scratch(const double* ax, const double* ay, int64_t na, const double* bx,
                      const double* by, int64_t nb, int k, int32_t* idx, int64_t ld,
                      void* scratch, size_t scratch_bytes, int64_t max_cells, cudaStream_t st) {
  const int sms = sm_count();
  const int bb_blocks = 64;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  char* b = (char*)scratch;
  const size_t o_bb = carve(sizeof(double) * 4 * bb_blocks);
  double* d_bb = (double*)(b + o_bb);
  bbox_partial<<<bb_blocks, 256, 0, st>>>(ax, ay, na, bx, by, nb, d_bb);
  double h_bb[4 * 64];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h_bb, d_bb, sizeof(h_bb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RBFFD_ERR_CUDA;
  double x0 = DBL_MAX, y0 = DBL_MAX, x1 = -DBL_MAX, y1 = -DBL_MAX;
  for (int q = 0; q < bb_blocks; ++q) {
    x0 = fmin(x0, h_bb[4 * q + 0]);
    y0 = fmin(y0, h_bb[4 * q + 1]);
    x1 = fmax(x1, h_bb[4 * q + 2]);
    y1 = fmax(y1, h_bb[4 * q + 3]);
  }
  if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(x1) || !std::isfinite(y1))
    return RBFFD_ERR_NONFINITE;
  double w = x1 - x0, h = y1 - y0;
  const double span = fmax(fmax(w, h), 1e-300);
  if (w < 1e-9 * span) w = 1e-9 * span;
  if (h < 1e-9 * span) h = 1e-9 * span;
  double cell = sqrt(w * h * 2.0 / (double)nb);
  Grid g;
  for (;;) {
    const double gx = ceil(w / cell), gy = ceil(h / cell);
    if (gx * gy <= (double)max_cells && gx < 1e8 && gy < 1e8) {
      g.gx = (int)fmax(gx, 1.0);
      g.gy = (int)fmax(gy, 1.0);
      break;
    }
    cell *= 1.5;
  }
  g.x0 = x0;
  g.y0 = y0;
  g.cell = cell;
  g.inv_cell = 1.0 / cell;
  const int cells = g.gx * g.gy;
  const int scan_blocks_n = (cells + kScanBlock - 1) / kScanBlock;
  const size_t o_cid = carve(sizeof(int) * nb);
  const size_t o_cnt = carve(sizeof(int) * (cells + 1));
  const size_t o_start = carve(sizeof(int) * (cells + 1));
  const size_t o_cur = carve(sizeof(int) * cells);
  const size_t o_pts = carve(sizeof(int) * nb);
  const size_t o_tot = carve(sizeof(int) * (scan_blocks_n + 1));
  if (off > scratch_bytes) return RBFFD_ERR_INVALID_ARG;
  int* d_cid = (int*)(b + o_cid);
  int* d_cnt = (int*)(b + o_cnt);
  int* d_start = (int*)(b + o_start);
  int* d_cur = (int*)(b + o_cur);
  int* d_pts = (int*)(b + o_pts);
  int* d_tot = (int*)(b + o_tot);
  // the scratch keeps the previous call's contents: the counters start at zero
  if (cudaMemsetAsync(d_cnt, 0, sizeof(int) * (cells + 1), st) != cudaSuccess)
    return RBFFD_ERR_CUDA;
  const int gblocks = 4 * sms;
  bucket_count<<<gblocks, 256, 0, st>>>(bx, by, nb, nullptr, g, d_cid, d_cnt);
  scan_blocks<<<scan_blocks_n, kScanBlock, 0, st>>>(d_cnt, d_start, cells, d_tot);
  scan_totals<<<1, kScanBlock, 0, st>>>(d_tot, scan_blocks_n);
  scan_add<<<scan_blocks_n, kScanBlock, 0, st>>>(d_start, cells, d_tot, d_cur, d_cnt);
  bucket_scatter<<<gblocks, 256, 0, st>>>(nb, d_cid, d_cur, d_pts);
  const int qblocks = (int)std::min<int64_t>((na + 127) / 128, (int64_t)sms * 32);
  if (k <= 32)
    knn_query<32><<<qblocks, 128, 0, st>>>(ax, ay, na, bx, by, d_start, d_pts, g, k, nullptr,
                                           idx, ld);
  else
    knn_query<64><<<qblocks, 128, 0, st>>>(ax, ay, na, bx, by, d_start, d_pts, g, k, nullptr,
                                           idx, ld);
  return cudaGetLastError() == cudaSuccess ? RBFFD_OK : RBFFD_ERR_CUDA;
}

}  // namespace rbffd
