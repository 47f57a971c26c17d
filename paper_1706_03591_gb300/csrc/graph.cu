// Graph ingest for the normalized Laplacian (Section 2.1): degrees and D^{-1/2}.
//
// L = I - D^{-1/2} W D^{-1/2}; the recursion runs on L~ = L - I = -D^{-1/2} W D^{-1/2}
// (spectrum in [-1, 1]).  An isolated node keeps scale 0, so its L~ row is zero.
// vs / ivs are the row scales of the value-free recursion (V_j = vs T_j): D^{-1/2} and
// D^{1/2}, with 1 for isolated nodes (no row gathers from them, so any nonzero value works).
#include <algorithm>

#include "csc_internal.h"

namespace csc {

namespace {

__global__ void graph_prep_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                  const float* __restrict__ val, double* __restrict__ deg,
                                  float* __restrict__ scale, float* __restrict__ vs,
                                  float* __restrict__ ivs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    double dsum;
    if (val == nullptr) {
      dsum = (double)(e - b);
    } else {
      dsum = 0.0;
      for (int64_t p = b; p < e; ++p) dsum += (double)val[p];
    }
    deg[i] = dsum;
    scale[i] = dsum > 0.0 ? (float)(1.0 / sqrt(dsum)) : 0.0f;
    vs[i] = dsum > 0.0 ? (float)(1.0 / sqrt(dsum)) : 1.0f;
    ivs[i] = dsum > 0.0 ? (float)sqrt(dsum) : 1.0f;
  }
}

// Counts CSR violations: bad row pointers, column out of range, self-loops,
// unsorted or duplicate columns within a row, non-positive weights.
__global__ void graph_check_kernel(int64_t n, int64_t nnz, const int64_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col, const float* __restrict__ val,
                                   unsigned long long* bad) {
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    if (b < 0 || e < b || e > nnz) { ++local; continue; }
    int32_t prev = -1;
    for (int64_t p = b; p < e; ++p) {
      const int32_t c = col[p];
      if (c < 0 || c >= n || c == i || c <= prev) ++local;
      if (val != nullptr && !(val[p] > 0.0f)) ++local;
      prev = c;
    }
  }
  if (local) atomicAdd(bad, local);
}

// Edge-block partition for the recursion: block b holds the rows whose first stored edge
// lies in [b*E, (b+1)*E) (lower bound on row_ptr); the last block ends at row n.
__global__ void block_rows_kernel(int64_t n, const int64_t* __restrict__ row_ptr, int64_t per_block,
                                  int nblk, int32_t* __restrict__ blk_row) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nblk; b += gridDim.x * blockDim.x) {
    if (b == 0) { blk_row[0] = 0; continue; }
    if (b == nblk) { blk_row[nblk] = (int32_t)n; continue; }
    const int64_t target = (int64_t)b * per_block;
    int64_t lo = 0, hi = n;  // first r in [0, n] with row_ptr[r] >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] < target) lo = mid + 1; else hi = mid;
    }
    blk_row[b] = (int32_t)lo;
  }
}

// First row whose weight row_ptr[r] + kRowCost r reaches b * kBlockWeight, for every block b.
__global__ void weight_rows_kernel(int64_t n, const int64_t* __restrict__ row_ptr, int nblk,
                                   int32_t* __restrict__ srow) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nblk; b += gridDim.x * blockDim.x) {
    if (b == 0) { srow[0] = 0; continue; }
    if (b == nblk) { srow[nblk] = (int32_t)n; continue; }
    const int64_t target = (int64_t)b * kBlockWeight;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] + kRowCost * mid < target) lo = mid + 1; else hi = mid;
    }
    srow[b] = (int32_t)lo;
  }
}

// deg[i] = degree of caller row perm[i].
__global__ void internal_degree_kernel(int64_t n, const int64_t* __restrict__ urp, const int32_t* __restrict__ perm,
                                       long long* __restrict__ deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = perm[i];
    deg[i] = (long long)(urp[u + 1] - urp[u]);
  }
}

// row_ptr[0] = 0, row_ptr[i + 1] = inclusive scan of the internal degrees.
__global__ void shift_offsets_kernel(int64_t n, const long long* __restrict__ incl, int64_t* __restrict__ rp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    rp[i] = i == 0 ? 0 : (int64_t)incl[i - 1];
}

// Internal row i: the caller row perm[i] with its neighbours mapped through iperm (one warp per row).
__global__ void permute_rows_kernel(int64_t n, const int64_t* __restrict__ urp, const int32_t* __restrict__ ucol,
                                    const float* __restrict__ uval, const int32_t* __restrict__ perm,
                                    const int32_t* __restrict__ iperm, const int64_t* __restrict__ rp,
                                    int32_t* __restrict__ col, float* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t src = urp[perm[i]], len = urp[perm[i] + 1] - src, dst = rp[i];
    for (int64_t k = lane; k < len; k += 32) {
      col[dst + k] = iperm[ucol[src + k]];
      if (val != nullptr) val[dst + k] = uval[src + k];
    }
  }
}

__global__ void gather_i32_kernel(int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                                  const int32_t* __restrict__ map, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[map[i]];
}

__global__ void scatter_edges_kernel(int64_t n, const int64_t* __restrict__ rp, const int64_t* __restrict__ urp,
                                     const int32_t* __restrict__ perm, const float* __restrict__ src,
                                     float* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t b = rp[i], len = rp[i + 1] - b, u = urp[perm[i]];
    for (int64_t k = lane; k < len; k += 32) dst[u + k] = src[b + k];
  }
}

int flat_grid(int64_t items) {
  int64_t g = (items + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

cudaError_t launch_permute_graph(Graph& g, long long* deg_tmp, long long* sums, cudaStream_t s) {
  const int64_t n = g.n;
  // the internal degrees go to g.deg (recomputed from the new CSR by launch_graph_prep)
  long long* deg = (long long*)g.deg.ptr;
  internal_degree_kernel<<<flat_grid(n), 256, 0, s>>>(n, (const int64_t*)g.urp.ptr, (const int32_t*)g.perm.ptr,
                                                      deg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = inclusive_scan_i64(deg, deg_tmp, n, sums, s)) != cudaSuccess) return e;
  shift_offsets_kernel<<<flat_grid(n + 1), 256, 0, s>>>(n, deg_tmp, (int64_t*)g.row_ptr.ptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int warps_grid = std::max(1, std::min(num_sms() * 16, (int)((n + 7) / 8)));
  permute_rows_kernel<<<warps_grid, 256, 0, s>>>(n, (const int64_t*)g.urp.ptr, (const int32_t*)g.ucol.ptr,
                                                 g.weighted ? (const float*)g.uval.ptr : nullptr,
                                                 (const int32_t*)g.perm.ptr, (const int32_t*)g.iperm.ptr,
                                                 (const int64_t*)g.row_ptr.ptr, (int32_t*)g.col.ptr,
                                                 g.weighted ? (float*)g.val.ptr : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gather_i32(int32_t* dst, const int32_t* src, const int32_t* map, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_i32_kernel<<<flat_grid(n), 256, 0, s>>>(dst, src, map, n);
  return cudaGetLastError();
}

cudaError_t launch_scatter_edges(const Graph& g, const float* src, float* dst, cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  const int warps_grid = std::max(1, std::min(num_sms() * 16, (int)((g.n + 7) / 8)));
  scatter_edges_kernel<<<warps_grid, 256, 0, s>>>(g.n, (const int64_t*)g.row_ptr.ptr, (const int64_t*)g.urp.ptr,
                                                  (const int32_t*)g.perm.ptr, src, dst);
  return cudaGetLastError();
}

int row_blocks(int64_t n, int64_t nnz) {
  const int64_t nb = (nnz + kRowCost * n + kBlockWeight - 1) / kBlockWeight;
  return (int)(nb < 1 ? 1 : nb);
}

int edge_blocks(int64_t nnz) {
  const int64_t nb = (nnz + kEdgesPerBlock - 1) / kEdgesPerBlock;
  return (int)(nb < 1 ? 1 : nb);
}

cudaError_t launch_block_rows(const Graph& g, cudaStream_t s) {
  const int nblk = edge_blocks(g.nnz);
  const int grid = (nblk + 1 + 255) / 256;
  block_rows_kernel<<<grid, 256, 0, s>>>(g.n, (const int64_t*)g.row_ptr.ptr, kEdgesPerBlock, nblk,
                                         (int32_t*)g.blk_row.ptr);
  const int nsblk = row_blocks(g.n, g.nnz);
  weight_rows_kernel<<<(nsblk + 1 + 255) / 256, 256, 0, s>>>(g.n, (const int64_t*)g.row_ptr.ptr, nsblk,
                                                            (int32_t*)g.srow.ptr);
  return cudaGetLastError();
}

cudaError_t launch_graph_prep(const Graph& g, cudaStream_t s) {
  if (g.n == 0) return cudaSuccess;
  const int block = 256;
  int grid = (int)((g.n + block - 1) / block);
  if (grid > num_sms() * 8) grid = num_sms() * 8;
  graph_prep_kernel<<<grid, block, 0, s>>>(g.n, (const int64_t*)g.row_ptr.ptr,
                                           g.weighted ? (const float*)g.val.ptr : nullptr,
                                           (double*)g.deg.ptr, (float*)g.scale.ptr,
                                           (float*)g.vs.ptr, (float*)g.ivs.ptr);
  return cudaGetLastError();
}

cudaError_t launch_graph_check(const Graph& g, unsigned long long* bad, cudaStream_t s) {
  if (g.n == 0) return cudaSuccess;
  const int block = 256;
  int grid = (int)((g.n + block - 1) / block);
  if (grid > num_sms() * 8) grid = num_sms() * 8;
  graph_check_kernel<<<grid, block, 0, s>>>(g.n, g.nnz, (const int64_t*)g.row_ptr.ptr,
                                            (const int32_t*)g.col.ptr,
                                            g.weighted ? (const float*)g.val.ptr : nullptr, bad);
  return cudaGetLastError();
}

}  // namespace csc
