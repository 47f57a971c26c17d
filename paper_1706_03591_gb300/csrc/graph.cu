// Graph ingest for the normalized Laplacian (Section 2.1): degrees and D^{-1/2}.
//
// L = I - D^{-1/2} W D^{-1/2}; the recursion runs on L~ = L - I = -D^{-1/2} W D^{-1/2}
// (spectrum in [-1, 1]).  An isolated node keeps scale 0, so its L~ row is zero.
// vs / ivs are the row scales of the value-free recursion (V_j = vs T_j): D^{-1/2} and
// D^{1/2}, with 1 for isolated nodes (no row gathers from them, so any nonzero value works).
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

}  // namespace

int edge_blocks(int64_t nnz) {
  const int64_t nb = (nnz + kEdgesPerBlock - 1) / kEdgesPerBlock;
  return (int)(nb < 1 ? 1 : nb);
}

cudaError_t launch_block_rows(const Graph& g, cudaStream_t s) {
  const int nblk = edge_blocks(g.nnz);
  const int grid = (nblk + 1 + 255) / 256;
  block_rows_kernel<<<grid, 256, 0, s>>>(g.n, (const int64_t*)g.row_ptr.ptr, kEdgesPerBlock, nblk,
                                         (int32_t*)g.blk_row.ptr);
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
