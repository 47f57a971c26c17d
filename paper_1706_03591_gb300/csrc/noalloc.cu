// Allocation-free Chebyshev filtering for small graphs (csc_cheb_filter_noalloc).
//
// Some callers cannot call cudaMalloc while they run.  A framework whose caching allocator
// reserved the device memory up front may have nothing left to give, and an allocation outside
// that allocator fragments what it manages.  A latency-bound service may forbid allocation
// after start-up, because cudaMalloc and cudaFree can synchronise the whole device and stall
// every other stream.  This entry point takes only caller-owned device buffers (graph,
// signals, output) and keeps all of its scratch in one file-scope static device array of fixed
// size, sized for graphs of at most kMaxN nodes and kMaxNnz stored edges and orders of at most
// kMaxM.  The array exists on every GPU that loads this library, until the process exits.
//
// It runs the same kernels as csc_cheb_filter with a column tile of 8.  The host reads the
// moments of each tile back through host memory and synchronises the caller's stream before
// returning.  The scratch address is looked up once per device with cudaGetSymbolAddress: the
// first call on a device does that look-up, which loads the module, so that first call should
// come before any stream capture.  All calls share the one array, which keeps the last call's
// contents (every region a call reads is written by that call first): calls that overlap on
// the GPU (different streams, or different host threads) race on it and must be serialised by
// the caller.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "csc_internal.h"

namespace {

constexpr int64_t kMaxN = 65536;
constexpr int64_t kMaxNnz = int64_t(1) << 22;
constexpr int kMaxM = 128;
constexpr int kTile = 8;
constexpr int kMaxGrid = 512;
constexpr int kMaxRows = 2 * kMaxM + 1;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Scratch layout (bytes).
constexpr size_t kOffScale = 0;
constexpr size_t kOffVs = kOffScale + align256(kMaxN * 4);
constexpr size_t kOffIvs = kOffVs + align256(kMaxN * 4);
constexpr size_t kOffDeg = kOffIvs + align256(kMaxN * 4);
constexpr size_t kOffBlk = kOffDeg + align256(kMaxN * 8);
constexpr size_t kOffSrow = kOffBlk + align256((kMaxNnz / csc::kEdgesPerBlock + 2) * 4);
constexpr size_t kOffT =
    kOffSrow + align256(((kMaxNnz + csc::kRowCost * kMaxN) / csc::kBlockWeight + 2) * 4);
constexpr size_t kOffPsi = kOffT + 3 * align256(kMaxN * kTile * 4);
constexpr size_t kOffCoef = kOffPsi + align256(kMaxN * kTile * 4);
constexpr size_t kOffPart = kOffCoef + align256((kMaxM + 1) * 4);
constexpr size_t kOffEf = kOffPart + align256((size_t)kMaxRows * kMaxGrid * 8);
constexpr size_t kScratchBytes = kOffEf + align256(kMaxRows * 8);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

#define NA_CHECK(call)                           \
  do {                                           \
    if ((call) != cudaSuccess) return CSC_ECUDA; \
  } while (0)

extern "C" csc_status csc_cheb_filter_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr,
                                              const int32_t* col_idx, const float* vals, int m,
                                              double lambda_c, const float* R, int c, int64_t ldr,
                                              float* psi_out, int64_t ldp, double* mu_out,
                                              void* cuda_stream) {
  if (n < 1 || nnz < 0 || !row_ptr || (nnz > 0 && !col_idx) || m < 1 || c < 1 || !R || ldr < c ||
      !(lambda_c >= 0.0 && lambda_c <= 2.0) || (psi_out && ldp < c))
    return CSC_EINVAL;
  if (n > kMaxN || nnz > kMaxNnz || m > kMaxM) return CSC_ELIMIT;
  // every array is read or written by kernels: host pointers are refused
  const void* dev_ptrs[] = {row_ptr, nnz > 0 ? col_idx : nullptr, vals, R, psi_out};
  for (const void* p : dev_ptrs) {
    if (p == nullptr) continue;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return CSC_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return CSC_EINVAL;
  }
  unsigned char* base = nullptr;
  NA_CHECK(scratch_address(&base));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  using csc::DevBuf;
  // graph view over caller buffers and scratch (no ownership)
  csc::Graph g;
  g.n = n;
  g.nnz = nnz;
  g.weighted = vals != nullptr;
  g.row_ptr.ptr = const_cast<int64_t*>(row_ptr);
  g.col.ptr = const_cast<int32_t*>(col_idx);
  g.val.ptr = const_cast<float*>(vals);
  g.scale.ptr = base + kOffScale;
  g.vs.ptr = base + kOffVs;
  g.ivs.ptr = base + kOffIvs;
  g.deg.ptr = base + kOffDeg;
  g.blk_row.ptr = base + kOffBlk;
  g.srow.ptr = base + kOffSrow;
  NA_CHECK(csc::launch_graph_prep(g, s));
  NA_CHECK(csc::launch_block_rows(g, s));
  float* tb[3] = {reinterpret_cast<float*>(base + kOffT),
                  reinterpret_cast<float*>(base + kOffT + align256(kMaxN * kTile * 4)),
                  reinterpret_cast<float*>(base + kOffT + 2 * align256(kMaxN * kTile * 4))};
  float* psi = reinterpret_cast<float*>(base + kOffPsi);
  float* coef = reinterpret_cast<float*>(base + kOffCoef);
  double* part = reinterpret_cast<double*>(base + kOffPart);
  double* ef = reinterpret_cast<double*>(base + kOffEf);
  double a[kMaxM + 1];
  float af[kMaxM + 1];
  csc::filter_coeffs(m, lambda_c, a);
  for (int j = 0; j <= m; ++j) af[j] = (float)a[j];
  NA_CHECK(cudaMemcpyAsync(coef, af, (size_t)(m + 1) * 4, cudaMemcpyHostToDevice, s));
  const int grid = std::min(csc::cheb_grid(kTile), kMaxGrid);
  const int rows = 2 * m + 1;
  double ef_sum[kMaxRows];
  double ef_tile[kMaxRows];
  for (int r = 0; r < rows; ++r) ef_sum[r] = 0.0;
  const int ntiles = (c + kTile - 1) / kTile;
  for (int tile = 0; tile < ntiles; ++tile) {
    const int c0 = tile * kTile;
    const int valid = std::min(kTile, c - c0);
    NA_CHECK(csc::launch_copy_tile(tb[0], R, CSC_F32, n, kTile, ldr, c0, valid, s));
    csc::StepArgs sa{};
    sa.n = n;
    sa.row_ptr = row_ptr;
    sa.col = col_idx;
    sa.val = vals;
    sa.scale = static_cast<const float*>(g.scale.ptr);
    sa.vs = static_cast<const float*>(g.vs.ptr);
    sa.ivs = static_cast<const float*>(g.ivs.ptr);
    sa.blk_row = static_cast<const int32_t*>(g.blk_row.ptr);
    sa.nblk = csc::edge_blocks(nnz);
    sa.srow = static_cast<const int32_t*>(g.srow.ptr);
    sa.nsblk = csc::row_blocks(n, nnz);
    sa.psi = psi;
    sa.ldp = kTile;
    sa.coef = coef;
    sa.w = kTile;
    sa.tg = tb[0];
    sa.tp = nullptr;
    sa.tn = tb[1];
    sa.j = 0;
    sa.part = part;
    NA_CHECK(csc::launch_cheb_first(sa, CSC_F32, grid, s));
    for (int j = 1; j < m; ++j) {
      sa.tg = tb[j % 3];
      sa.tp = tb[(j - 1) % 3];
      sa.tn = tb[(j + 1) % 3];
      sa.j = j;
      sa.part = part + (size_t)(2 * (j + 1) - 1) * grid;
      sa.tp_unscaled = j == 1;
      NA_CHECK(csc::launch_cheb_step(sa, CSC_F32, grid, s));
    }
    NA_CHECK(csc::launch_reduce_partials(part, rows, grid, 1, 0, ef, s));
    if (psi_out)
      NA_CHECK(csc::launch_convert(psi, CSC_F32, kTile, psi_out + c0, CSC_F32, ldp, n, valid, s));
    NA_CHECK(cudaMemcpyAsync(ef_tile, ef, (size_t)rows * 8, cudaMemcpyDeviceToHost, s));
    NA_CHECK(cudaStreamSynchronize(s));
    for (int r = 0; r < rows; ++r) ef_sum[r] += ef_tile[r];
  }
  if (mu_out) {
    mu_out[0] = ef_sum[0];
    mu_out[1] = ef_sum[2];
    for (int q = 1; q <= m; ++q) {
      mu_out[2 * q] = 2.0 * ef_sum[2 * q - 1] - mu_out[0];
      if (q >= 2) mu_out[2 * q - 1] = 2.0 * ef_sum[2 * q] - mu_out[1];
    }
  }
  return CSC_OK;
}
