// Edge similarity of two snapshots (Definition 4.1): rho = ||L_b - L_a||_F for the
// normalized Laplacians L = I - D^-1/2 W D^-1/2 of two graphs on the same node set.  The
// identity cancels, so rho^2 sums (l_b(u,v) - l_a(u,v))^2 over the union of the two edge
// sets, l(u,v) = -w_uv / sqrt(d_u d_v) and 0 for an absent edge.  Every stored entry of a
// finds its partner in b by binary search in b's row (and vice versa for the entries of b
// absent from a); the sums are float64 block partials reduced in a fixed order.
#include <algorithm>
#include <cmath>

#include "csc_internal.h"

namespace csc {
namespace {

constexpr int kSimBlock = 256;

// inv_sqrt_deg[u] = 1 / sqrt(sum_v w_uv), 0 for an isolated node: one warp per row.
__global__ void inv_sqrt_degree_kernel(int64_t n, const int64_t* __restrict__ rp, const float* __restrict__ val,
                                       double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nw) {
    double d = 0.0;
    for (int64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) d += val != nullptr ? (double)val[e] : 1.0;
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) out[u] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
}

__device__ __forceinline__ int64_t find_col(const int32_t* col, int64_t lo, int64_t hi, int32_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Sum over the entries of x of (l_x - l_y)^2 (mode 0) or, for entries absent from y only, l_x^2
// (mode 1); one warp per row, block partials into part[blockIdx.x].
__global__ void laplacian_diff_kernel(int64_t n, const int64_t* __restrict__ rpx, const int32_t* __restrict__ cx,
                                      const float* __restrict__ vx, const double* __restrict__ sx,
                                      const int64_t* __restrict__ rpy, const int32_t* __restrict__ cy,
                                      const float* __restrict__ vy, const double* __restrict__ sy, int mode,
                                      double* __restrict__ part) {
  __shared__ double red[kSimBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t u = warp; u < n; u += nw) {
    const int64_t ylo = rpy[u], yhi = rpy[u + 1];
    for (int64_t e = rpx[u] + lane; e < rpx[u + 1]; e += 32) {
      const int32_t v = cx[e];
      // explicit roundings: no fused multiply-add may mix a rounded and an unrounded entry
      const double lx = -__dmul_rn(__dmul_rn(vx != nullptr ? (double)vx[e] : 1.0, sx[u]), sx[v]);
      const int64_t p = find_col(cy, ylo, yhi, v);
      const bool in_y = p < yhi && cy[p] == v;
      if (mode == 0) {
        const double ly = in_y ? -__dmul_rn(__dmul_rn(vy != nullptr ? (double)vy[p] : 1.0, sy[u]), sy[v]) : 0.0;
        acc += (lx - ly) * (lx - ly);
      } else if (!in_y) {
        acc += lx * lx;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kSimBlock / 32; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_kernel(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double red[kSimBlock / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kSimBlock / 32; ++i) t += red[i];
    *out = t;
  }
}

}  // namespace
}  // namespace csc

extern "C" csc_status csc_laplacian_distance(csc_ctx* ctx, int64_t n, const int64_t* rp_a, const int32_t* col_a,
                                             const float* val_a, const int64_t* rp_b, const int32_t* col_b,
                                             const float* val_b, double* rho_out) {
  if (!ctx) return CSC_EINVAL;
  if (n < 1 || !rp_a || !rp_b || !rho_out) {
    ctx->err = "csc_laplacian_distance: bad arguments";
    return CSC_EINVAL;
  }
  cudaStream_t s = ctx->stream;
  const int grid = csc::num_sms() * 8;
  if (!csc::ensure(ctx->sim, ((size_t)2 * n + 2 * grid + 8) * 8)) {
    ctx->err = "csc_laplacian_distance: device allocation failed";
    return CSC_ENOMEM;
  }
  double* sa = csc::as<double>(ctx->sim);
  double* sb = sa + n;
  double* part = sb + n;
  double* out = part + 2 * grid;
  auto check = [&](cudaError_t e) {
    if (e != cudaSuccess) ctx->err = std::string("csc_laplacian_distance: ") + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  csc::inv_sqrt_degree_kernel<<<grid, csc::kSimBlock, 0, s>>>(n, rp_a, val_a, sa);
  csc::inv_sqrt_degree_kernel<<<grid, csc::kSimBlock, 0, s>>>(n, rp_b, val_b, sb);
  csc::laplacian_diff_kernel<<<grid, csc::kSimBlock, 0, s>>>(n, rp_a, col_a, val_a, sa, rp_b, col_b, val_b, sb, 0, part);
  csc::laplacian_diff_kernel<<<grid, csc::kSimBlock, 0, s>>>(n, rp_b, col_b, val_b, sb, rp_a, col_a, val_a, sa, 1,
                                                             part + grid);
  csc::sum_kernel<<<1, csc::kSimBlock, 0, s>>>(part, 2 * grid, out);
  if (!check(cudaGetLastError())) return CSC_ECUDA;
  ctx->launches += 5;
  double r2 = 0.0;
  if (!check(cudaMemcpyAsync(&r2, out, 8, cudaMemcpyDeviceToHost, s)) || !check(cudaStreamSynchronize(s)))
    return CSC_ECUDA;
  *rho_out = std::sqrt(r2);
  return CSC_OK;
}
