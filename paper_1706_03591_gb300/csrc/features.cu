// Feature matrix Theta_t (Eq. 6) and its row normalisation.
//
// Theta_t is a ring of d column slots (n x d float32, row-major).  After a filtering
// pass the new columns of Psi~ replace the oldest slots (Eq. 6 with the dp kept
// columns); in the same pass every row is normalised, y_i = theta_i / ||theta_i||
// (a zero row stays zero), for the k-means step.  One warp per row; the row's d values
// stay in registers between the norm and the scaled write.
#include <type_traits>

#include "csc_internal.h"

namespace csc {

namespace {

constexpr int kMaxPerLane = 32;  // d <= 1024

template <typename T>
__device__ __forceinline__ void put(T* p, float v);
template <>
__device__ __forceinline__ void put<float>(float* p, float v) { *p = v; }
template <>
__device__ __forceinline__ void put<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}
__device__ __forceinline__ float get(const float* p) { return *p; }
__device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// PER: values per lane (d <= 32 PER), so a row lives in registers without dead slots.
template <typename TY, int PER>
__global__ void assemble_kernel(float* __restrict__ theta, int64_t ldt, const float* __restrict__ psi,
                                int64_t ldp, const int* __restrict__ src, int d, TY* __restrict__ y,
                                int64_t ldy, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < n; row += nwarps) {
    float v[PER];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int q = lane + 32 * i;
      v[i] = 0.f;
      if (q < d) {
        const int s = src != nullptr ? __ldg(src + q) : -1;
        if (s >= 0) {
          v[i] = psi[row * ldp + s];
          theta[row * ldt + q] = v[i];
        } else {
          v[i] = theta[row * ldt + q];
        }
        ss = fmaf(v[i], v[i], ss);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int q = lane + 32 * i;
      if (q < d) put<TY>(y + row * ldy + q, v[i] * inv);
    }
  }
}

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ src, int64_t ld_src, TD* __restrict__ dst,
                               int64_t ld_dst, int64_t n, int d, const int32_t* __restrict__ src_row) {
  const int64_t total = n * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / d;
    const int q = (int)(e - row * d);
    const int64_t r = src_row != nullptr ? (int64_t)src_row[row] : row;
    put<TD>(dst + row * ld_dst + q, get(src + r * ld_src + q));
  }
}

int grid_rows(int64_t n, int rows_per_block) {
  int64_t g = (n + rows_per_block - 1) / rows_per_block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_assemble(float* theta, int64_t ldt, const float* psi, int64_t ldp,
                            const int* src, int d, void* y, int y_dtype, int64_t ldy, int64_t n,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (d > 32 * kMaxPerLane) return cudaErrorInvalidValue;
  const int grid = grid_rows(n, 8);
  auto go = [&](auto per) {
    constexpr int P = decltype(per)::value;
    if (y_dtype == CSC_BF16)
      assemble_kernel<__nv_bfloat16, P><<<grid, 256, 0, s>>>(theta, ldt, psi, ldp, src, d, (__nv_bfloat16*)y,
                                                             ldy, n);
    else
      assemble_kernel<float, P><<<grid, 256, 0, s>>>(theta, ldt, psi, ldp, src, d, (float*)y, ldy, n);
  };
  if (d <= 32) go(std::integral_constant<int, 1>{});
  else if (d <= 64) go(std::integral_constant<int, 2>{});
  else if (d <= 128) go(std::integral_constant<int, 4>{});
  else if (d <= 256) go(std::integral_constant<int, 8>{});
  else if (d <= 512) go(std::integral_constant<int, 16>{});
  else go(std::integral_constant<int, 32>{});
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_dtype, int64_t ld_src, void* dst,
                           int dst_dtype, int64_t ld_dst, int64_t n, int d, cudaStream_t s,
                           const int32_t* src_row) {
  if (n == 0 || d == 0) return cudaSuccess;
  const int grid = grid_rows(n * (int64_t)d, 256);
  if (src_dtype == CSC_BF16) {
    if (dst_dtype == CSC_BF16)
      convert_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, 256, 0, s>>>(
          (const __nv_bfloat16*)src, ld_src, (__nv_bfloat16*)dst, ld_dst, n, d, src_row);
    else
      convert_kernel<__nv_bfloat16, float><<<grid, 256, 0, s>>>((const __nv_bfloat16*)src, ld_src,
                                                                (float*)dst, ld_dst, n, d, src_row);
  } else {
    if (dst_dtype == CSC_BF16)
      convert_kernel<float, __nv_bfloat16><<<grid, 256, 0, s>>>((const float*)src, ld_src,
                                                                (__nv_bfloat16*)dst, ld_dst, n, d, src_row);
    else
      convert_kernel<float, float><<<grid, 256, 0, s>>>((const float*)src, ld_src, (float*)dst,
                                                        ld_dst, n, d, src_row);
  }
  return cudaGetLastError();
}

}  // namespace csc
