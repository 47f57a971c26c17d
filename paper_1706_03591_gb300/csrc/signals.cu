// Random signal block R (Section 2.2, approximate features): i.i.d. centred Gaussians of variance 1/d.
//
// Counter-based so that every (row, global column) entry is addressable on its own:
// a reused column (Eq. 6) is never regenerated and a refiltered column sees the same
// signal (generator in philox.cuh).
#include "csc_internal.h"
#include "philox.cuh"

namespace csc {

namespace {

template <typename T>
__device__ __forceinline__ T cvt(float v);
template <>
__device__ __forceinline__ float cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__global__ void signals_kernel(T* __restrict__ out, int64_t n, int w, int64_t ld, uint32_t k0,
                               uint32_t k1, int64_t col0, int valid, float inv_sqrt_d,
                               const int32_t* __restrict__ rowid) {
  const int64_t total = n * (int64_t)w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / w;
    const int v = (int)(e - row * w);
    float val = 0.0f;
    const uint64_t key = rowid != nullptr ? (uint64_t)rowid[row] : (uint64_t)row;
    if (v < valid) val = gauss_signal(key, (uint64_t)(col0 + v), k0, k1) * inv_sqrt_d;
    out[row * ld + v] = cvt<T>(val);
  }
}

template <typename T>
__global__ void copy_tile_kernel(T* __restrict__ dst, const T* __restrict__ src, int64_t n, int w,
                                 int64_t ld_src, int c0, int valid, const int32_t* __restrict__ src_row) {
  const int64_t total = n * (int64_t)w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / w;
    const int v = (int)(e - row * w);
    const int64_t r = src_row != nullptr ? (int64_t)src_row[row] : row;
    dst[e] = v < valid ? src[r * ld_src + c0 + v] : cvt<T>(0.0f);
  }
}

int elementwise_grid(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_signals(void* out, int dtype, int64_t n, int w, int64_t ld, uint64_t seed,
                           int64_t col0, int valid, float inv_sqrt_d, cudaStream_t s, const int32_t* rowid) {
  if (n == 0) return cudaSuccess;
  const int grid = elementwise_grid(n * (int64_t)w);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (dtype == CSC_BF16)
    signals_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((__nv_bfloat16*)out, n, w, ld, k0, k1, col0,
                                                       valid, inv_sqrt_d, rowid);
  else
    signals_kernel<float><<<grid, 256, 0, s>>>((float*)out, n, w, ld, k0, k1, col0, valid,
                                               inv_sqrt_d, rowid);
  return cudaGetLastError();
}

cudaError_t launch_copy_tile(void* dst, const void* src, int dtype, int64_t n, int w,
                             int64_t ld_src, int c0, int valid, cudaStream_t s, const int32_t* src_row) {
  if (n == 0) return cudaSuccess;
  const int grid = elementwise_grid(n * (int64_t)w);
  if (dtype == CSC_BF16)
    copy_tile_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(
        (__nv_bfloat16*)dst, (const __nv_bfloat16*)src, n, w, ld_src, c0, valid, src_row);
  else
    copy_tile_kernel<float><<<grid, 256, 0, s>>>((float*)dst, (const float*)src, n, w, ld_src, c0,
                                                 valid, src_row);
  return cudaGetLastError();
}

}  // namespace csc
