// Random signal block R (Section 2.2, approximate features): i.i.d. centred Gaussians of variance 1/d.
//
// Counter-based so that every (row, global column) entry is addressable on its own:
// a reused column (Eq. 6) is never regenerated and a refiltered column sees the same
// signal.  Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) with counter
// (row lo, row hi, column, 0) and key (seed lo, seed hi); Box-Muller (1958) on
// u1 = (x0 >> 8 + 1) 2^-24 in (0, 1] and u2 = (x1 >> 8) 2^-24, both exact in float32.
#include "csc_internal.h"

namespace csc {

namespace {

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

__device__ __forceinline__ float gauss(uint64_t row, uint64_t gcol, uint32_t k0, uint32_t k1) {
  const U4 x = philox10(U4{(uint32_t)row, (uint32_t)(row >> 32), (uint32_t)gcol, 0u}, k0, k1);
  const float u1 = ((float)(x.x >> 8) + 1.0f) * 5.9604644775390625e-8f;  // 2^-24
  const float u2 = (float)(x.y >> 8) * 5.9604644775390625e-8f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <typename T>
__device__ __forceinline__ T cvt(float v);
template <>
__device__ __forceinline__ float cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__global__ void signals_kernel(T* __restrict__ out, int64_t n, int w, int64_t ld, uint32_t k0,
                               uint32_t k1, int64_t col0, int valid, float inv_sqrt_d) {
  const int64_t total = n * (int64_t)w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / w;
    const int v = (int)(e - row * w);
    float val = 0.0f;
    if (v < valid) val = gauss((uint64_t)row, (uint64_t)(col0 + v), k0, k1) * inv_sqrt_d;
    out[row * ld + v] = cvt<T>(val);
  }
}

template <typename T>
__global__ void copy_tile_kernel(T* __restrict__ dst, const T* __restrict__ src, int64_t n, int w,
                                 int64_t ld_src, int c0, int valid) {
  const int64_t total = n * (int64_t)w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / w;
    const int v = (int)(e - row * w);
    dst[e] = v < valid ? src[row * ld_src + c0 + v] : cvt<T>(0.0f);
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
                           int64_t col0, int valid, float inv_sqrt_d, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = elementwise_grid(n * (int64_t)w);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (dtype == CSC_BF16)
    signals_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((__nv_bfloat16*)out, n, w, ld, k0, k1, col0,
                                                       valid, inv_sqrt_d);
  else
    signals_kernel<float><<<grid, 256, 0, s>>>((float*)out, n, w, ld, k0, k1, col0, valid,
                                               inv_sqrt_d);
  return cudaGetLastError();
}

cudaError_t launch_copy_tile(void* dst, const void* src, int dtype, int64_t n, int w,
                             int64_t ld_src, int c0, int valid, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = elementwise_grid(n * (int64_t)w);
  if (dtype == CSC_BF16)
    copy_tile_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(
        (__nv_bfloat16*)dst, (const __nv_bfloat16*)src, n, w, ld_src, c0, valid);
  else
    copy_tile_kernel<float><<<grid, 256, 0, s>>>((float*)dst, (const float*)src, n, w, ld_src, c0,
                                                 valid);
  return cudaGetLastError();
}

}  // namespace csc
