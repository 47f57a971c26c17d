// Counter-based Gaussian signals on the device (Section 2.2, approximate features).
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) with counter (row lo, row hi, column,
// 0) and key (seed lo, seed hi); Box-Muller (1958) on u1 = (x0 >> 8 + 1) 2^-24 in (0, 1] and
// u2 = (x1 >> 8) 2^-24, both exact in float32.  Shared by the signal and batched kernels.
#pragma once

#include <stdint.h>

namespace csc {

struct PhiloxU4 { uint32_t x, y, z, w; };

__device__ __forceinline__ PhiloxU4 philox10(PhiloxU4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = PhiloxU4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Standard normal draw for (row, global column) under key (k0, k1).
__device__ __forceinline__ float gauss_signal(uint64_t row, uint64_t gcol, uint32_t k0, uint32_t k1) {
  const PhiloxU4 x = philox10(PhiloxU4{(uint32_t)row, (uint32_t)(row >> 32), (uint32_t)gcol, 0u}, k0, k1);
  const float u1 = ((float)(x.x >> 8) + 1.0f) * 5.9604644775390625e-8f;  // 2^-24
  const float u2 = (float)(x.y >> 8) * 5.9604644775390625e-8f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

}  // namespace csc
