// Compressive k-means (Section 2.2, step 2; cost in Section 4.2): the device kernels of the
// sampling, the reduced feature block, the interpolation right-hand side and the final
// assignment.  The host side is csc_compressive_cluster in api.cu; the reduced k-means and the
// interpolation filter reuse the Lloyd and Chebyshev kernels.
//
// Sampling is exact integer work, so the sampled set does not depend on thread order:
//   s_i  = float64 sum over l = 0..d-1, in order, of theta_il^2 (each square is exact);
//   q_i  = floor(s_i 2^E), E = 62 - ceil(log2 n) - e with 2^(e-1) <= max s < 2^e, so every
//          prefix sum P_i = q_0 + ... + q_i is an exact int64 below 2^62;
//   draw t: Philox-4x32-10 counter (t, 0, 0, 2), key = seed; U = x0 2^32 + x1,
//          u = floor(U T / 2^64) with T = P_(n-1); the drawn node is the smallest i with P_i > u;
//   Omega: the distinct drawn nodes in increasing order (flags, then an inclusive scan).
// The interpolation right-hand side puts w_i = T / (n q_i) (the inverse sampling density,
// weight 1 under uniform sampling) at (i, a_i) for every sampled node i with reduced label a_i.
#include <algorithm>

#include "csc_internal.h"
#include "philox.cuh"

namespace csc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // elements per block of the first scan level

// Float64 sum of squares of each row in column order, and the running maximum
// (non-negative doubles order like their bit patterns).  A block owns 256 rows and walks
// the columns in chunks of 32: the chunk is staged in shared memory with coalesced 16-byte
// loads (a padded row stride keeps the column reads conflict-free), then each thread adds
// its row's 32 squares in order, so the sum is the same as a plain left-to-right loop.
constexpr int kEnergyRows = 256;
constexpr int kEnergyCols = 32;

__global__ void __launch_bounds__(kEnergyRows) row_energy_kernel(const float* __restrict__ theta, int64_t ld,
                                                                 int64_t n, int d, double* __restrict__ s,
                                                                 unsigned long long* __restrict__ smax_bits) {
  __shared__ float tile[kEnergyRows][kEnergyCols + 1];
  const bool vec = (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(theta) % 16) == 0;
  double mx = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * kEnergyRows; r0 < n; r0 += (int64_t)gridDim.x * kEnergyRows) {
    double acc = 0.0;
    for (int c0 = 0; c0 < d; c0 += kEnergyCols) {
      // 256 rows x 32 columns: thread t loads column group t % 8 of rows t / 8 + 32 i
      const int cg = threadIdx.x & 7;
      for (int i = 0; i < kEnergyRows / 32; ++i) {
        const int rl = (threadIdx.x >> 3) + 32 * i;
        const int64_t row = r0 + rl;
        const int col = c0 + cg * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
          const float* src = theta + row * ld + col;
          if (vec && col + 4 <= d) {
            v = *reinterpret_cast<const float4*>(src);
          } else {
            if (col < d) v.x = src[0];
            if (col + 1 < d) v.y = src[1];
            if (col + 2 < d) v.z = src[2];
            if (col + 3 < d) v.w = src[3];
          }
        }
        tile[rl][cg * 4] = v.x;
        tile[rl][cg * 4 + 1] = v.y;
        tile[rl][cg * 4 + 2] = v.z;
        tile[rl][cg * 4 + 3] = v.w;
      }
      __syncthreads();
      const int cols = min(kEnergyCols, d - c0);
      for (int l = 0; l < cols; ++l) {
        const double v = (double)tile[threadIdx.x][l];
        acc = fma(v, v, acc);  // v * v is exact, so this is the rounded sum acc + v^2
      }
      __syncthreads();
    }
    const int64_t row = r0 + threadIdx.x;
    if (row < n) {
      s[row] = acc;
      mx = fmax(mx, acc);
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(smax_bits, (unsigned long long)__double_as_longlong(mx));
}

__global__ void quantise_kernel(const double* __restrict__ s, int64_t n, int lg_n,
                                const unsigned long long* __restrict__ smax_bits, long long* __restrict__ q) {
  int e = 0;
  frexp(__longlong_as_double((long long)*smax_bits), &e);
  const int big_e = 62 - lg_n - e;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = (long long)floor(ldexp(s[i], big_e));
}

// Inclusive block-wide scan of one value per thread (kScanThreads threads).
template <typename T>
__device__ T block_inclusive_scan(T v, T* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    T t = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T o = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += o;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  if (warp > 0) v += warp_tot[warp - 1];
  __syncthreads();
  return v;
}

// Level 1: inclusive scan inside each chunk of kScanChunk elements; chunk totals to sums.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                   int64_t n, T* __restrict__ sums) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int64_t base = blockIdx.x * (int64_t)kScanChunk + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    run += base + i < n ? in[base + i] : T(0);
    v[i] = run;
  }
  const T incl = block_inclusive_scan<T>(run, warp_tot);
  const T excl = incl - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] = v[i] + excl;
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = incl;
}

// Level 2: inclusive scan of the chunk totals by one block, carrying a running offset.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(T* __restrict__ sums, int64_t nb) {
  __shared__ T warp_tot[kScanThreads / 32];
  T carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    const T v = b < nb ? sums[b] : T(0);
    const T incl = block_inclusive_scan<T>(v, warp_tot);
    if (b < nb) sums[b] = incl + carry;
    __shared__ T last;
    if (threadIdx.x == kScanThreads - 1) last = incl;
    __syncthreads();
    carry += last;
    __syncthreads();
  }
}

// Level 3: add the total of the preceding chunks.
template <typename T>
__global__ void scan_add_kernel(T* __restrict__ out, int64_t n, const T* __restrict__ sums) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / kScanChunk;
    if (b > 0) out[i] += sums[b - 1];
  }
}

template <typename T>
cudaError_t inclusive_scan(const T* in, T* out, int64_t n, T* sums, cudaStream_t s) {
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  scan_chunks_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  scan_sums_kernel<T><<<1, kScanThreads, 0, s>>>(sums, nb);
  if (nb > 1) scan_add_kernel<T><<<num_sms() * 8, 256, 0, s>>>(out, n, sums);
  return cudaGetLastError();
}

__global__ void draw_kernel(uint64_t seed, int64_t n_draws, const long long* __restrict__ prefix, int64_t n,
                            int* __restrict__ flags) {
  const unsigned long long total = (unsigned long long)prefix[n - 1];
  if (total == 0) return;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_draws;
       t += (int64_t)gridDim.x * blockDim.x) {
    const PhiloxU4 x = philox10(PhiloxU4{(uint32_t)t, 0u, 0u, 2u}, k0, k1);
    const unsigned long long big_u = ((unsigned long long)x.x << 32) | x.y;
    const unsigned long long u = __umul64hi(big_u, total);  // < total
    // smallest i with prefix[i] > u
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if ((unsigned long long)prefix[mid] > u) hi = mid; else lo = mid + 1;
    }
    flags[lo] = 1;
  }
}

__global__ void compact_kernel(const int* __restrict__ flags, const int* __restrict__ pos, int64_t n,
                               int32_t* __restrict__ omega) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) omega[pos[i] - 1] = (int32_t)i;
}

// Rows y[omega[r]] -> out[r] (n_omega x d, leading dimension d), one warp per row.
template <typename TY>
__global__ void gather_rows_kernel(const TY* __restrict__ y, int64_t ldy, const int32_t* __restrict__ omega,
                                   int64_t no, int d, TY* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < no;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const TY* src = y + (int64_t)omega[r] * ldy;
    for (int l = lane; l < d; l += 32) out[r * d + l] = src[l];
  }
}

// z[omega[r]][labels[r]] = (float)(T / (n q_omega[r])) in float64 with one rounding per operation.
__global__ void build_rhs_kernel(const int32_t* __restrict__ omega, const int32_t* __restrict__ labels, int64_t no,
                                 const long long* __restrict__ q, const long long* __restrict__ prefix, int64_t n,
                                 float* __restrict__ z, int64_t ldz) {
  const double total = (double)prefix[n - 1];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < no; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = omega[r];
    const double w = __ddiv_rn(total, __dmul_rn((double)n, (double)q[i]));
    z[i * ldz + labels[r]] = (float)w;
  }
}

// Lowest column index of each row maximum, one warp per row (coalesced row reads, then a
// shuffle reduction that prefers the larger value and, among equal values, the lower index).
__global__ void argmax_kernel(const float* __restrict__ x, int64_t ldx, int64_t n, int k, int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float* r = x + i * ldx;
    float best = -INFINITY;
    int bi = k;
    for (int j = lane; j < k; j += 32) {
      const float v = r[j];
      if (v > best || bi == k) { best = v; bi = j; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (oi < k && (bi == k || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
    }
    if (lane == 0) out[i] = bi;
  }
}

}  // namespace

int64_t scan_sums_len(int64_t n) { return (n + kScanChunk - 1) / kScanChunk + 1; }

cudaError_t inclusive_scan_i64(const long long* in, long long* out, int64_t n, long long* sums, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return inclusive_scan<long long>(in, out, n, sums, s);
}

cudaError_t compressive_sample(CompressiveState& cs, const float* theta, int64_t ld, int64_t n, int d,
                               int64_t n_draws, uint64_t seed, cudaStream_t s) {
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (!ensure(cs.s, (size_t)n * 8) || !ensure(cs.q, (size_t)n * 8) || !ensure(cs.prefix, (size_t)n * 8) ||
      !ensure(cs.flags, (size_t)n * 4) || !ensure(cs.pos, (size_t)n * 4) || !ensure(cs.sums, (size_t)nb * 8 + 8) ||
      !ensure(cs.omega, (size_t)std::min<int64_t>(n, n_draws) * 4) || !ensure(cs.smax, 8))
    return cudaErrorMemoryAllocation;
  const int grid = num_sms() * 8;
  cudaError_t e = cudaMemsetAsync(cs.smax.ptr, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cs.flags.ptr, 0, (size_t)n * 4, s);
  if (e != cudaSuccess) return e;
  row_energy_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms() * 4, (n + kEnergyRows - 1) / kEnergyRows)),
                      kEnergyRows, 0, s>>>(theta, ld, n, d, as<double>(cs.s), as<unsigned long long>(cs.smax));
  int lg_n = 0;
  while ((int64_t(1) << lg_n) < std::max<int64_t>(n, 2)) ++lg_n;
  quantise_kernel<<<grid, 256, 0, s>>>(as<double>(cs.s), n, lg_n, as<unsigned long long>(cs.smax),
                                       as<long long>(cs.q));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = inclusive_scan<long long>(as<long long>(cs.q), as<long long>(cs.prefix), n, as<long long>(cs.sums), s)) !=
      cudaSuccess)
    return e;
  draw_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(grid, (n_draws + 255) / 256)), 256, 0, s>>>(
      seed, n_draws, as<long long>(cs.prefix), n, as<int>(cs.flags));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = inclusive_scan<int>(as<int>(cs.flags), as<int>(cs.pos), n, as<int>(cs.sums), s)) != cudaSuccess)
    return e;
  compact_kernel<<<grid, 256, 0, s>>>(as<int>(cs.flags), as<int>(cs.pos), n, as<int32_t>(cs.omega));
  return cudaGetLastError();
}

cudaError_t compressive_gather(const void* y, int y_dtype, int64_t ldy, const int32_t* omega, int64_t no, int d,
                               void* out, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms() * 8, (no + 7) / 8));
  if (y_dtype == CSC_BF16)
    gather_rows_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(y), ldy, omega, no, d,
                                                          static_cast<__nv_bfloat16*>(out));
  else
    gather_rows_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(y), ldy, omega, no, d,
                                                  static_cast<float*>(out));
  return cudaGetLastError();
}

cudaError_t compressive_rhs(const CompressiveState& cs, const int32_t* labels, int64_t no, int64_t n, float* z,
                            int64_t ldz, cudaStream_t s) {
  build_rhs_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms() * 4, (no + 255) / 256)), 256, 0,
                     s>>>(static_cast<const int32_t*>(cs.omega.ptr), labels, no,
                          static_cast<const long long*>(cs.q.ptr), static_cast<const long long*>(cs.prefix.ptr), n,
                          z, ldz);
  return cudaGetLastError();
}

cudaError_t compressive_argmax(const float* x, int64_t ldx, int64_t n, int k, int32_t* out, cudaStream_t s) {
  argmax_kernel<<<num_sms() * 8, 256, 0, s>>>(x, ldx, n, k, out);
  return cudaGetLastError();
}

void compressive_release(CompressiveState& cs) {
  DevBuf* all[] = {&cs.s, &cs.q, &cs.prefix, &cs.flags, &cs.pos, &cs.sums, &cs.omega, &cs.smax,
                   &cs.yo, &cs.labels, &cs.z, &cs.x, &cs.assign, &cs.theta_stage, &cs.y_stage};
  for (DevBuf* b : all) release(*b);
}

}  // namespace csc
