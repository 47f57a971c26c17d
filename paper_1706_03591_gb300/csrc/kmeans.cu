// k-means (Lloyd) on the feature rows (Section 2.1, Eq. 1-2; Algorithm 1 step 8).
//
// Assignment: a register-tiled float32 pass computes f_j = |c_j|^2 - 2 <y, c_j> for every
// centroid and keeps, per row, the best and second-best value.  |f_j - e_j| (e_j the exact
// value with the float64 centroids) is bounded by
//     B = u (3.1 cmax^2 + 2 (1.01 d + 1) |y| cmax),   u = 2^-24,
// (recursive float32 summation of d products plus the rounding of the centroids and their
// norms).  A row whose top-2 gap is at most 4B is re-decided in float64 on all centroids
// (sum_l (y_l - c_jl)^2, lowest index on ties), so every assignment equals the float64
// argmin, as in the reference definition.
//
// Update: centroid sums are accumulated exactly in 64-bit fixed point (y * 2^S rounded to
// an integer, S chosen so that n max|y| 2^S < 2^62), privatised per block in shared memory
// when k*d fits, then converted to float64 means.  Integer addition is associative, so the
// result does not depend on scheduling; an empty cluster keeps its centroid.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "csc_internal.h"

namespace csc {

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int kAssignBlock = 256;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename TY>
__global__ void maxabs_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                              unsigned int* out) {
  float m = 0.f;
  const int64_t total = n * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / d;
    const int l = (int)(e - row * d);
    m = fmaxf(m, fabsf(ldf(y + row * ldy + l)));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <typename TY>
__global__ void forgy_kernel(const TY* __restrict__ y, int64_t ldy, const int64_t* __restrict__ idx,
                             int k, int d, double* __restrict__ c64) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * d; e += gridDim.x * blockDim.x) {
    const int j = e / d, l = e - (e / d) * d;
    c64[e] = (double)ldf(y + idx[j] * ldy + l);
  }
}

// Fixed-point centroid sums.  SMEM: per-block privatisation in dynamic shared memory.
template <typename TY, bool SMEM>
__global__ void update_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                              const int32_t* __restrict__ assign, int k, float scale,
                              unsigned long long* __restrict__ sums, int* __restrict__ counts) {
  extern __shared__ unsigned long long sh[];
  unsigned long long* tsum = sums;
  int* tcnt = counts;
  if (SMEM) {
    tsum = sh;
    tcnt = reinterpret_cast<int*>(sh + (size_t)k * d);
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) tsum[e] = 0ull;
    for (int e = threadIdx.x; e < k; e += blockDim.x) tcnt[e] = 0;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int a = assign[row];
    for (int l = lane; l < d; l += 32) {
      const long long q = __float2ll_rn(ldf(y + row * ldy + l) * scale);
      atomicAdd(tsum + (size_t)a * d + l, (unsigned long long)q);
    }
    if (lane == 0) atomicAdd(tcnt + a, 1);
  }
  if (SMEM) {
    __syncthreads();
    for (int e = threadIdx.x; e < k * d; e += blockDim.x)
      if (tsum[e] != 0ull) atomicAdd(sums + e, tsum[e]);
    for (int e = threadIdx.x; e < k; e += blockDim.x)
      if (tcnt[e] != 0) atomicAdd(counts + e, tcnt[e]);
  }
}

// Means from the fixed-point sums (empty clusters keep c64), float32 copies, |c32|^2, max |c|.
__global__ void finalize_kernel(const unsigned long long* __restrict__ sums,
                                const int* __restrict__ counts, int k, int d, double inv_scale,
                                double* __restrict__ c64, float* __restrict__ c32,
                                float* __restrict__ cn2, unsigned int* __restrict__ cmax_bits) {
  for (int e = threadIdx.x; e < k * d; e += blockDim.x) {
    const int j = e / d;
    const int cnt = counts[j];
    if (cnt > 0) c64[e] = (double)(long long)sums[e] * inv_scale / (double)cnt;
    c32[e] = (float)c64[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double s = 0.0;
    for (int l = lane; l < d; l += 32) {
      const double v = (double)c32[(size_t)j * d + l];
      s += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      cn2[j] = (float)s;
      atomicMax(cmax_bits, __float_as_uint((float)sqrt(s) * 1.0000002f));
    }
  }
}

struct AssignArgs {
  const void* y;
  int64_t ldy, n;
  int d, k;
  const float* c32;   // [k][d]
  const float* cn2;   // [k]
  const unsigned int* cmax_bits;
  const int32_t* old_assign;  // nullptr on the first pass
  int32_t* new_assign;
  int32_t* flagged;
  unsigned long long* counters;  // [0] changed rows, [1] flagged rows
};

__device__ __forceinline__ void merge_best(float& b, int& bi, float& s, float b2, int bi2, float s2) {
  if (b2 < b || (b2 == b && bi2 < bi)) {
    s = fminf(s2, b);
    b = b2;
    bi = bi2;
  } else {
    s = fminf(s, b2);
  }
}

template <typename TY>
__global__ void __launch_bounds__(kAssignBlock) assign_kernel(AssignArgs a) {
  __shared__ __align__(16) float Ys[BK][BM + 4];
  __shared__ __align__(16) float Cs[BK][BN + 4];
  __shared__ unsigned long long block_changed;
  const TY* __restrict__ y = static_cast<const TY*>(a.y);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float cmax = __uint_as_float(*a.cmax_bits);
  const float u = 5.9604644775390625e-8f;
  const int64_t ntiles = (a.n + BM - 1) / BM;
  if (tid == 0) block_changed = 0;
  __syncthreads();
  unsigned long long changed = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * BM;
    float best[4], second[4], yn2[4];
    int bidx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { best[i] = INFINITY; second[i] = INFINITY; bidx[i] = 0; yn2[i] = 0.f; }
    for (int n0 = 0; n0 < a.k; n0 += BN) {
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      for (int k0 = 0; k0 < a.d; k0 += BK) {
        for (int e = tid; e < BM * BK; e += kAssignBlock) {
          const int r = e / BK, kk = e % BK;
          const int64_t row = row0 + r;
          const int col = k0 + kk;
          Ys[kk][r] = (row < a.n && col < a.d) ? ldf(y + row * a.ldy + col) : 0.f;
        }
        for (int e = tid; e < BN * BK; e += kAssignBlock) {
          const int jj = e / BK, kk = e % BK;
          const int cj = n0 + jj, col = k0 + kk;
          Cs[kk][jj] = (cj < a.k && col < a.d) ? a.c32[(size_t)cj * a.d + col] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
          const float4 av = *reinterpret_cast<const float4*>(&Ys[kk][ty * 4]);
          const float4 bv = *reinterpret_cast<const float4*>(&Cs[kk][tx * 4]);
          const float ar[4] = {av.x, av.y, av.z, av.w};
          const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
            if (n0 == 0) yn2[i] = fmaf(ar[i], ar[i], yn2[i]);
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cj = n0 + tx * 4 + j;
        if (cj < a.k) {
          const float c2 = __ldg(a.cn2 + cj);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float f = fmaf(-2.0f, acc[i][j], c2);
            if (f < best[i]) { second[i] = best[i]; best[i] = f; bidx[i] = cj; }
            else if (f < second[i]) second[i] = f;
          }
        }
      }
    }
    // combine the 16 column-threads of each row (lanes differing in tx within the warp)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int off = 1; off < 16; off <<= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best[i], off);
        const int i2 = __shfl_xor_sync(0xffffffffu, bidx[i], off);
        const float s2 = __shfl_xor_sync(0xffffffffu, second[i], off);
        merge_best(best[i], bidx[i], second[i], b2, i2, s2);
      }
    }
    if (tx == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t row = row0 + ty * 4 + i;
        if (row >= a.n) continue;
        const float bound = u * (3.1f * cmax * cmax + 2.0f * (1.01f * a.d + 1.0f) * sqrtf(yn2[i]) * cmax);
        const bool tie = !(second[i] - best[i] > 4.0f * bound);
        if (tie) {
          const unsigned long long slot = atomicAdd(a.counters + 1, 1ull);
          a.flagged[slot] = (int32_t)row;
        } else {
          a.new_assign[row] = bidx[i];
          if (a.old_assign != nullptr && a.old_assign[row] != bidx[i]) ++changed;
        }
      }
    }
  }
  if (changed) atomicAdd(&block_changed, changed);
  __syncthreads();
  if (tid == 0 && block_changed) atomicAdd(a.counters, block_changed);
}

// Float64 decision for the flagged rows: one warp per row, all centroids, lowest index on ties.
template <typename TY>
__global__ void recheck_kernel(const TY* __restrict__ y, int64_t ldy, int d, int k,
                               const double* __restrict__ c64, const int32_t* __restrict__ flagged,
                               const unsigned long long* __restrict__ counters,
                               const int32_t* __restrict__ old_assign, int32_t* __restrict__ new_assign,
                               unsigned long long* changed) {
  const unsigned long long nflag = counters[1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < (int64_t)nflag; w += nwarps) {
    const int64_t row = flagged[w];
    double best = INFINITY;
    int bi = 0;
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int l = lane; l < d; l += 32) {
        const double diff = (double)ldf(y + row * ldy + l) - c64[(size_t)j * d + l];
        s = fma(diff, diff, s);
      }
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (s < best) { best = s; bi = j; }
    }
    if (lane == 0) {
      new_assign[row] = bi;
      if (old_assign != nullptr && old_assign[row] != bi) atomicAdd(changed, 1ull);
    }
  }
}

template <typename TY>
__global__ void inertia_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                               const float* __restrict__ c32, const int32_t* __restrict__ assign,
                               double* __restrict__ part) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int a = assign[row];
    float s = 0.f;
    for (int l = lane; l < d; l += 32) {
      const float diff = ldf(y + row * ldy + l) - c32[(size_t)a * d + l];
      s = fmaf(diff, diff, s);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) acc += (double)s;
  }
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    part[blockIdx.x] = s;
  }
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      if (err) *err = std::string(#call ": ") + cudaGetErrorString(e_); \
      return CSC_ECUDA;                                   \
    }                                                     \
  } while (0)

template <typename TY>
csc_status run_typed(KmeansState& st, const TY* y, int64_t n, int d, int64_t ldy, int k,
                     const int64_t* init_idx, const int32_t* prev_assign, int max_iter,
                     cudaStream_t s, KmeansResult* res, std::string* err) {
  const size_t kd = (size_t)k * d;
  if (!ensure(st.c64, kd * 8) || !ensure(st.c32, kd * 4) || !ensure(st.cn2, (size_t)k * 4) ||
      !ensure(st.cmax, 16) || !ensure(st.sums, kd * 8) || !ensure(st.counts, (size_t)k * 4) ||
      !ensure(st.assign_a, (size_t)n * 4) || !ensure(st.assign_b, (size_t)n * 4) ||
      !ensure(st.flagged, (size_t)n * 4) || !ensure(st.counters, 64) || !ensure(st.maxabs, 16) ||
      !ensure(st.init_idx, (size_t)k * 8) || !ensure(st.inertia_part, (size_t)num_sms() * 8 * 8)) {
    if (err) *err = "k-means: device allocation failed";
    return CSC_ENOMEM;
  }
  const int sms = num_sms();
  int64_t launches = 0;
  // fixed-point scale from max |y|
  CK(cudaMemsetAsync(st.maxabs.ptr, 0, 4, s));
  maxabs_kernel<TY><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, as<unsigned int>(st.maxabs));
  CK(cudaGetLastError());
  ++launches;
  unsigned int mbits = 0;
  CK(cudaMemcpyAsync(&mbits, st.maxabs.ptr, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float maxabs;
  std::memcpy(&maxabs, &mbits, 4);
  if (!(maxabs < 1e30f)) {
    if (err) *err = "k-means: features contain inf/nan or are too large";
    return CSC_EINVAL;
  }
  const int lg_n = (int)std::ceil(std::log2((double)std::max<int64_t>(n, 2)));
  const int lg_m = maxabs > 0.f ? (int)std::ceil(std::log2((double)maxabs)) : 0;
  const int S = 61 - lg_n - lg_m;
  const float scale = std::ldexp(1.0f, S);
  const double inv_scale = std::ldexp(1.0, -S);

  // initial centroids
  CK(cudaMemcpyAsync(st.init_idx.ptr, init_idx, (size_t)k * 8, cudaMemcpyHostToDevice, s));
  forgy_kernel<TY><<<std::max(1, (int)std::min<size_t>((kd + 255) / 256, 1024)), 256, 0, s>>>(
      y, ldy, as<int64_t>(st.init_idx), k, d, as<double>(st.c64));
  CK(cudaGetLastError());
  ++launches;
  const size_t smem = kd * 8 + (size_t)k * 4;
  const bool use_smem = smem <= 220 * 1024;
  auto accumulate = [&](const int32_t* asg) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(st.sums.ptr, 0, kd * 8, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.counts.ptr, 0, (size_t)k * 4, s);
    if (e != cudaSuccess) return e;
    if (asg == nullptr) return cudaSuccess;
    ++launches;
    if (use_smem) {
      auto fn = update_kernel<TY, true>;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      fn<<<sms, 1024, smem, s>>>(y, ldy, n, d, asg, k, scale, as<unsigned long long>(st.sums),
                                 as<int>(st.counts));
    } else {
      update_kernel<TY, false><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, asg, k, scale,
                                                       as<unsigned long long>(st.sums),
                                                       as<int>(st.counts));
    }
    return cudaGetLastError();
  };
  auto finalize = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(st.cmax.ptr, 0, 4, s);
    if (e != cudaSuccess) return e;
    ++launches;
    finalize_kernel<<<1, 1024, 0, s>>>(as<unsigned long long>(st.sums), as<int>(st.counts), k, d,
                                       inv_scale, as<double>(st.c64), as<float>(st.c32),
                                       as<float>(st.cn2), as<unsigned int>(st.cmax));
    return cudaGetLastError();
  };
  CK(accumulate(prev_assign));
  CK(finalize());

  int32_t* cur = as<int32_t>(st.assign_a);
  int32_t* other = as<int32_t>(st.assign_b);
  const int32_t* old = nullptr;
  int assign_grid = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&assign_grid, assign_kernel<TY>, kAssignBlock, 0);
  assign_grid = std::max(1, assign_grid) * sms;
  const int64_t ntiles = (n + BM - 1) / BM;
  if ((int64_t)assign_grid > ntiles) assign_grid = (int)std::max<int64_t>(1, ntiles);
  int it = 0;
  bool converged = false;
  for (it = 1; it <= max_iter; ++it) {
    CK(cudaMemsetAsync(st.counters.ptr, 0, 16, s));
    AssignArgs aa{y, ldy, n, d, k, as<float>(st.c32), as<float>(st.cn2), as<unsigned int>(st.cmax),
                  old, cur, as<int32_t>(st.flagged), as<unsigned long long>(st.counters)};
    assign_kernel<TY><<<assign_grid, kAssignBlock, 0, s>>>(aa);
    CK(cudaGetLastError());
    recheck_kernel<TY><<<sms * 2, 256, 0, s>>>(y, ldy, d, k, as<double>(st.c64),
                                               as<int32_t>(st.flagged),
                                               as<unsigned long long>(st.counters), old, cur,
                                               as<unsigned long long>(st.counters));
    CK(cudaGetLastError());
    launches += 2;
    unsigned long long changed = 0;
    CK(cudaMemcpyAsync(&changed, st.counters.ptr, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    converged = it > 1 && changed == 0;
    if (converged || it == max_iter) break;
    CK(accumulate(cur));
    CK(finalize());
    old = cur;
    std::swap(cur, other);
  }
  if (it > max_iter) it = max_iter;
  // inertia against the centroids the final assignment was computed with
  const int igrid = sms * 8;
  inertia_kernel<TY><<<igrid, 256, 0, s>>>(y, ldy, n, d, as<float>(st.c32), cur,
                                            as<double>(st.inertia_part));
  CK(cudaGetLastError());
  CK(launch_reduce_partials(as<double>(st.inertia_part), 1, igrid, 1, 0,
                            as<double>(st.inertia_part) + igrid, s));
  launches += 2;
  double inertia = 0.0;
  CK(cudaMemcpyAsync(&inertia, as<double>(st.inertia_part) + igrid, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  res->iters = it;
  res->converged = converged;
  res->inertia = inertia;
  res->assign = cur;
  res->launches = launches;
  return CSC_OK;
}

}  // namespace

csc_status kmeans_run(KmeansState& st, const void* y, int y_dtype, int64_t n, int d, int64_t ldy,
                      int k, const int64_t* init_idx, const int32_t* prev_assign, int max_iter,
                      cudaStream_t s, KmeansResult* res, std::string* err) {
  if (y_dtype == CSC_BF16)
    return run_typed<__nv_bfloat16>(st, static_cast<const __nv_bfloat16*>(y), n, d, ldy, k,
                                    init_idx, prev_assign, max_iter, s, res, err);
  return run_typed<float>(st, static_cast<const float*>(y), n, d, ldy, k, init_idx, prev_assign,
                          max_iter, s, res, err);
}

void kmeans_release(KmeansState& st) {
  DevBuf* all[] = {&st.c64, &st.c32, &st.cn2, &st.cmax, &st.sums, &st.counts, &st.assign_a,
                   &st.assign_b, &st.flagged, &st.counters, &st.maxabs, &st.inertia_part,
                   &st.init_idx};
  for (DevBuf* b : all) release(*b);
}

}  // namespace csc
