// k-means (Lloyd) on the feature rows (Section 2.1, Eq. 1-2; the clustering of Algorithm 1).
//
// Pruning (Elkan's bounds): each row keeps an upper bound on its distance to its centroid and
// a lower bound on its distance to each centroid.  After an update moves centroid j by
// delta_j, the bounds become ub + delta_a and lb_j - delta_j (rounded outward); only the
// centroids whose lower bound falls below ub are re-measured, and a row with none keeps its
// centroid without reading its features.  The decisions are the same as without pruning.
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
// result does not depend on scheduling; an empty cluster keeps its centroid.  After the first
// pass only the rows that changed cluster add and subtract their quantised features, which
// gives exactly the same sums.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "csc_internal.h"

namespace csc {

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int kAssignBlock = 256;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Fixed-point value of a feature: x = y * 2^S (exact in float) rounded to the nearest integer,
// ties to even, from the float's fields with integer operations (the float-to-int64 conversion
// instruction runs on the FP64 pipe, which this part has little of).  Finite x, |x| < 2^63.
__device__ __forceinline__ long long fixed_rn(float x) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFFu);
  const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;  // x = m 2^(e - 150) for e >= 1
  long long q;
  if (e >= 150) {
    q = (long long)m << (e - 150);
  } else if (e < 126) {
    q = 0;  // |x| < 1/2
  } else {
    const int sh = 150 - e;  // 1 .. 24
    const uint32_t qi = m >> sh, r = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
    q = (long long)(qi + ((r > half || (r == half && (qi & 1u))) ? 1u : 0u));
  }
  return (b >> 31) ? -q : q;
}

// fixed_rn(y * 2^S) of a bfloat16 feature from its bits h: y = m 2^(e - 134), so the value is
// m shifted by e - 134 + S, rounded to nearest, ties to even, when the shift is negative.
// Equal to fixed_rn(float(y) * 2^S) (the same real number, the same rounding).
__device__ __forceinline__ long long fixed_bf16(uint32_t h, int S) {
  const int e = (int)((h >> 7) & 0xFFu);
  const uint32_t m = (h & 0x7Fu) | 0x80u;
  const int sh = e - 134 + S;
  long long q;
  if (e == 0) {
    q = 0;  // zero or subnormal: |y| 2^S < 2^(S - 126) < 1/2
  } else if (sh >= 0) {
    q = (long long)m << sh;
  } else if (sh < -8) {
    q = 0;  // m 2^sh < 2^(8 + sh) <= 1/2 exclusive
  } else {
    const int r = -sh;  // 1 .. 8
    const uint32_t qi = m >> r, rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
    q = (long long)(qi + ((rem > half || (rem == half && (qi & 1u))) ? 1u : 0u));
  }
  return (h & 0x8000u) ? -q : q;
}

template <typename TY>
__global__ void maxabs_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                              unsigned int* out) {
  float m = 0.f;
  const int64_t total = n * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / d;
    const int l = (int)(e - row * d);
    const float a = fabsf(ldf(y + row * ldy + l));
    m = a <= 3.0e38f ? fmaxf(m, a) : INFINITY;  // NaN/inf -> inf
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Counts labels outside [0, k) (a caller's previous assignment on the device).
__global__ void label_check_kernel(const int32_t* __restrict__ a, int64_t n, int k,
                                   unsigned long long* __restrict__ bad) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (a[i] < 0 || a[i] >= k) ? 1ull : 0ull;
  if (c) atomicAdd(bad, c);
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
      const long long q = fixed_rn(ldf(y + row * ldy + l) * scale);
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

// Fixed-point centroid sums by cluster-sorted rows (d <= 256).  The rows are bucketed by
// cluster with a counting sort (per-block histograms, a scan, a scatter); each warp then sums a
// run of consecutive bucketed rows in int64 registers and adds a partial to the global sums only
// when the cluster changes.  Integer sums, so the result does not depend on the order.
constexpr int kSortBlock = 256;

// Block b owns rows [b R, b R + R), R = ceil(n / gridDim.x); hist[b][j] = its rows in cluster j.
__global__ void sort_hist_kernel(const int32_t* __restrict__ assign, int64_t n, int k,
                                 int* __restrict__ hist) {
  extern __shared__ int sh_hist[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) sh_hist[j] = 0;
  __syncthreads();
  const int64_t R = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * R, r1 = min(n, r0 + R);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) atomicAdd(sh_hist + assign[r], 1);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) hist[(size_t)blockIdx.x * k + j] = sh_hist[j];
}

// One block: counts[j] = sum_b hist[b][j]; hist[b][j] becomes the first bucket slot of block b
// in cluster j (clusters in index order, blocks in order within a cluster).
__global__ void sort_scan_kernel(int* __restrict__ hist, int nblk, int k, int* __restrict__ counts) {
  __shared__ int tot[1024];
  __shared__ int base[1024];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int t = 0;
    for (int b = 0; b < nblk; ++b) t += hist[(size_t)b * k + j];
    tot[j] = t;
    counts[j] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int j = 0; j < k; ++j) { base[j] = acc; acc += tot[j]; }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int acc = base[j];
    for (int b = 0; b < nblk; ++b) {
      const int h = hist[(size_t)b * k + j];
      hist[(size_t)b * k + j] = acc;
      acc += h;
    }
  }
}

__global__ void sort_scatter_kernel(const int32_t* __restrict__ assign, int64_t n, int k,
                                    const int* __restrict__ hist, int32_t* __restrict__ perm) {
  extern __shared__ int cursor[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cursor[j] = hist[(size_t)blockIdx.x * k + j];
  __syncthreads();
  const int64_t R = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * R, r1 = min(n, r0 + R);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) perm[atomicAdd(cursor + assign[r], 1)] = (int32_t)r;
}

// Warp w sums bucketed rows [w C, w C + C); lane owns elements lane + 32 i, i < DW.
template <typename TY, int DW>
__global__ void seg_sum_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                               const int32_t* __restrict__ perm, const int32_t* __restrict__ assign,
                               float scale, unsigned long long* __restrict__ sums) {
  constexpr int C = 64;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = warp * C; c0 < n; c0 += nwarps * C) {
    const int64_t c1 = min(n, c0 + C);
    long long acc[DW];
#pragma unroll
    for (int i = 0; i < DW; ++i) acc[i] = 0;
    int cur = assign[perm[c0]];
    for (int64_t p = c0; p < c1; ++p) {
      const int64_t row = perm[p];
      const int a = assign[row];
      if (a != cur) {
#pragma unroll
        for (int i = 0; i < DW; ++i) {
          const int l = lane + 32 * i;
          if (l < d && acc[i] != 0) atomicAdd(sums + (size_t)cur * d + l, (unsigned long long)acc[i]);
          acc[i] = 0;
        }
        cur = a;
      }
#pragma unroll
      for (int i = 0; i < DW; ++i) {
        const int l = lane + 32 * i;
        if (l < d) acc[i] += fixed_rn(ldf(y + row * ldy + l) * scale);
      }
    }
#pragma unroll
    for (int i = 0; i < DW; ++i) {
      const int l = lane + 32 * i;
      if (l < d && acc[i] != 0) atomicAdd(sums + (size_t)cur * d + l, (unsigned long long)acc[i]);
    }
  }
}

// The same sums with eight values per lane (rows read with 16-byte loads) over runs of C
// bucketed rows, C chosen so that each warp of the grid takes about one run.  The cluster of
// bucket slot p follows from the bucket starts (prefix sums of counts, in shared memory), so a
// row costs one dependent load: the warp reads 32 slots of perm at once and keeps U rows in
// flight.  d <= 256, k <= 1024, rows_vec8.  The per-element fixed-point values and therefore
// the integer sums are those of seg_sum_kernel.
template <typename TY>
__global__ void seg_sum_vec_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                                   const int32_t* __restrict__ perm, const int* __restrict__ counts, int k,
                                   float scale, int S, unsigned long long* __restrict__ sums, int64_t C) {
  constexpr int U = 8;
  constexpr bool kBf16 = sizeof(TY) == 2;  // bfloat16 rows: fixed point from the bits (fixed_bf16)
  __shared__ long long start[1025];
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int j = 0; j < k; ++j) { start[j] = acc; acc += counts[j]; }
    start[k] = acc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const bool act = 8 * lane < d;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = warp * C; c0 < n; c0 += nwarps * C) {
    const int64_t c1 = min(n, c0 + C);
    // cluster of slot c0: the last j with start[j] <= c0
    int lo = 0, hi = k - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= c0) lo = mid; else hi = mid - 1;
    }
    int cur = lo;
    long long next = start[cur + 1];
    long long acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0;
    for (int64_t p32 = c0; p32 < c1; p32 += 32) {
      const int32_t pv = p32 + lane < c1 ? perm[p32 + lane] : 0;
      const int cnt = (int)min((int64_t)32, c1 - p32);
      for (int b = 0; b < cnt; b += U) {
        float v[U][8];
        uint4 raw[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t row = __shfl_sync(0xffffffffu, pv, (b + u) & 31);
          if constexpr (kBf16) {
            raw[u] = (b + u < cnt && act) ? __ldg(reinterpret_cast<const uint4*>(y + row * ldy + 8 * lane))
                                          : make_uint4(0u, 0u, 0u, 0u);
          } else if (b + u < cnt && act) {
            ld8(y + row * ldy + 8 * lane, v[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[u][e] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (b + u >= cnt) break;
          const int64_t p = p32 + b + u;
          if (p >= next) {
            if (act)
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (acc[e] != 0) atomicAdd(sums + (size_t)cur * d + 8 * lane + e, (unsigned long long)acc[e]);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] = 0;
            while (p >= next) next = start[++cur + 1];
          }
          if constexpr (kBf16) {
            const uint32_t w[4] = {raw[u].x, raw[u].y, raw[u].z, raw[u].w};
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += fixed_bf16((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu, S);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += fixed_rn(v[u][e] * scale);
          }
        }
      }
    }
    if (act)
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (acc[e] != 0) atomicAdd(sums + (size_t)cur * d + 8 * lane + e, (unsigned long long)acc[e]);
  }
}

// Means from the fixed-point sums (an empty cluster keeps its centroid), the float32 copies,
// |c32|^2, and for the pruning bounds the movement of every centroid (rounded up) and the
// largest movement.  One block per centroid.
__global__ void finalize_kernel(const unsigned long long* __restrict__ sums,
                                const int* __restrict__ counts, int k, int d, double inv_scale,
                                double* __restrict__ c64, float* __restrict__ c32,
                                float* __restrict__ cn2, float* __restrict__ cmove,
                                unsigned int* __restrict__ cmax_bits,
                                unsigned int* __restrict__ dmax_bits) {
  __shared__ double red[2][32];
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int cnt = counts[j];
  const double f = cnt > 0 ? inv_scale / (double)cnt : 0.0;
  double mv = 0.0, nrm = 0.0;
  for (int l = threadIdx.x; l < d; l += blockDim.x) {
    const size_t e = (size_t)j * d + l;
    const double old = c64[e];
    const double nwv = cnt > 0 ? (double)(long long)sums[e] * f : old;
    mv += (nwv - old) * (nwv - old);
    c64[e] = nwv;
    const float fv = (float)nwv;
    c32[e] = fv;
    nrm += (double)fv * (double)fv;
  }
  for (int off = 16; off > 0; off >>= 1) {
    mv += __shfl_xor_sync(0xffffffffu, mv, off);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  }
  if (lane == 0) { red[0][wid] = mv; red[1][wid] = nrm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    mv = 0.0; nrm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { mv += red[0][w]; nrm += red[1][w]; }
    cn2[j] = (float)nrm;
    const float move = __double2float_ru(sqrt(mv) * (1.0 + 1e-12));
    cmove[j] = move;
    atomicMax(cmax_bits, __float_as_uint(__double2float_ru(sqrt(nrm) * (1.0 + 1e-7))));
    atomicMax(dmax_bits, __float_as_uint(move));
  }
}

struct AssignArgs {
  const void* y;
  int64_t ldy, n;
  int d, k;
  const float* c32;   // [k][d]
  const float* cn2;   // [k]
  const unsigned int* cmax_bits;
  const int32_t* work;           // rows to decide (nullptr: all rows)
  int32_t* assign;               // in/out
  float* ub;                     // upper bound on the distance to the assigned centroid
  float* lbk;                    // [n][k] lower bounds on the distance to every centroid
  int32_t* flagged;
  int32_t* moved;                // [3][n]: row, old, new
  unsigned long long* counters;  // [0] moved, [1] flagged, [2] work
  int track;                     // append changed rows to `moved`
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

__device__ __forceinline__ void record_move(const AssignArgs& a, int64_t row, int old, int nw) {
  const unsigned long long m = atomicAdd(a.counters, 1ull);
  a.moved[m] = (int32_t)row;
  a.moved[a.n + m] = old;
  a.moved[2 * a.n + m] = nw;
}

template <typename TY>
__global__ void __launch_bounds__(kAssignBlock) assign_kernel(AssignArgs a) {
  __shared__ __align__(16) float Ys[BK][BM + 4];
  __shared__ __align__(16) float Cs[BK][BN + 4];
  __shared__ int64_t rows_s[BM];
  const TY* __restrict__ y = static_cast<const TY*>(a.y);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float cmax = __uint_as_float(*a.cmax_bits);
  const double u = 5.9604644775390625e-8;
  const int64_t count = a.work != nullptr ? (int64_t)a.counters[2] : a.n;
  const int64_t ntiles = (count + BM - 1) / BM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    if (tid < BM) {
      const int64_t t = tile * BM + tid;
      rows_s[tid] = t < count ? (a.work != nullptr ? (int64_t)a.work[t] : t) : -1;
    }
    __syncthreads();
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
          const int64_t row = rows_s[r];
          const int col = k0 + kk;
          Ys[kk][r] = (row >= 0 && col < a.d) ? ldf(y + row * a.ldy + col) : 0.f;
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
            const int64_t row = rows_s[ty * 4 + i];
            if (row >= 0) {
              // lower bound on |y - c_j| from f_j and its error bound (squared distance = |y|^2 + f)
              const double yn = (double)yn2[i];
              const double slack = u * (3.1 * cmax * cmax + 2.0 * (1.01 * a.d + 1.0) * sqrt(yn) * cmax) +
                                   2.0 * (a.d + 2.0) * u * yn;
              const double dl = (double)f + yn - slack;
              a.lbk[row * a.k + cj] = dl > 0.0 ? __double2float_rd(sqrt(dl) * (1.0 - 1e-6)) : 0.0f;
            }
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
        const int64_t row = rows_s[ty * 4 + i];
        if (row < 0) continue;
        const double yn = (double)yn2[i];
        const double bound = u * (3.1 * cmax * cmax + 2.0 * (1.01 * a.d + 1.0) * sqrt(yn) * cmax);
        if (!((double)second[i] - (double)best[i] > 4.0 * bound)) {
          const unsigned long long slot = atomicAdd(a.counters + 1, 1ull);
          a.flagged[slot] = (int32_t)row;
          continue;
        }
        // squared distance = yn2 + f, each known to within its error bound
        const double slack = bound + 2.0 * (a.d + 2.0) * u * yn;
        const double dmin = (double)best[i] + yn + slack;
        a.ub[row] = __double2float_ru(sqrt(fmax(dmin, 0.0)) * (1.0 + 1e-6));
        const int old = a.assign[row];
        a.assign[row] = bidx[i];
        if (a.track && old != bidx[i]) record_move(a, row, old, bidx[i]);
      }
    }
  }
}

// Float64 decision for the flagged rows: one warp per row, all centroids, lowest index on ties.
template <typename TY>
__global__ void recheck_kernel(AssignArgs a, const double* __restrict__ c64) {
  const TY* __restrict__ y = static_cast<const TY*>(a.y);
  const unsigned long long nflag = a.counters[1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < (int64_t)nflag; w += nwarps) {
    const int64_t row = a.flagged[w];
    double best = INFINITY, second = INFINITY;
    int bi = 0;
    for (int j = 0; j < a.k; ++j) {
      double s = 0.0;
      for (int l = lane; l < a.d; l += 32) {
        const double diff = (double)ldf(y + row * a.ldy + l) - c64[(size_t)j * a.d + l];
        s = fma(diff, diff, s);
      }
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) a.lbk[row * a.k + j] = __double2float_rd(sqrt(s) * (1.0 - 1e-9));
      if (s < best) { second = best; best = s; bi = j; }
      else if (s < second) second = s;
    }
    if (lane == 0) {
      a.ub[row] = __double2float_ru(sqrt(best) * (1.0 + 1e-9));
      const int old = a.assign[row];
      a.assign[row] = bi;
      if (a.track && old != bi) record_move(a, row, old, bi);
    }
  }
}

// Pruned Lloyd pass (Elkan's bounds), lazily updated.  A row's bounds refer to the centroid
// version vstamp[row] at which they were last written; drift[v][j] (rounded up) bounds how far
// centroid j moved since version v, so the current bounds are ub + drift[v][a] and
// lb_j - drift[v][j].  Rows whose bounds still exclude every other centroid are neither read
// again nor rewritten.

// Scan: marks the rows with at least one candidate centroid (lb_j <= ub, j != a).
__global__ void elkan_scan_kernel(int64_t n, int k, const int32_t* __restrict__ assign,
                                  const int32_t* __restrict__ vstamp, const float* __restrict__ ub,
                                  const float* __restrict__ lbk, const float* __restrict__ drift,
                                  int32_t* __restrict__ work, unsigned long long* __restrict__ counters) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int asg = __ldg(assign + row);
    const float* dv = drift + (size_t)__ldg(vstamp + row) * k;
    const float u = __fadd_ru(__ldg(ub + row), __ldg(dv + asg));
    const float* lrow = lbk + row * k;
    bool cand = false;
    for (int j = lane; j < k; j += 32)
      cand |= (j != asg) && !(u < __fsub_rd(__ldcs(lrow + j), __ldg(dv + j)));
    if (__any_sync(0xffffffffu, cand) && lane == 0) {
      const unsigned long long slot = atomicAdd(counters + 2, 1ull);
      work[slot] = (int32_t)row;
    }
  }
}

// Refine: one warp per listed row.  Brings the bounds to the current version, measures the
// distance to the own centroid (tightening ub) and to every remaining candidate in float32
// with its error bound e(D) = (d+3) u D + 2u sqrt(D) cmax, and decides.  When the best two are
// closer than their error bounds, the candidates that can still be the minimum are measured
// in float64 (lowest index on ties); the other centroids are provably farther.
template <typename TY, int DW>
__global__ void elkan_refine_kernel(AssignArgs a, const int32_t* __restrict__ work,
                                    const float* __restrict__ drift, int32_t* __restrict__ vstamp,
                                    int version, const double* __restrict__ c64) {
  const TY* __restrict__ y = static_cast<const TY*>(a.y);
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float cmax = __uint_as_float(*a.cmax_bits);
  const float u = 5.9604644775390625e-8f;
  const int d = a.d, k = a.k;
  const float erel = (d + 3.0f) * u;
  const float eabs = 2.0f * u * cmax;
  const int64_t nwork = (int64_t)a.counters[2];
  for (int64_t w = warp; w < nwork; w += nwarps) {
    const int64_t row = work[w];
    const int asg = a.assign[row];
    const float* dv = drift + (size_t)vstamp[row] * k;
    float* lrow = a.lbk + row * k;
    for (int j = lane; j < k; j += 32) lrow[j] = fmaxf(__fsub_rd(lrow[j], __ldg(dv + j)), 0.0f);
    float yv[DW];
#pragma unroll
    for (int i = 0; i < DW; ++i) {
      const int l = lane + 32 * i;
      yv[i] = l < d ? ldf(y + row * a.ldy + l) : 0.0f;
    }
    __syncwarp();
    auto dist = [&](int j) {
      const float* c = a.c32 + (size_t)j * d;
      float sacc = 0.f;
#pragma unroll
      for (int i = 0; i < DW; ++i) {
        const int l = lane + 32 * i;
        if (l < d) {
          const float df = yv[i] - __ldg(c + l);
          sacc = fmaf(df, df, sacc);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
      return sacc;
    };
    auto dist64 = [&](int j) {
      const double* c = c64 + (size_t)j * d;
      double sacc = 0.0;
#pragma unroll
      for (int i = 0; i < DW; ++i) {
        const int l = lane + 32 * i;
        if (l < d) {
          const double df = (double)yv[i] - c[l];
          sacc = fma(df, df, sacc);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
      return sacc;
    };
    const float da = dist(asg), ea = erel * da + eabs * sqrtf(da);
    const float ub = __fsqrt_ru(__fadd_ru(da, ea));
    float best = da, ebest = ea;
    int bi = asg;
    float second = INFINITY, esecond = 0.f;
    for (int j0 = 0; j0 < k; j0 += 32) {
      const int j = j0 + lane;
      const bool cand = j < k && j != asg && !(ub < lrow[j]);
      unsigned mask = __ballot_sync(0xffffffffu, cand);
      while (mask) {
        const int q = j0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const float dq = dist(q), eq = erel * dq + eabs * sqrtf(dq);
        if (lane == (q & 31)) lrow[q] = __fsqrt_rd(fmaxf(__fsub_rd(dq, eq), 0.0f));
        if (dq < best || (dq == best && q < bi)) {
          second = best; esecond = ebest;
          best = dq; ebest = eq; bi = q;
        } else if (dq < second) {
          second = dq; esecond = eq;
        }
      }
    }
    if (!(second - best > ebest + esecond)) {
      // near tie: float64 on every centroid whose lower bound still admits the minimum
      // (true distance^2 <= best + ebest); the others are provably farther
      __syncwarp();
      const float limit = __fsqrt_ru(__fadd_ru(best, 2.0f * ebest));
      double b64 = dist64(asg);
      int b64i = asg;
      for (int j0 = 0; j0 < k; j0 += 32) {
        const int j = j0 + lane;
        const bool maybe = j < k && j != asg && lrow[j] <= limit;
        unsigned mask = __ballot_sync(0xffffffffu, maybe);
        while (mask) {
          const int q = j0 + __ffs(mask) - 1;
          mask &= mask - 1;
          const double dq = dist64(q);
          if (dq < b64 || (dq == b64 && q < b64i)) { b64 = dq; b64i = q; }
        }
      }
      bi = b64i;
      best = (float)b64;
      ebest = __fmul_ru((float)b64, 1e-6f) + eabs;
    }
    if (lane == 0) {
      a.ub[row] = __fsqrt_ru(__fadd_ru(best, ebest));
      vstamp[row] = version;
      if (bi != asg) {
        lrow[asg] = __fsqrt_rd(fmaxf(__fsub_rd(da, ea), 0.0f));
        a.assign[row] = bi;
        if (a.track) record_move(a, row, asg, bi);
      }
    }
  }
}

// Fused pruned pass for k <= 32*KC, d <= 128*DW4, d a multiple of 4 (16-byte rows): one warp
// per row, no work list.  The row's bounds (KC per lane) and features (DW4 float4 per lane)
// are loaded up front; rows whose bounds exclude every other centroid write nothing (their
// bounds stay lazy).  Distances use f_j = |c_j|^2 - 2 <y, c_j> with the error bound
// B = u (3.1 cmax^2 + 2 (1.01 d + 1) |y| cmax) of the distance pass (|y|^2 is common to all
// centroids of the row and cancels in the decision).  The first batch (own centroid plus up to
// three candidates) tightens ub; the remaining candidates are listed once and measured four
// at a time.
__device__ __forceinline__ float4 ld4f(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4f(const __nv_bfloat16* p) {
  const uint2 raw = *reinterpret_cast<const uint2*>(p);
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <typename TY, int DW4, int KC>
__global__ void __launch_bounds__(256) elkan_pass_kernel(AssignArgs a, const float* __restrict__ drift,
                                                         int32_t* __restrict__ vstamp, int version,
                                                         const double* __restrict__ c64) {
  __shared__ int clist[8][32 * KC];
  const TY* __restrict__ y = static_cast<const TY*>(a.y);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float cmax = __uint_as_float(*a.cmax_bits);
  const float u = 5.9604644775390625e-8f;
  const int d = a.d, k = a.k;
  int* cl = clist[wid];
  for (int64_t row = warp; row < a.n; row += nwarps) {
    const int asg = a.assign[row];
    const int vs = vstamp[row];
    const float ub0 = a.ub[row];
    float* lrow = a.lbk + row * k;
    float l[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      const int j = lane + 32 * i;
      l[i] = j < k ? __ldcs(lrow + j) : INFINITY;
    }
    const float* dv = drift + (size_t)vs * k;
    float ubv = __fadd_ru(ub0, __ldg(dv + asg));
    bool any = false;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      const int j = lane + 32 * i;
      if (j < k) l[i] = fmaxf(__fsub_rd(l[i], __ldg(dv + j)), 0.0f);
      any |= j < k && j != asg && !(ubv < l[i]);
    }
    if (!__any_sync(0xffffffffu, any)) continue;  // keeps its centroid; bounds stay lazy
    // features: lane owns elements 128 t + 4 lane .. +3
    float4 yv[DW4];
    float yn = 0.f;
#pragma unroll
    for (int t = 0; t < DW4; ++t) {
      const int e = 128 * t + 4 * lane;
      yv[t] = e < d ? ld4f(y + row * a.ldy + e) : make_float4(0.f, 0.f, 0.f, 0.f);
      yn = fmaf(yv[t].x, yv[t].x, fmaf(yv[t].y, yv[t].y, fmaf(yv[t].z, yv[t].z, fmaf(yv[t].w, yv[t].w, yn))));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) yn += __shfl_xor_sync(0xffffffffu, yn, off);
    const float B = u * (3.1f * cmax * cmax + 2.0f * (1.01f * d + 1.0f) * sqrtf(yn) * cmax);
    const float ey = (d + 2.0f) * u * yn;  // error of yn itself (bounds only)
    auto measure = [&](const int (&q)[4], int nq, float (&f)[4]) {
      float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t < nq) {
          const float* c = a.c32 + (size_t)q[t] * d;
#pragma unroll
          for (int w = 0; w < DW4; ++w) {
            const int e = 128 * w + 4 * lane;
            if (e < d) {
              const float4 cv = ld4f(c + e);
              part[t] = fmaf(yv[w].x, cv.x, fmaf(yv[w].y, cv.y, fmaf(yv[w].z, cv.z, fmaf(yv[w].w, cv.w, part[t]))));
            }
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int t = 0; t < 4; ++t) part[t] += __shfl_xor_sync(0xffffffffu, part[t], off);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nq) f[t] = fmaf(-2.0f, part[t], __ldg(a.cn2 + q[t]));
    };
    float best = INFINITY, second = INFINITY, fa = 0.f;
    int bi = asg;
    auto consider = [&](int qq, float f) {
      if (qq == asg) {
        fa = f;
        ubv = __fsqrt_ru(fmaxf(__fadd_ru(__fadd_ru(yn, f), B + ey), 0.0f));  // tightened
      } else {
        const float lq = __fsqrt_rd(fmaxf(__fsub_rd(__fadd_rd(yn, f), B + ey), 0.0f));
#pragma unroll
        for (int i = 0; i < KC; ++i)
          if (lane == (qq & 31) && i == (qq >> 5)) l[i] = lq;
      }
      if (f < best || (f == best && qq < bi)) {
        second = best; best = f; bi = qq;
      } else if (f < second) {
        second = f;
      }
    };
    // batch 0: own centroid + up to three loose candidates (index order)
    int q[4] = {asg, 0, 0, 0};
    int nq = 1;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      const int j = lane + 32 * i;
      unsigned mask = __ballot_sync(0xffffffffu, j < k && j != asg && !(ubv < l[i]));
#pragma unroll
      for (int t = 1; t < 4; ++t) {
        if (t == nq && mask) {
          q[t] = 32 * i + __ffs(mask) - 1;
          mask &= mask - 1;
          ++nq;
        }
      }
    }
    {
      float f[4];
      measure(q, nq, f);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nq) consider(q[t], f[t]);
    }
    // remaining candidates under the tightened bound, listed once
    int nc = 0;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      const int j = lane + 32 * i;
      bool cand = j < k && j != asg && !(ubv < l[i]);
#pragma unroll
      for (int t = 1; t < 4; ++t) cand &= !(t < nq && j == q[t]);
      const unsigned mask = __ballot_sync(0xffffffffu, cand);
      if (cand) cl[nc + __popc(mask & ((1u << lane) - 1u))] = j;
      nc += __popc(mask);
    }
    __syncwarp();
    for (int c0 = 0; c0 < nc; c0 += 4) {
      int qb[4];
      const int nb = min(4, nc - c0);
#pragma unroll
      for (int t = 0; t < 4; ++t) qb[t] = t < nb ? cl[c0 + t] : 0;
      float f[4];
      measure(qb, nb, f);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nb) consider(qb[t], f[t]);
    }
    __syncwarp();
    if (!(second - best > 2.0f * B)) {
      // near tie: float64 on every centroid whose lower bound still admits the minimum
      const float limit = __fsqrt_ru(__fadd_ru(__fadd_ru(yn, best), 2.0f * B + ey));
      double b64 = INFINITY;
      int b64i = asg;
      for (int i = 0; i < KC; ++i) {
        const int j = lane + 32 * i;
        const bool maybe = j < k && (j == asg || l[i] <= limit);
        unsigned mask = __ballot_sync(0xffffffffu, maybe);
        while (mask) {
          const int qq = 32 * i + __ffs(mask) - 1;
          mask &= mask - 1;
          const double* c = c64 + (size_t)qq * d;
          double sacc = 0.0;
#pragma unroll
          for (int w = 0; w < DW4; ++w) {
            const int e = 128 * w + 4 * lane;
            if (e < d) {
              const double d0 = (double)yv[w].x - c[e], d1 = (double)yv[w].y - c[e + 1];
              const double d2 = (double)yv[w].z - c[e + 2], d3 = (double)yv[w].w - c[e + 3];
              sacc = fma(d0, d0, fma(d1, d1, fma(d2, d2, fma(d3, d3, sacc))));
            }
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
          if (sacc < b64 || (sacc == b64 && qq < b64i)) { b64 = sacc; b64i = qq; }
        }
      }
      bi = b64i;
      best = __fsub_ru((float)b64, yn);  // back to the f scale; bounds below use B + ey slack
    }
    // write back the bounds at the current version
    if (bi != asg) {
      const float la = __fsqrt_rd(fmaxf(__fsub_rd(__fadd_rd(yn, fa), B + ey), 0.0f));
#pragma unroll
      for (int i = 0; i < KC; ++i)
        if (lane == (asg & 31) && i == (asg >> 5)) l[i] = la;
    }
#pragma unroll
    for (int i = 0; i < KC; ++i) {
      const int j = lane + 32 * i;
      if (j < k) lrow[j] = l[i];
    }
    if (lane == 0) {
      a.ub[row] = __fsqrt_ru(fmaxf(__fadd_ru(__fadd_ru(yn, best), B + ey + 1e-6f * (yn + fabsf(best))), 0.0f));
      vstamp[row] = version;
      if (bi != asg) {
        a.assign[row] = bi;
        if (a.track) record_move(a, row, asg, bi);
      }
    }
  }
}

// Applies the fixed-point deltas of the rows that changed cluster: one warp per row.
template <typename TY>
__global__ void move_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                            const int32_t* __restrict__ moved, const unsigned long long* counters,
                            float scale, unsigned long long* __restrict__ sums,
                            int* __restrict__ counts) {
  const unsigned long long nm = counters[0];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = warp; m < (int64_t)nm; m += nwarps) {
    const int64_t row = moved[m];
    const int old = moved[n + m], nw = moved[2 * n + m];
    for (int l = lane; l < d; l += 32) {
      const long long q = fixed_rn(ldf(y + row * ldy + l) * scale);
      atomicAdd(sums + (size_t)nw * d + l, (unsigned long long)q);
      atomicAdd(sums + (size_t)old * d + l, (unsigned long long)(-q));
    }
    if (lane == 0) {
      atomicAdd(counts + nw, 1);
      atomicAdd(counts + old, -1);
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

// The same inertia with eight values per lane (rows_vec8): each warp takes a contiguous run
// of rows, reads their labels 32 at a time, keeps U rows in flight, and sums its lanes' float
// partials in float64, reduced once at the end.
template <typename TY>
__global__ void inertia_vec_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d,
                                   const float* __restrict__ c32, const int32_t* __restrict__ assign,
                                   double* __restrict__ part) {
  constexpr int U = 4;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int groups = d / 8;
  const int64_t C = (n + nwarps - 1) / nwarps;
  const int64_t r0 = warp * C, r1 = min(n, r0 + C);
  double acc = 0.0;
  for (int64_t p32 = r0; p32 < r1; p32 += 32) {
    const int av = p32 + lane < r1 ? assign[p32 + lane] : 0;
    const int cnt = (int)min((int64_t)32, r1 - p32);
    for (int b = 0; b < cnt; b += U) {
      int a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = __shfl_sync(0xffffffffu, av, (b + u) & 31);
      float s = 0.f;
      for (int g = lane; g < groups; g += 32) {
        float v[U][8], q[U][8];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (b + u < cnt) {
            ld8(y + (p32 + b + u) * ldy + 8 * g, v[u]);
            ld8(c32 + (size_t)a[u] * d + 8 * g, q[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[u][e] = q[u][e] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float df = v[u][e] - q[u][e];
            s = fmaf(df, df, s);
          }
      }
      acc += (double)s;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

bool debug_on() {
  static int on = -1;
  if (on < 0) on = getenv("CSC_DEBUG") != nullptr;
  return on == 1;
}
#define TRACE(msg) \
  do { if (debug_on()) { fprintf(stderr, "[csc] %s\n", msg); fflush(stderr); } } while (0)

#define CK(call)                                          \
  do {                                                    \
    TRACE(#call);                                         \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      if (err) *err = std::string(#call ": ") + cudaGetErrorString(e_); \
      return CSC_ECUDA;                                   \
    }                                                     \
  } while (0)

template <typename TY>
cudaError_t launch_refine(int d, int sms, cudaStream_t s, const AssignArgs& aa, const int32_t* work,
                          const float* drift, int32_t* vstamp, int version, const double* c64) {
  const int grid = sms * 8, block = 256;
  if (d <= 64)
    elkan_refine_kernel<TY, 2><<<grid, block, 0, s>>>(aa, work, drift, vstamp, version, c64);
  else if (d <= 128)
    elkan_refine_kernel<TY, 4><<<grid, block, 0, s>>>(aa, work, drift, vstamp, version, c64);
  else if (d <= 256)
    elkan_refine_kernel<TY, 8><<<grid, block, 0, s>>>(aa, work, drift, vstamp, version, c64);
  else if (d <= 512)
    elkan_refine_kernel<TY, 16><<<grid, block, 0, s>>>(aa, work, drift, vstamp, version, c64);
  else
    elkan_refine_kernel<TY, 32><<<grid, block, 0, s>>>(aa, work, drift, vstamp, version, c64);
  return cudaGetLastError();
}

template <typename TY, int DW4>
cudaError_t launch_fused_k(int k, int sms, cudaStream_t s, const AssignArgs& aa, const float* drift,
                           int32_t* vstamp, int version, const double* c64) {
  const int grid = sms * 8;
  if (k <= 32)
    elkan_pass_kernel<TY, DW4, 1><<<grid, 256, 0, s>>>(aa, drift, vstamp, version, c64);
  else if (k <= 64)
    elkan_pass_kernel<TY, DW4, 2><<<grid, 256, 0, s>>>(aa, drift, vstamp, version, c64);
  else
    elkan_pass_kernel<TY, DW4, 4><<<grid, 256, 0, s>>>(aa, drift, vstamp, version, c64);
  return cudaGetLastError();
}

template <typename TY>
cudaError_t launch_fused(int d, int k, int sms, cudaStream_t s, const AssignArgs& aa,
                         const float* drift, int32_t* vstamp, int version, const double* c64) {
  if (d <= 128) return launch_fused_k<TY, 1>(k, sms, s, aa, drift, vstamp, version, c64);
  return launch_fused_k<TY, 2>(k, sms, s, aa, drift, vstamp, version, c64);
}

template <typename TY>
csc_status run_typed(KmeansState& st, const TY* y, int64_t n, int d, int64_t ldy, int k,
                     const int64_t* init_idx, const int32_t* prev_assign, int max_iter,
                     cudaStream_t s, KmeansResult* res, std::string* err) {
  const size_t kd = (size_t)k * d;
  const int sms = num_sms();
  const bool vec8 = rows_vec8(y, d, ldy);  // rows read with 16-byte loads
  const int y_dtype = sizeof(TY) == 2 ? CSC_BF16 : CSC_F32;
  const TcPlan tp = kmeans_tc_plan(n, k, d, y_dtype);
  const bool use_tc = tp.ok;
  if (!ensure(st.c64, kd * 8) || !ensure(st.c32, kd * 4) || !ensure(st.cn2, (size_t)k * 4) ||
      !ensure(st.cmove, (size_t)k * 4) || !ensure(st.bits, 16) || !ensure(st.sums, kd * 8) ||
      !ensure(st.counts, (size_t)k * 4) || !ensure(st.assign, (size_t)n * 4) ||
      !ensure(st.flagged, (size_t)n * 4) || !ensure(st.moved, (size_t)n * 12) ||
      !ensure(st.counters, 64) || !ensure(st.init_idx, (size_t)k * 8) ||
      !ensure(st.inertia_part, ((size_t)sms * 8 + 1) * 8) ||
      (!use_tc && (!ensure(st.ub, (size_t)n * 4) || !ensure(st.lbk, (size_t)n * k * 4) ||
                   !ensure(st.work, (size_t)n * 4) || !ensure(st.vstamp, (size_t)n * 4) ||
                   !ensure(st.drift, (size_t)(max_iter + 1) * k * 4)))) {
    if (err) *err = "k-means: device allocation failed";
    return CSC_ENOMEM;
  }
  unsigned int* bits = as<unsigned int>(st.bits);  // [0] max|c|, [1] max move, [2] max|y|
  unsigned long long* counters = as<unsigned long long>(st.counters);
  int64_t launches = 0;
  // fixed-point scale from max |y|
  CK(cudaMemsetAsync(st.bits.ptr, 0, 16, s));
  if (use_tc) {
    // the bfloat16 split for the tensor-core pass also yields max |y|
    CK(kmeans_tc_prepare(st, tp, y, y_dtype, n, d, ldy, bits + 2, s));
  } else {
    TRACE("maxabs");
    maxabs_kernel<TY><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, bits + 2);
    CK(cudaGetLastError());
  }
  ++launches;
  CK(cudaMemsetAsync(counters + 5, 0, 8, s));
  if (prev_assign != nullptr) {
    label_check_kernel<<<sms * 2, 256, 0, s>>>(prev_assign, n, k, counters + 5);
    CK(cudaGetLastError());
    ++launches;
  }
  unsigned int mbits = 0;
  unsigned long long bad_labels = 0;
  CK(cudaMemcpyAsync(&mbits, bits + 2, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&bad_labels, counters + 5, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad_labels != 0) {
    if (err) *err = "k-means: previous assignment has labels outside [0, k)";
    return CSC_EINVAL;
  }
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
  TRACE("forgy");
  forgy_kernel<TY><<<std::max(1, (int)std::min<size_t>((kd + 255) / 256, 1024)), 256, 0, s>>>(
      y, ldy, as<int64_t>(st.init_idx), k, d, as<double>(st.c64));
  CK(cudaGetLastError());
  ++launches;
  const size_t smem = kd * 8 + (size_t)k * 4;
  const bool use_smem = smem <= 220 * 1024;
  const bool use_sort = d <= 256 && k <= 1024;
  const int sort_grid = sms * 2;
  if (use_sort && (!ensure(st.perm, (size_t)n * 4) || !ensure(st.hist, (size_t)sort_grid * k * 4))) {
    if (err) *err = "k-means: device allocation failed";
    return CSC_ENOMEM;
  }
  auto accumulate = [&](const int32_t* asg) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(st.sums.ptr, 0, kd * 8, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.counts.ptr, 0, (size_t)k * 4, s);
    if (e != cudaSuccess) return e;
    if (asg == nullptr) return cudaSuccess;
    if (use_sort) {
      int* hist = as<int>(st.hist);
      int32_t* perm = as<int32_t>(st.perm);
      sort_hist_kernel<<<sort_grid, kSortBlock, (size_t)k * 4, s>>>(asg, n, k, hist);
      sort_scan_kernel<<<1, 1024, 0, s>>>(hist, sort_grid, k, as<int>(st.counts));
      sort_scatter_kernel<<<sort_grid, kSortBlock, (size_t)k * 4, s>>>(asg, n, k, hist, perm);
      const int g = sms * 8;
      unsigned long long* sums = as<unsigned long long>(st.sums);
      if (vec8)
        seg_sum_vec_kernel<TY><<<g, 256, 0, s>>>(y, ldy, n, d, perm, as<int>(st.counts), k, scale, S, sums,
                                                 std::max<int64_t>(64, (n + (int64_t)g * 8 - 1) / ((int64_t)g * 8)));
      else if (d <= 32)
        seg_sum_kernel<TY, 1><<<g, 256, 0, s>>>(y, ldy, n, d, perm, asg, scale, sums);
      else if (d <= 64)
        seg_sum_kernel<TY, 2><<<g, 256, 0, s>>>(y, ldy, n, d, perm, asg, scale, sums);
      else if (d <= 128)
        seg_sum_kernel<TY, 4><<<g, 256, 0, s>>>(y, ldy, n, d, perm, asg, scale, sums);
      else
        seg_sum_kernel<TY, 8><<<g, 256, 0, s>>>(y, ldy, n, d, perm, asg, scale, sums);
      launches += 4;
      return cudaGetLastError();
    }
    ++launches;
    if (use_smem) {
      e = cudaFuncSetAttribute(update_kernel<TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      update_kernel<TY, true><<<sms, 1024, smem, s>>>(y, ldy, n, d, asg, k, scale,
                                                      as<unsigned long long>(st.sums),
                                                      as<int>(st.counts));
    } else {
      update_kernel<TY, false><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, asg, k, scale,
                                                       as<unsigned long long>(st.sums),
                                                       as<int>(st.counts));
    }
    return cudaGetLastError();
  };
  auto finalize = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(st.bits.ptr, 0, 8, s);
    if (e != cudaSuccess) return e;
    ++launches;
    finalize_kernel<<<k, 128, 0, s>>>(as<unsigned long long>(st.sums), as<int>(st.counts), k, d,
                                       inv_scale, as<double>(st.c64), as<float>(st.c32),
                                       as<float>(st.cn2), as<float>(st.cmove), bits, bits + 1);
    return cudaGetLastError();
  };
  CK(accumulate(prev_assign));
  CK(finalize());

  if (use_tc) {
    // Tensor-core distance pass (every row in the first pass; later passes skip the rows whose
    // Hamerly bounds certify their centroid); near ties decided in float64.  The
    // host queues pass it before it reads the counters of pass it - kPassLag (copied to pinned
    // memory), so the GPU does not wait for the host between passes.  A lag of 2 would also
    // cover a host slower than a pass, but its second update is then always the full
    // recomputation (2.5 ms more per call on the 8e6-node power-law features), so it is 1.  The update after pass
    // it is either the full recomputation or the incremental one from the moved rows; both
    // give the same integer sums, and the choice (full after the first pass and whenever the
    // previous pass moved more than n / 16 rows) only affects speed.  When pass j turns out
    // to have converged, passes j + 1 .. j + kPassLag are already queued: they find no move and
    // leave the assignment, the sums and the centroids as they were, so the result is the one
    // at j.
    if (st.hist_cap < (size_t)max_iter * 5) {
      if (st.hist_host) cudaFreeHost(st.hist_host);
      st.hist_host = nullptr;
      st.hist_cap = 0;
      CK(cudaHostAlloc(reinterpret_cast<void**>(&st.hist_host), (size_t)max_iter * 5 * 8, cudaHostAllocDefault));
      st.hist_cap = (size_t)max_iter * 5;
    }
    for (cudaEvent_t& e : st.pass_ev)
      if (e == nullptr) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaMemsetAsync(counters + 4, 0, 8, s));
    int examined = 0, stop = 0;
    unsigned long long last_moved = ~0ull;
    // bound selection per pass; it stops while it does not pay (the last examined selecting pass
    // evaluated every row in place) and is tried again every kSelectRetry passes
    constexpr int kSelectRetry = 4;
    constexpr int kPassLag = 1, kPassLag1 = kPassLag + 1;  // passes queued ahead of the host
    std::vector<char> selected((size_t)max_iter + 2, 0);
    bool select_paid = true;
    int last_select = 0;
    bool converged = false;
    int64_t decided = 0;
    // reads the counters of pass j (1-based) once its copy has completed
    auto examine = [&](int j) -> csc_status {
      cudaError_t e = cudaEventSynchronize(st.pass_ev[j % kPassLag1]);
      if (e != cudaSuccess) {
        if (err) *err = std::string("k-means: ") + cudaGetErrorString(e);
        return CSC_ECUDA;
      }
      const unsigned long long* cnt = st.hist_host + (size_t)(j - 1) * 5;
      if (cnt[4] != 0) {
        if (err) *err = "k-means: a bounded wait in the tensor-core pass expired (code " +
                        std::to_string(cnt[4]) + ")";
        return CSC_ETIMEOUT;
      }
      res->near_ties += (int64_t)cnt[1];
      decided += selected[j] ? (int64_t)cnt[2] : n;  // a selecting pass evaluates cnt[2] rows
      if (selected[j]) select_paid = cnt[2] < (unsigned long long)n;
      examined = j;
      // a cold first pass does not record moves; a warm one records them against prev_assign
      last_moved = (j == 1 && prev_assign == nullptr) ? ~0ull : cnt[0];
      if (debug_on()) {
        fprintf(stderr, "[csc] kmeans tc pass %d: near ties %llu moved %llu\n", j, cnt[1], cnt[0]);
        fflush(stderr);
      }
      if (j > 1 && cnt[0] == 0) converged = true;
      return CSC_OK;
    };
    for (int it = 1; it <= max_iter; ++it) {
      CK(cudaMemsetAsync(counters, 0, 32, s));
      TRACE("tc pass");
      const bool sel = it > 1 && (select_paid || it - last_select >= kSelectRetry);
      selected[it] = sel;
      if (sel) last_select = it;
      if (it == 1 && prev_assign != nullptr)
        CK(cudaMemcpyAsync(st.assign.ptr, prev_assign, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
      CK(kmeans_tc_pass(st, tp, y, y_dtype, n, d, ldy, k, it > 1 || prev_assign != nullptr, sel, s));
      launches += 3;
      CK(cudaMemcpyAsync(st.hist_host + (size_t)(it - 1) * 5, counters, 40, cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(st.pass_ev[it % kPassLag1], s));
      stop = it;
      if (it > kPassLag) {
        const csc_status cs = examine(it - kPassLag);
        if (cs != CSC_OK) return cs;
        if (converged) break;
      }
      if (it == max_iter) break;
      if (it == 1 || last_moved > (unsigned long long)(n / 16)) {
        CK(accumulate(as<int32_t>(st.assign)));
      } else {
        move_kernel<TY><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, as<int32_t>(st.moved), counters, scale,
                                                as<unsigned long long>(st.sums), as<int>(st.counts));
        CK(cudaGetLastError());
        ++launches;
      }
      CK(finalize());
    }
    for (int j = examined + 1; j <= stop && !converged; ++j) {
      const csc_status cs = examine(j);
      if (cs != CSC_OK) return cs;
    }
    res->iters = examined;
    res->converged = converged;
    res->decided = decided;
  }

  int assign_grid = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&assign_grid, assign_kernel<TY>, kAssignBlock, 0);
  assign_grid = std::max(1, assign_grid) * sms;
  AssignArgs aa{y, ldy, n, d, k, as<float>(st.c32), as<float>(st.cn2), bits, nullptr,
                as<int32_t>(st.assign), as<float>(st.ub), as<float>(st.lbk), as<int32_t>(st.flagged),
                as<int32_t>(st.moved), counters, 0};
  std::vector<double> cum((size_t)(max_iter + 1) * k, 0.0);
  std::vector<float> drift_h((size_t)(max_iter + 1) * k, 0.0f), move_h(k, 0.0f);
  int it = 0;
  bool converged = false;
  int64_t decided = 0;
  for (it = 1; it <= max_iter && !use_tc; ++it) {
    CK(cudaMemsetAsync(counters, 0, 32, s));
    int64_t rows = n;
    if (it == 1) {
      // first pass: every row against every centroid (register-tiled distance pass); the
      // bounds it writes refer to centroid version 0
      aa.track = 0;
      CK(cudaMemsetAsync(st.vstamp.ptr, 0, (size_t)n * 4, s));
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(assign_grid, (n + BM - 1) / BM));
      TRACE("assign");
      assign_kernel<TY><<<grid, kAssignBlock, 0, s>>>(aa);
      CK(cudaGetLastError());
      recheck_kernel<TY><<<sms * 2, 256, 0, s>>>(aa, as<double>(st.c64));
      CK(cudaGetLastError());
      launches += 2;
    } else {
      // drift[v][j]: movement of centroid j from version v to the current version (it - 1)
      const int cur = it - 1;
      for (int v = 0; v <= cur; ++v)
        for (int j = 0; j < k; ++j) {
          const double dj = (cum[(size_t)cur * k + j] - cum[(size_t)v * k + j]) * (1.0 + 1e-9);
          float f = (float)dj;
          if ((double)f < dj) f = std::nextafter(f, INFINITY);
          drift_h[(size_t)v * k + j] = f;
        }
      CK(cudaMemcpyAsync(st.drift.ptr, drift_h.data(), (size_t)(cur + 1) * k * 4,
                         cudaMemcpyHostToDevice, s));
      aa.track = 1;
      // the fused pass reads rows with 16-byte (8-byte for bf16) vector loads
      const bool aligned = d % 4 == 0 && ldy % 4 == 0 &&
                           (reinterpret_cast<uintptr_t>(y) % (4 * sizeof(TY))) == 0;
      if (k <= 128 && d <= 256 && aligned) {
        TRACE("elkan pass");
        CK(launch_fused<TY>(d, k, sms, s, aa, as<float>(st.drift), as<int32_t>(st.vstamp), cur,
                            as<double>(st.c64)));
        launches += 1;
      } else {
        TRACE("elkan scan");
        elkan_scan_kernel<<<sms * 8, 256, 0, s>>>(n, k, as<int32_t>(st.assign), as<int32_t>(st.vstamp),
                                                  as<float>(st.ub), as<float>(st.lbk),
                                                  as<float>(st.drift), as<int32_t>(st.work), counters);
        CK(cudaGetLastError());
        TRACE("elkan refine");
        CK(launch_refine<TY>(d, sms, s, aa, as<int32_t>(st.work), as<float>(st.drift),
                             as<int32_t>(st.vstamp), cur, as<double>(st.c64)));
        launches += 2;
      }
    }
    decided += rows;
    unsigned long long cnt[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(cnt, counters, 32, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const unsigned long long changed = cnt[0];
    res->near_ties += (int64_t)cnt[1];
    if (it > 1) rows = (int64_t)cnt[2];
    if (debug_on()) {
      fprintf(stderr, "[csc] kmeans pass %d: refined %lld flagged %llu moved %llu candidates %llu\n",
              it, (long long)rows, cnt[1], changed, cnt[3]);
      fflush(stderr);
    }
    converged = it > 1 && changed == 0;
    if (converged || it == max_iter) break;
    if (it == 1 || changed > (unsigned long long)(n / 16)) {
      CK(accumulate(as<int32_t>(st.assign)));
    } else {
      TRACE("move");
      move_kernel<TY><<<sms * 4, 256, 0, s>>>(y, ldy, n, d, as<int32_t>(st.moved), counters, scale,
                                              as<unsigned long long>(st.sums), as<int>(st.counts));
      CK(cudaGetLastError());
      ++launches;
    }
    CK(finalize());
    // cumulative movement per centroid (version it), for the lazy bounds
    CK(cudaMemcpyAsync(move_h.data(), st.cmove.ptr, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int j = 0; j < k; ++j)
      cum[(size_t)it * k + j] = cum[(size_t)(it - 1) * k + j] + (double)move_h[j];
  }
  if (!use_tc) {
    if (it > max_iter) it = max_iter;
    res->iters = it;
    res->converged = converged;
    res->decided = decided;
  }
  // inertia against the centroids the final assignment was computed with
  const int igrid = sms * 8;
  TRACE("inertia");
  if (vec8)
    inertia_vec_kernel<TY><<<igrid, 256, 0, s>>>(y, ldy, n, d, as<float>(st.c32), as<int32_t>(st.assign),
                                                as<double>(st.inertia_part));
  else
    inertia_kernel<TY><<<igrid, 256, 0, s>>>(y, ldy, n, d, as<float>(st.c32), as<int32_t>(st.assign),
                                              as<double>(st.inertia_part));
  CK(cudaGetLastError());
  CK(launch_reduce_partials(as<double>(st.inertia_part), 1, igrid, 1, 0,
                            as<double>(st.inertia_part) + igrid, s));
  launches += 2;
  double inertia = 0.0;
  CK(cudaMemcpyAsync(&inertia, as<double>(st.inertia_part) + igrid, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  res->inertia = inertia;
  res->assign = as<int32_t>(st.assign);
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
  DevBuf* all[] = {&st.c64, &st.c32, &st.cn2, &st.cmove, &st.bits, &st.sums, &st.counts,
                   &st.assign, &st.ub, &st.lbk, &st.work, &st.flagged, &st.moved, &st.counters,
                   &st.inertia_part, &st.init_idx, &st.vstamp, &st.drift};
  for (DevBuf* b : all) release(*b);
  release(st.perm);
  release(st.hist);
  if (st.hist_host) cudaFreeHost(st.hist_host);
  st.hist_host = nullptr;
  st.hist_cap = 0;
  for (cudaEvent_t& e : st.pass_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  kmeans_tc_release(st);
}

}  // namespace csc
