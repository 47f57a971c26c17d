// Chebyshev recursion on the shifted normalized Laplacian (Sections 2.2 and 3.3).
//
//   T_0 = R,  T_1 = L~ R,  T_{j+1} = 2 L~ T_j - T_{j-1},  L~ = -D^{-1/2} W D^{-1/2}
//   Psi~ = sum_j a_j T_j R                                     (filter output)
//   E_j = <T_j, T_j>,  F_j = <T_j, T_{j-1}>                     (float64 trace sums)
//
// so that mu_0 = E_0, mu_1 = F_1, mu_{2j} = 2 E_j - mu_0, mu_{2j-1} = 2 F_j - mu_1
// (from T_i T_j = (T_{i+j} + T_{|i-j|}) / 2) give every moment mu_l = tr(R^T T_l R),
// l <= 2m, and the eigencount of any cutoff without refiltering.
//
// One launch per step and column tile.  The tile is n x w float32 (w = 4 * LPR columns),
// row-major with leading dimension w, so a gathered row is 4*w contiguous bytes.
// A warp owns one row at a time; its 32 lanes form S = 32/LPR neighbour slots of LPR
// lanes, each lane holding 4 consecutive columns (one 16-byte load per neighbour), so a
// warp keeps S gathered rows in flight per iteration.  The S partial sums are folded with
// xor shuffles; the slot-0 lanes run the epilogue (recursion, Psi update, dot products).
// Rows are dealt round-robin to warps of a grid sized to fill every SM.
#include "csc_internal.h"

namespace csc {

namespace {

constexpr int kBlock = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 raw = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__device__ __forceinline__ void fma4(float4& acc, float s, float4 v) {
  acc.x = fmaf(s, v.x, acc.x);
  acc.y = fmaf(s, v.y, acc.y);
  acc.z = fmaf(s, v.z, acc.z);
  acc.w = fmaf(s, v.w, acc.w);
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ float4 shfl_xor4(float4 v, int off) {
  v.x += __shfl_xor_sync(kFull, v.x, off);
  v.y += __shfl_xor_sync(kFull, v.y, off);
  v.z += __shfl_xor_sync(kFull, v.z, off);
  v.w += __shfl_xor_sync(kFull, v.w, off);
  return v;
}

// sum_{p in row} w_p s_{col_p} T[col_p, 4 columns of this lane], folded over the S slots.
template <int LPR, typename TG>
__device__ __forceinline__ float4 gather_row(const StepArgs& a, const TG* __restrict__ tg,
                                             int64_t row, int slot, int sub) {
  constexpr int S = 32 / LPR;
  const int64_t beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
  const int w = a.w;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int64_t e = beg + slot;
  for (; e + S < end; e += 2 * S) {
    const int c0 = __ldg(a.col + e), c1 = __ldg(a.col + e + S);
    float s0 = __ldg(a.scale + c0), s1 = __ldg(a.scale + c1);
    if (a.val != nullptr) { s0 *= __ldg(a.val + e); s1 *= __ldg(a.val + e + S); }
    const float4 v0 = ld4(tg + (int64_t)c0 * w + sub * 4);
    const float4 v1 = ld4(tg + (int64_t)c1 * w + sub * 4);
    fma4(acc, s0, v0);
    fma4(acc, s1, v1);
  }
  if (e < end) {
    const int c0 = __ldg(a.col + e);
    float s0 = __ldg(a.scale + c0);
    if (a.val != nullptr) s0 *= __ldg(a.val + e);
    fma4(acc, s0, ld4(tg + (int64_t)c0 * w + sub * 4));
  }
#pragma unroll
  for (int off = LPR; off < 32; off <<= 1) acc = shfl_xor4(acc, off);
  return acc;
}

// Folds per-lane float partials over the LPR lanes of slot 0 and accumulates them in float64
// on lane 0.
template <int LPR>
__device__ __forceinline__ void fold_dot(float v, double& acc, int lane) {
#pragma unroll
  for (int off = 1; off < LPR; off <<= 1) v += __shfl_xor_sync(kFull, v, off);
  if (lane == 0) acc += (double)v;
}

template <int NQ>
__device__ __forceinline__ void block_store(double (&acc)[NQ], double* part) {
  __shared__ double red[NQ][kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][wid] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) s += red[threadIdx.x][i];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

template <int LPR, typename T0>
__global__ void __launch_bounds__(kBlock) cheb_first_kernel(StepArgs a) {
  const int lane = threadIdx.x & 31;
  const int slot = lane / LPR, sub = lane % LPR;
  const int64_t warp = (blockIdx.x * (int64_t)kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  const T0* __restrict__ t0 = static_cast<const T0*>(a.tg);
  const int w = a.w;
  float a0 = 0.f, a1 = 0.f;
  if (a.psi != nullptr) { a0 = __ldg(a.coef); a1 = __ldg(a.coef + 1); }
  double acc[3] = {0.0, 0.0, 0.0};  // <T0,T0>, <T1,T1>, <T1,T0>
  for (int64_t row = warp; row < a.n; row += nwarps) {
    const float4 g = gather_row<LPR, T0>(a, t0, row, slot, sub);
    const float si = -__ldg(a.scale + row);
    float e0 = 0.f, e1 = 0.f, f1 = 0.f;
    if (slot == 0) {
      const float4 t1 = make_float4(si * g.x, si * g.y, si * g.z, si * g.w);
      const float4 own = ld4(t0 + row * w + sub * 4);
      st4(a.tn + row * w + sub * 4, t1);
      if (a.psi != nullptr) {
        float4 p;
        p.x = fmaf(a1, t1.x, a0 * own.x);
        p.y = fmaf(a1, t1.y, a0 * own.y);
        p.z = fmaf(a1, t1.z, a0 * own.z);
        p.w = fmaf(a1, t1.w, a0 * own.w);
        st4(a.psi + row * a.ldp + sub * 4, p);
      }
      e0 = dot4(own, own);
      e1 = dot4(t1, t1);
      f1 = dot4(t1, own);
    }
    fold_dot<LPR>(e0, acc[0], lane);
    fold_dot<LPR>(e1, acc[1], lane);
    fold_dot<LPR>(f1, acc[2], lane);
  }
  block_store<3>(acc, a.part);
}

template <int LPR, typename TP>
__global__ void __launch_bounds__(kBlock) cheb_step_kernel(StepArgs a) {
  const int lane = threadIdx.x & 31;
  const int slot = lane / LPR, sub = lane % LPR;
  const int64_t warp = (blockIdx.x * (int64_t)kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  const float* __restrict__ tg = static_cast<const float*>(a.tg);
  const TP* __restrict__ tp = static_cast<const TP*>(a.tp);
  const int w = a.w;
  const float aj = a.psi != nullptr ? __ldg(a.coef + a.j + 1) : 0.f;
  double acc[2] = {0.0, 0.0};  // <T_{j+1},T_{j+1}>, <T_{j+1},T_j>
  for (int64_t row = warp; row < a.n; row += nwarps) {
    const float4 g = gather_row<LPR, float>(a, tg, row, slot, sub);
    const float si2 = -2.0f * __ldg(a.scale + row);
    float e = 0.f, f = 0.f;
    if (slot == 0) {
      const float4 prev = ld4(tp + row * w + sub * 4);
      const float4 own = ld4(tg + row * w + sub * 4);
      float4 t;
      t.x = fmaf(si2, g.x, -prev.x);
      t.y = fmaf(si2, g.y, -prev.y);
      t.z = fmaf(si2, g.z, -prev.z);
      t.w = fmaf(si2, g.w, -prev.w);
      st4(a.tn + row * w + sub * 4, t);
      if (a.psi != nullptr) {
        float* pp = a.psi + row * a.ldp + sub * 4;
        float4 p = ld4(pp);
        p.x = fmaf(aj, t.x, p.x);
        p.y = fmaf(aj, t.y, p.y);
        p.z = fmaf(aj, t.z, p.z);
        p.w = fmaf(aj, t.w, p.w);
        st4(pp, p);
      }
      e = dot4(t, t);
      f = dot4(t, own);
    }
    fold_dot<LPR>(e, acc[0], lane);
    fold_dot<LPR>(f, acc[1], lane);
  }
  block_store<2>(acc, a.part);
}

template <typename T0>
const void* first_kernel_for(int lpr) {
  switch (lpr) {
    case 2: return (const void*)cheb_first_kernel<2, T0>;
    case 4: return (const void*)cheb_first_kernel<4, T0>;
    case 8: return (const void*)cheb_first_kernel<8, T0>;
    case 16: return (const void*)cheb_first_kernel<16, T0>;
    case 32: return (const void*)cheb_first_kernel<32, T0>;
  }
  return nullptr;
}

template <typename TP>
const void* step_kernel_for(int lpr) {
  switch (lpr) {
    case 2: return (const void*)cheb_step_kernel<2, TP>;
    case 4: return (const void*)cheb_step_kernel<4, TP>;
    case 8: return (const void*)cheb_step_kernel<8, TP>;
    case 16: return (const void*)cheb_step_kernel<16, TP>;
    case 32: return (const void*)cheb_step_kernel<32, TP>;
  }
  return nullptr;
}

cudaError_t launch_any(const void* fn, const StepArgs& a, int grid, cudaStream_t s) {
  if (fn == nullptr) return cudaErrorInvalidValue;
  StepArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, 0, s);
}

// Fixed-order reduction of block partials: one block per output row.
__global__ void reduce_partials_kernel(const double* __restrict__ part, int grid, int tiles,
                                       int64_t tile_stride, double* __restrict__ out) {
  __shared__ double red[256];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int t = 0; t < tiles; ++t) {
    const double* p = part + t * tile_stride + (int64_t)r * grid;
    for (int b = threadIdx.x; b < grid; b += blockDim.x) s += p[b];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = red[0];
}

}  // namespace

int cheb_grid(int w) {
  (void)w;
  static int grid = 0;
  if (grid == 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_step_kernel<4, float>, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * num_sms();
  }
  return grid;
}

cudaError_t launch_cheb_first(const StepArgs& a, int t0_dtype, int grid, cudaStream_t s) {
  const int lpr = a.w / 4;
  const void* fn = t0_dtype == CSC_BF16 ? first_kernel_for<__nv_bfloat16>(lpr)
                                        : first_kernel_for<float>(lpr);
  return launch_any(fn, a, grid, s);
}

cudaError_t launch_cheb_step(const StepArgs& a, int tp_dtype, int grid, cudaStream_t s) {
  const int lpr = a.w / 4;
  const void* fn = tp_dtype == CSC_BF16 ? step_kernel_for<__nv_bfloat16>(lpr)
                                        : step_kernel_for<float>(lpr);
  return launch_any(fn, a, grid, s);
}

cudaError_t launch_reduce_partials(const double* part, int nrows, int grid, int tiles,
                                   int64_t tile_stride, double* out, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  reduce_partials_kernel<<<nrows, 256, 0, s>>>(part, grid, tiles, tile_stride, out);
  return cudaGetLastError();
}

}  // namespace csc
