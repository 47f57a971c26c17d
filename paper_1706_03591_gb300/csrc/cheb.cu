// Chebyshev recursion on the shifted normalized Laplacian (Sections 2.2 and 3.3).
//
//   T_0 = R,  T_1 = L~ R,  T_{j+1} = 2 L~ T_j - T_{j-1},  L~ = -D^{-1/2} W D^{-1/2}
//   Psi~ = sum_j a_j T_j R                                     (filter output)
//   E_j = <T_j, T_j>,  F_j = <T_j, T_{j-1}>                     (float64 trace sums)
//
// Value-free form: the blocks are stored as V_j = S T_j (S = D^{-1/2}, 1 on isolated rows), so
// V_{j+1} = -2 S^2 W V_j - V_{j-1}: a step gathers plain rows of V_j and needs only the edge
// weights (none for unit weights), not D^{-1/2} of every neighbour.  Psi and the trace sums use
// T = V / S.  The first step gathers T_0 = R with the weights w_e D^{-1/2}[col_e].
//
// so that mu_0 = E_0, mu_1 = F_1, mu_{2j} = 2 E_j - mu_0, mu_{2j-1} = 2 F_j - mu_1
// (from T_i T_j = (T_{i+j} + T_{|i-j|}) / 2) give every moment mu_l = tr(R^T T_l R),
// l <= 2m, and the eigencount of any cutoff without refiltering.
//
// One launch per step and column tile.  The tile is n x w float32 (w = 4 * LPR columns),
// row-major with leading dimension w, so a gathered row is 4*w contiguous bytes.
// The rows are cut into blocks of about kEdgesPerBlock stored edges.  A CTA stages a
// block's row offsets, column indices and edge weights w_e D^{-1/2}[col] in shared memory
// with coalesced loads, so the gathers that follow depend on shared memory only.  A warp
// then owns one row at a time: its 32 lanes form S = 32/LPR neighbour slots of LPR lanes,
// each lane holding 4 consecutive columns (one 16-byte load per neighbour, four in
// flight per lane), and the slot partials are folded with xor shuffles.  The own-row
// operands (T_{j-1}, T_j, Psi) are loaded before the gather; the slot-0 lanes run the
// epilogue (recursion, Psi update, dot products).  CTAs stride over the blocks of a grid
// sized to fill every SM.
#include <type_traits>

#include "csc_internal.h"
#include "philox.cuh"

namespace csc {

namespace {

constexpr int kBlock = 256;
constexpr unsigned kFull = 0xffffffffu;

// Loads of the recursion blocks and of Psi bypass L1 (cache at L2 only): a block written by
// one step is read by other SMs in the next, and within a persistent launch L1 is not coherent.
__device__ __forceinline__ float4 ld4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 raw = __ldcg(reinterpret_cast<const uint2*>(p));
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// L2 eviction priorities: rows gathered from T_j are kept (evict_last) against the streams
// that pass through once per step (T_{j-1}, Psi), which are marked evict_first.
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld4h(const float* ptr, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ float4 ld4h(const __nv_bfloat16* ptr, uint64_t pol) {
  uint32_t x, y;
  asm volatile("ld.global.cg.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(x), "=r"(y)
               : "l"(ptr), "l"(pol));
  const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x));
  const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&y));
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void st4h(float* ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}

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

constexpr int kStageUnroll = 4;

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

// ------------------------------------------------------------------ standalone step kernels
//
// One launch per step and column tile.  The rows are cut into blocks of about kBlockWeight
// units, a row weighing its stored edges plus kRowCost (g.srow, built at set_graph), so that
// every block carries about the same gather and stream work whatever the degree distribution.
// A CTA walks its blocks in chunks: one coalesced load of the row offsets (one per thread) finds
// the longest run of rows whose edges fit the shared-memory buffer, and their column indices
// and edge weights are staged there.  Each row of a chunk is reduced by spr slots of LPR lanes
// (spr the smallest power of two with 64 spr >= the chunk's largest degree, so that a long row
// spreads over up to a whole warp while short rows keep one slot each); the slots stride over the row's
// edges with kRowUnroll 16-byte loads in flight per lane and are folded with xor shuffles in a
// fixed order.  A row too long for the buffer on its own (a hub) is reduced by the whole CTA
// straight from global memory: every slot of every warp strides over its edges, the warps
// fold their slots, and the first warp adds the warp sums in warp order.  The gathered block
// T_j is read-only during a launch, so its rows are loaded through the non-coherent L1 path,
// which keeps hub rows that many rows share in L1.

constexpr int kChunkRows = kBlock - 1;  // at most one row offset per thread
constexpr int kChunkEdges = 5632;       // staged columns and weights: 45 KB
constexpr int kEdgesPerSlot = 64;       // spr: smallest power of two with spr * 64 >= max degree
constexpr int kRowUnroll = 8;           // 16-byte gathers in flight per lane

struct StageChunk {
  union {
    struct {
      int col[kChunkEdges];
      float wt[kChunkEdges];
    } e;
    float4 red[kBlock / 32][32];  // cooperative rows: the warps' partial sums
  } u;
  int rp[kChunkRows + 1];
  int64_t base;
  int maxdeg;
};

// Loads of gathered and own rows: through L1 (ld.global.nc) in the standalone step kernels, where
// the blocks are read-only for the launch; at L2 only (ld.global.cg) in the persistent batched
// kernel, whose blocks are written by other CTAs of the same launch.
template <bool CG, typename T>
__device__ __forceinline__ float4 ldr(const T* ptr);

// Gathered-row loads through L1 (ld.global.nc).
__device__ __forceinline__ float4 ldg_row(const float* ptr) { return __ldg(reinterpret_cast<const float4*>(ptr)); }
__device__ __forceinline__ float4 ldg_row(const __nv_bfloat16* ptr) {
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(ptr));
  const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
  const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <bool CG, typename T>
__device__ __forceinline__ float4 ldr(const T* ptr) {
  if constexpr (CG) return ld4(ptr);
  else return ldg_row(ptr);
}

// Stages the longest run of rows [r, r + rows) of a block ending at re whose edges fit the
// buffer (at most kChunkRows rows): row offsets relative to st.base, the largest degree, the
// column indices and the edge weights (w_e, times D^-1/2[col_e] when SCALED).  Returns rows;
// 0 when row r alone exceeds the buffer.  Block-uniform; starts with a barrier that protects
// the previous chunk's shared data.
template <bool SCALED>
__device__ __forceinline__ int stage_chunk(const StepArgs& a, StageChunk& st, int r, int re) {
  const int lim = min(kChunkRows, re - r);
  const bool have = (int)threadIdx.x <= lim;
  int64_t off = 0;
  __syncthreads();
  if (have) off = __ldg(a.row_ptr + r + threadIdx.x);
  if (threadIdx.x == 0) {
    st.base = off;
    st.maxdeg = 0;
  }
  __syncthreads();
  const int64_t base = st.base;
  // row_ptr is non-decreasing, so the offsets that fit form a prefix
  const int cnt = __syncthreads_count(have && off - base <= kChunkEdges);
  const int rows = cnt - 1;
  if (rows == 0) return 0;
  if ((int)threadIdx.x < cnt) st.rp[threadIdx.x] = (int)(off - base);
  __syncthreads();
  const int ne = st.rp[rows];
  int deg = (int)threadIdx.x < rows ? st.rp[threadIdx.x + 1] - st.rp[threadIdx.x] : 0;
  deg = __reduce_max_sync(kFull, deg);
  if ((threadIdx.x & 31) == 0 && deg > 0) atomicMax(&st.maxdeg, deg);
  const bool weighted = a.val != nullptr;
  for (int b0 = 0; b0 < ne; b0 += kStageUnroll * kBlock) {
    int c[kStageUnroll];
    float v[kStageUnroll];
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u) {
      const int e = b0 + u * kBlock + threadIdx.x;
      c[u] = e < ne ? __ldcs(a.col + base + e) : 0;
      v[u] = (e < ne && weighted) ? __ldcs(a.val + base + e) : 1.0f;
      if (SCALED && e < ne) v[u] *= __ldg(a.scale + c[u]);
    }
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u) {
      const int e = b0 + u * kBlock + threadIdx.x;
      if (e < ne) {
        st.u.e.col[e] = c[u];
        if (SCALED || weighted) st.u.e.wt[e] = v[u];
      }
    }
  }
  __syncthreads();
  return rows;
}

// Epilogue of one row (the LPR lanes of its first slot, 4 columns each): FIRST: T_1 = -S^2... in
// the stored form V_1 = vs T_1 with T_1 = -D^-1/2 g, Psi = a_0 T_0 + a_1 T_1, dots <T0,T0>,
// <T1,T1>, <T1,T0>; else V_{j+1} = -2 vs^2 g - V_{j-1}, Psi += a_{j+1} T_{j+1}, dots
// <T_{j+1},T_{j+1}>, <T_{j+1},T_j>.  own: T_0 (FIRST) or V_j; prev: V_{j-1} (T_0 when
// tp_unscaled); p: the Psi row.
template <bool FIRST>
__device__ __forceinline__ void row_epilogue(const StepArgs& a, int64_t row, int sub, float4 g, float4 own,
                                             float4 prev, float4 p, float c0, float c1, float sc, float vsi,
                                             float ivsi, float (&dots)[3]) {
  const int w = a.w;
  if constexpr (FIRST) {
    const float4 t1 = make_float4(sc * g.x, sc * g.y, sc * g.z, sc * g.w);
    st4(a.tn + row * w + sub * 4, make_float4(vsi * t1.x, vsi * t1.y, vsi * t1.z, vsi * t1.w));
    if (a.psi != nullptr) {
      float4 q;
      q.x = fmaf(c1, t1.x, c0 * own.x);
      q.y = fmaf(c1, t1.y, c0 * own.y);
      q.z = fmaf(c1, t1.z, c0 * own.z);
      q.w = fmaf(c1, t1.w, c0 * own.w);
      st4(a.psi + row * a.ldp + sub * 4, q);
    }
    dots[0] = dot4(own, own);
    dots[1] = dot4(t1, t1);
    dots[2] = dot4(t1, own);
  } else {
    const float c2 = -2.0f * vsi * vsi;
    if (a.tp_unscaled) { prev.x *= vsi; prev.y *= vsi; prev.z *= vsi; prev.w *= vsi; }
    float4 v;
    v.x = fmaf(c2, g.x, -prev.x);
    v.y = fmaf(c2, g.y, -prev.y);
    v.z = fmaf(c2, g.z, -prev.z);
    v.w = fmaf(c2, g.w, -prev.w);
    st4(a.tn + row * w + sub * 4, v);
    const float4 t = make_float4(v.x * ivsi, v.y * ivsi, v.z * ivsi, v.w * ivsi);
    const float4 tc = make_float4(own.x * ivsi, own.y * ivsi, own.z * ivsi, own.w * ivsi);
    if (a.psi != nullptr) {
      p.x = fmaf(c1, t.x, p.x);
      p.y = fmaf(c1, t.y, p.y);
      p.z = fmaf(c1, t.z, p.z);
      p.w = fmaf(c1, t.w, p.w);
      st4h(a.psi + row * a.ldp + sub * 4, p, l2_stream());
    }
    dots[0] = dot4(t, t);
    dots[1] = dot4(t, tc);
    dots[2] = 0.f;
  }
}

// Own-row operands of a row, issued before its gather.
template <bool FIRST, typename TG, typename TP, bool CG = false>
__device__ __forceinline__ void row_operands(const StepArgs& a, int64_t row, int sub, float4& own,
                                             float4& prev, float4& p, float& sc, float& vsi, float& ivsi) {
  const uint64_t stream = l2_stream();
  const int w = a.w;
  vsi = __ldg(a.vs + row);
  if constexpr (FIRST) {
    own = ldr<CG>(static_cast<const TG*>(a.tg) + row * w + sub * 4);
    sc = -__ldg(a.scale + row);
  } else {
    ivsi = __ldg(a.ivs + row);
    prev = ld4h(static_cast<const TP*>(a.tp) + row * w + sub * 4, stream);
    own = ldr<CG>(static_cast<const float*>(a.tg) + row * w + sub * 4);
    if (a.psi != nullptr) p = ld4h(a.psi + row * a.ldp + sub * 4, stream);
  }
}

// Rows [r, r + rows) of a staged chunk; dot partials into acc (lane 0 of each row's lead slot).
template <int LPR, bool FIRST, typename TG, typename TP, bool CG = false>
__device__ __forceinline__ void process_chunk(const StepArgs& a, const StageChunk& st, int r, int rows,
                                              float c0, float c1, double (&acc)[FIRST ? 3 : 2]) {
  constexpr int S = 32 / LPR;
  constexpr int kLines = LPR >= 8 ? LPR / 8 : 1;  // 128-byte lines per gathered row (float)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = lane / LPR, sub = lane % LPR;
  int spr = 1;
  while (spr < S && spr * kEdgesPerSlot < st.maxdeg) spr <<= 1;
  const int rpw = S / spr;
  const int rpp = (kBlock / 32) * rpw;
  const int q = slot % spr;
  const int rw = slot / spr;
  const TG* __restrict__ base = static_cast<const TG*>(a.tg) + sub * 4;
  const int w = a.w;
  const bool scaled = FIRST || a.val != nullptr;
  for (int p0 = 0; p0 < rows; p0 += rpp) {
    const int rl = p0 + wid * rpw + rw;
    const bool valid = rl < rows;
    const bool lead = valid && q == 0;
    const int64_t row = (int64_t)r + (valid ? rl : 0);
    float4 own = make_float4(0.f, 0.f, 0.f, 0.f), prev = own, p = own;
    float sc = 0.f, vsi = 1.f, ivsi = 1.f;
    if (lead) row_operands<FIRST, TG, TP, CG>(a, row, sub, own, prev, p, sc, vsi, ivsi);
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      const int beg = st.rp[rl], end = st.rp[rl + 1];
      for (int e0 = beg + q; e0 < end; e0 += kRowUnroll * spr) {
        if (!FIRST && a.l2pf) {
          // the next batch's rows into L2 while this batch loads (pays off when the gathered
          // block exceeds the L2)
          for (int qq = sub; qq < kRowUnroll * kLines; qq += LPR) {
            const int ep = e0 + (kRowUnroll + qq / kLines) * spr;
            if (ep < end)
              asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(
                  static_cast<const float*>(a.tg) + (int64_t)st.u.e.col[ep] * w + (qq % kLines) * 32)
                           : "memory");
          }
        }
        float4 v[kRowUnroll];
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
          const int e = e0 + u * spr;
          v[u] = e < end ? ldr<CG>(base + (int64_t)st.u.e.col[e] * w) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (scaled) {
#pragma unroll
          for (int u = 0; u < kRowUnroll; ++u)
            if (e0 + u * spr < end) fma4(g, st.u.e.wt[e0 + u * spr], v[u]);
        } else {
#pragma unroll
          for (int u = 0; u < kRowUnroll; ++u) {
            g.x += v[u].x; g.y += v[u].y; g.z += v[u].z; g.w += v[u].w;
          }
        }
      }
    }
    for (int off = LPR; off < LPR * spr; off <<= 1) g = shfl_xor4(g, off);
    float dots[3] = {0.f, 0.f, 0.f};
    if (lead) row_epilogue<FIRST>(a, row, sub, g, own, prev, p, c0, c1, sc, vsi, ivsi, dots);
#pragma unroll
    for (int k = 0; k < (FIRST ? 3 : 2); ++k)
#pragma unroll
      for (int off = 1; off < LPR; off <<= 1) dots[k] += __shfl_xor_sync(kFull, dots[k], off);
    if (lead && sub == 0) {
      acc[0] += (double)dots[0];
      acc[1] += (double)dots[1];
      if constexpr (FIRST) acc[FIRST ? 2 : 0] += (double)dots[2];
    }
  }
}

// A row too long to stage, reduced by the whole CTA from global memory.
template <int LPR, bool FIRST, typename TG, typename TP, bool CG = false>
__device__ __forceinline__ void coop_row(const StepArgs& a, StageChunk& st, int64_t row, float c0, float c1,
                                         double (&acc)[FIRST ? 3 : 2]) {
  constexpr int S = 32 / LPR;
  constexpr int TS = (kBlock / 32) * S;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = lane / LPR, sub = lane % LPR;
  const int gs = wid * S + slot;
  const bool lead = threadIdx.x < LPR;
  float4 own = make_float4(0.f, 0.f, 0.f, 0.f), prev = own, p = own;
  float sc = 0.f, vsi = 1.f, ivsi = 1.f;
  if (lead) row_operands<FIRST, TG, TP, CG>(a, row, sub, own, prev, p, sc, vsi, ivsi);
  const TG* __restrict__ base = static_cast<const TG*>(a.tg) + sub * 4;
  const int w = a.w;
  const int64_t beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t e0 = beg + gs; e0 < end; e0 += (int64_t)kRowUnroll * TS) {
    int c[kRowUnroll];
    float wt[kRowUnroll];
#pragma unroll
    for (int u = 0; u < kRowUnroll; ++u) {
      const int64_t e = e0 + (int64_t)u * TS;
      c[u] = e < end ? __ldcs(a.col + e) : 0;
      wt[u] = e < end ? (a.val != nullptr ? __ldcs(a.val + e) : 1.0f) : 0.0f;
    }
    if (FIRST) {
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) wt[u] *= __ldg(a.scale + c[u]);
    }
    float4 v[kRowUnroll];
#pragma unroll
    for (int u = 0; u < kRowUnroll; ++u)
      v[u] = e0 + (int64_t)u * TS < end ? ldr<CG>(base + (int64_t)c[u] * w) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kRowUnroll; ++u) fma4(g, wt[u], v[u]);
  }
#pragma unroll
  for (int off = LPR; off < 32; off <<= 1) g = shfl_xor4(g, off);
  __syncthreads();  // the warp sums alias the previous chunk's staged edges
  if (slot == 0) st.u.red[wid][sub] = g;
  __syncthreads();
  if (wid == 0) {
    float4 tot = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lead) {
      for (int k = 0; k < kBlock / 32; ++k) {
        const float4 h = st.u.red[k][sub];
        tot.x += h.x; tot.y += h.y; tot.z += h.z; tot.w += h.w;
      }
    }
    float dots[3] = {0.f, 0.f, 0.f};
    if (lead) row_epilogue<FIRST>(a, row, sub, tot, own, prev, p, c0, c1, sc, vsi, ivsi, dots);
#pragma unroll
    for (int k = 0; k < (FIRST ? 3 : 2); ++k)
#pragma unroll
      for (int off = 1; off < LPR; off <<= 1) dots[k] += __shfl_xor_sync(kFull, dots[k], off);
    if (threadIdx.x == 0) {
      acc[0] += (double)dots[0];
      acc[1] += (double)dots[1];
      if constexpr (FIRST) acc[FIRST ? 2 : 0] += (double)dots[2];
    }
  }
}

// Rows [r, re) in chunks: staged chunks row by row, a row too long to stage by the whole CTA.
template <int LPR, bool FIRST, typename TG, typename TP, bool CG>
__device__ __forceinline__ void rows_range(const StepArgs& a, StageChunk& st, int r, int re, float c0, float c1,
                                           double (&acc)[FIRST ? 3 : 2]) {
  while (r < re) {
    const int rows = stage_chunk<FIRST>(a, st, r, re);
    if (rows == 0) {
      coop_row<LPR, FIRST, TG, TP, CG>(a, st, r, c0, c1, acc);
      r += 1;
    } else {
      process_chunk<LPR, FIRST, TG, TP, CG>(a, st, r, rows, c0, c1, acc);
      r += rows;
    }
  }
}

// FIRST: T_1 = L~ T_0 (stored as V_1 = vs T_1), Psi = a_0 T_0 + a_1 T_1, partials <T0,T0>,
// <T1,T1>, <T1,T0> (TG: storage type of T_0).  Else one general step (TP: storage type of
// T_{j-1}), partials <T_{j+1},T_{j+1}>, <T_{j+1},T_j>.  Three CTAs per SM (at most 85 registers
// per thread): at four (64 registers) the gather batch and the own-row operands spilled, and
// the spill traffic cost more than the extra warps gained.
template <int LPR, bool FIRST, typename TG, typename TP>
__global__ void __launch_bounds__(kBlock, 3) cheb_rows_kernel(StepArgs a) {
  constexpr int NQ = FIRST ? 3 : 2;
  __shared__ StageChunk st;
  double acc[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) acc[k] = 0.0;
  float c0 = 0.f, c1 = 0.f;
  if (a.psi != nullptr) {
    if (FIRST) {
      c0 = __ldg(a.coef);
      c1 = __ldg(a.coef + 1);
    } else {
      c1 = __ldg(a.coef + a.j + 1);
    }
  }
  for (int b = blockIdx.x; b < a.nsblk; b += gridDim.x)
    rows_range<LPR, FIRST, TG, TP, false>(a, st, __ldg(a.srow + b), __ldg(a.srow + b + 1), c0, c1, acc);
  // every lane may hold a partial: reduce the warp first
#pragma unroll
  for (int k = 0; k < NQ; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(kFull, acc[k], off);
  block_store<NQ>(acc, a.part);
}

// ------------------------------------------------------------------ batched filtering

template <int NQ>
__device__ __forceinline__ void block_atomic(double (&acc)[NQ], double* dst) {
  __shared__ double red[NQ][kBlock / 32];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][wid] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) v += red[threadIdx.x][i];
    atomicAdd(dst + threadIdx.x, v);
  }
}

template <int LPR>
__device__ void batched_signals(const BatchTile& t, int b) {
  if (b >= t.a.nsblk) return;
  const int rs = __ldg(t.a.srow + b), re = __ldg(t.a.srow + b + 1);
  const int w = t.a.w;
  const uint32_t k0 = (uint32_t)t.seed, k1 = (uint32_t)(t.seed >> 32);
  for (int e = threadIdx.x; e < (re - rs) * w; e += blockDim.x) {
    const int64_t row = rs + e / w;
    const int v = e % w;
    float val = 0.0f;
    if (v < t.valid) val = gauss_signal((uint64_t)row, (uint64_t)(t.col0 + v), k0, k1) * t.inv_sqrt_d;
    if (t.t0_dtype == CSC_BF16)
      static_cast<__nv_bfloat16*>(t.buf[0])[row * w + v] = __float2bfloat16_rn(val);
    else
      static_cast<float*>(t.buf[0])[row * w + v] = val;
  }
}

// One item of the persistent batched kernel: row block b of a tile at step s (s = 1: the first
// step), through the same chunked rows as the standalone step kernels, with coherent (L2) loads:
// the blocks a step gathers were written by other CTAs of the same launch.
template <int LPR>
__device__ void batched_item(const BatchTile& t, StageChunk& st, int b, int s) {
  StepArgs a = t.a;
  if (b >= a.nsblk) return;
  const int rs = __ldg(a.srow + b), re = __ldg(a.srow + b + 1);
  if (s == 1) {
    a.tg = t.buf[0];
    a.tn = static_cast<float*>(t.buf[1]);
    a.j = 0;
    double acc[3] = {0.0, 0.0, 0.0};
    const float c0 = a.psi != nullptr ? __ldg(a.coef) : 0.f, c1 = a.psi != nullptr ? __ldg(a.coef + 1) : 0.f;
    if (t.t0_dtype == CSC_BF16) rows_range<LPR, true, __nv_bfloat16, float, true>(a, st, rs, re, c0, c1, acc);
    else rows_range<LPR, true, float, float, true>(a, st, rs, re, c0, c1, acc);
    // first-step rows of the E/F table: E0, E1, F1
    block_atomic<3>(acc, t.mom);
  } else {
    const int j = s - 1;  // produces T_{j+1}
    a.tg = t.buf[j % 3];
    a.tp = t.buf[(j - 1) % 3];
    a.tn = static_cast<float*>(t.buf[(j + 1) % 3]);
    a.j = j;
    a.tp_unscaled = j == 1;
    double acc[2] = {0.0, 0.0};
    const float c1 = a.psi != nullptr ? __ldg(a.coef + j + 1) : 0.f;
    if (j == 1 && t.t0_dtype == CSC_BF16)
      rows_range<LPR, false, float, __nv_bfloat16, true>(a, st, rs, re, 0.f, c1, acc);
    else
      rows_range<LPR, false, float, float, true>(a, st, rs, re, 0.f, c1, acc);
    block_atomic<2>(acc, t.mom + 2 * (j + 1) - 1);
  }
}

// Dataflow schedule.  Work items are claimed from one counter in (wave, step, item) order;
// waves keep the working set of the tiles in flight near the L2 size.  Step s of a tile reads
// that tile's blocks of steps s - 1 and s - 2 and overwrites the one of step s - 3, so an item
// of step s waits (bounded) until every item of step s - 1 of its own tile is done; no grid
// barrier is needed, fast tiles run ahead, and the next wave starts while the last steps of
// the current one finish.  A claimed item only waits on items with smaller claim numbers, and
// all blocks are co-resident (cooperative launch), so the schedule cannot deadlock.
__global__ void __launch_bounds__(kBlock, 3) cheb_batched_kernel(const BatchTile* __restrict__ tiles,
                                                                 const int32_t* __restrict__ item_tile,
                                                                 const int64_t* __restrict__ wave_end,
                                                                 const int64_t* __restrict__ claim_end,
                                                                 int nwaves, int m,
                                                                 unsigned long long* work,
                                                                 unsigned int* done, int* err) {
  __shared__ StageChunk st;
  __shared__ int64_t claim;
  __shared__ int ready;
  const int64_t total = claim_end[nwaves - 1];
  for (;;) {
    __syncthreads();  // every thread has read the previous claim
    if (threadIdx.x == 0) claim = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t q = claim;
    if (q >= total) break;
    int wv = 0;
    while (claim_end[wv] <= q) ++wv;
    const int64_t c0 = wv > 0 ? claim_end[wv - 1] : 0, w0 = wv > 0 ? wave_end[wv - 1] : 0;
    const int64_t items = wave_end[wv] - w0;
    const int s = (int)((q - c0) / items);
    const int64_t it = w0 + (q - c0) % items;
    const int ti = __ldg(item_tile + it);
    const BatchTile& t = tiles[ti];
    const int b = (int)(it - t.blk0);
    if (s >= 1) {
      if (threadIdx.x == 0) {
        volatile unsigned int* dep = done + (size_t)ti * (m + 1) + (s - 1);
        long long spins = 0;
        int ok = 1;
        while (*dep < (unsigned int)t.a.nsblk) {
          if (++spins > (1ll << 23) || *(volatile int*)err != 0) {
            atomicExch(err, 1);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
        ready = ok;
      }
      __syncthreads();
      if (!ready) return;
    }
    if (s == 0) {
      switch (t.lpr) {
        case 2: batched_signals<2>(t, b); break;
        case 4: batched_signals<4>(t, b); break;
        case 8: batched_signals<8>(t, b); break;
        default: batched_signals<16>(t, b); break;
      }
    } else {
      switch (t.lpr) {
        case 4: batched_item<4>(t, st, b, s); break;
        case 8: batched_item<8>(t, st, b, s); break;
        default: batched_item<16>(t, st, b, s); break;
      }
    }
    __threadfence();  // this item's blocks are visible before it is counted
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(done + (size_t)ti * (m + 1) + s, 1u);
  }
}

template <bool FIRST, typename TG, typename TP>
const void* rows_kernel_for(int lpr) {
  switch (lpr) {
    case 2: return (const void*)cheb_rows_kernel<2, FIRST, TG, TP>;
    case 4: return (const void*)cheb_rows_kernel<4, FIRST, TG, TP>;
    case 8: return (const void*)cheb_rows_kernel<8, FIRST, TG, TP>;
    case 16: return (const void*)cheb_rows_kernel<16, FIRST, TG, TP>;
    case 32: return (const void*)cheb_rows_kernel<32, FIRST, TG, TP>;
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_rows_kernel<4, false, float, float>, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * num_sms();
  }
  return grid;
}

cudaError_t launch_cheb_first(const StepArgs& a, int t0_dtype, int grid, cudaStream_t s) {
  const int lpr = a.w / 4;
  const void* fn = t0_dtype == CSC_BF16 ? rows_kernel_for<true, __nv_bfloat16, float>(lpr)
                                        : rows_kernel_for<true, float, float>(lpr);
  return launch_any(fn, a, grid, s);
}

cudaError_t launch_cheb_step(const StepArgs& a, int tp_dtype, int grid, cudaStream_t s) {
  const int lpr = a.w / 4;
  StepArgs b = a;
  b.l2pf = (double)a.n * a.w * 4.0 > 64.0 * (1 << 20);
  const void* fn = tp_dtype == CSC_BF16 ? rows_kernel_for<false, float, __nv_bfloat16>(lpr)
                                        : rows_kernel_for<false, float, float>(lpr);
  return launch_any(fn, b, grid, s);
}

int cheb_batched_grid() {
  static int grid = 0;
  if (grid == 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_batched_kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * num_sms();
  }
  return grid;
}

cudaError_t launch_cheb_batched(const BatchTile* tiles, const int32_t* item_tile, const int64_t* wave_end,
                                const int64_t* claim_end, int nwaves, int m, unsigned long long* work,
                                unsigned int* done, int* err, int grid, cudaStream_t s) {
  void* args[] = {(void*)&tiles, (void*)&item_tile, (void*)&wave_end, (void*)&claim_end, (void*)&nwaves,
                  (void*)&m, (void*)&work, (void*)&done, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)cheb_batched_kernel, dim3(grid), dim3(kBlock), args,
                                     0, s);
}

cudaError_t launch_reduce_partials(const double* part, int nrows, int grid, int tiles,
                                   int64_t tile_stride, double* out, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  reduce_partials_kernel<<<nrows, 256, 0, s>>>(part, grid, tiles, tile_stride, out);
  return cudaGetLastError();
}

}  // namespace csc
