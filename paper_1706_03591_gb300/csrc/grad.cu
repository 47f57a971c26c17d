// Differentiation through the Chebyshev filter (csc_filter_forward, csc_filter_vjp,
// csc_kmeans_loss_grad).  The paper has no derivative; this grows its filter (Section 2.2
// features Psi = sum_j a_j T_j(L~) R, Section 3.3 coefficients, Section 2.1 normalized
// Laplacian L~ = -D^-1/2 W D^-1/2) into a differentiable layer.
//
// Adjoint of the recursion (L~ symmetric), G = dloss/dPsi:
//     Lambda_m = a_m G,  Lambda_j = a_j G + 2 L~ Lambda_{j+1} - Lambda_{j+2}  (j >= 1),
//     dloss/da_j = <G, T_j R>,
//     dloss/dL~_uv = <Lambda_1[u], T_0 R[v]> + 2 sum_{j>=1} <Lambda_{j+1}[u], T_j R[v]>.
// In the value-free variables of the forward kernels (V_j = vs T_j R, vs = D^-1/2, 1 for an
// isolated node) the adjoint is Phi_j = vs Lambda_j:
//     Phi_j = a_j vs G - 2 vs^2 (W Phi_{j+1}) - Phi_{j+2},
// the same sparse product as a forward step plus a source term, and with
//     H_uv = sum_j c_j <Phi_{j+1}[u], V_j[v]>   (c_0 = 1, c_j = 2; V_0 = vs R)
// one has dloss/dL~_uv = H_uv / (vs_u vs_v).  Through l~_uv = -w_uv / sqrt(d_u d_v) and the
// degrees d_u = sum_v w_uv, for a symmetric weight w_e stored at (u, v) and (v, u):
//     dloss/dw_e = -(H_uv + H_vu) - s_u / (2 d_u) - s_v / (2 d_v),
//     s_u = -sum_{b in row u} w_ub (H_ub + H_bu).
// The forward pass keeps the pair (V_{ks-1}, V_{ks}) for every segment k of `stride` steps;
// the backward pass walks the segments in reverse, recomputes each from its pair, and runs
// one fused kernel per step: the adjoint step, the per-edge update of H (gathering V_j and
// Phi_{j+1} of the neighbours) and the partial sums of <G, T_j R>.  With stride 1 the forward
// pass writes every V_j straight into its checkpoint slot and the backward pass reads them
// there: nothing is copied or recomputed.
#include <algorithm>
#include <cmath>

#include "csc_internal.h"

namespace csc {
namespace {

constexpr int kBlk = 256;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kEdgeUnroll = 4;

__device__ __forceinline__ float4 ldv(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float dot4v(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

template <int NQ>
__device__ __forceinline__ void block_partials(double (&acc)[NQ], double* out, int64_t stride) {
  __shared__ double red[NQ][kBlk / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(kAll, acc[q], off);
  if (lane == 0)
    for (int q = 0; q < NQ; ++q) red[q][wid] = acc[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int i = 0; i < kBlk / 32; ++i) v += red[threadIdx.x][i];
    out[threadIdx.x * stride + blockIdx.x] = v;
  }
}

struct AdjArgs {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const float* val;     // nullptr: unit weights
  const float* vs;
  const float* ivs;
  int w;
  const float* gt;      // G tile, n x w
  const float* vj;      // V_j, or the R tile when j == 0 (then V_0 = vs R)
  int j0;
  const float* phi1;    // Phi_{j+1}
  const float* phi2;    // Phi_{j+2}, nullptr when zero
  float* phi0;          // Phi_j (nullptr when j == 0)
  float aj;             // a_j
  float cj;             // 1 for j == 0, 2 otherwise
  float* H;             // [nnz]
  double* part;         // [grid]: partial sums of <G, T_j R>
  int l2pf;             // prefetch the next batch of gathered rows into L2
};

// One reverse step: row-parallel, the LPR = w / 4 lanes of a slot own a row.
template <int LPR>
__global__ void __launch_bounds__(kBlk, 4) adjoint_step_kernel(AdjArgs a) {
  constexpr int S = 32 / LPR;
  const int lane = threadIdx.x & 31;
  const int slot = lane / LPR, sub = lane % LPR;
  const int w = a.w;
  const int64_t wslots = ((int64_t)gridDim.x * blockDim.x >> 5) * S;
  const int64_t first = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * S;
  double acc_a = 0.0;
  for (int64_t r0 = first; r0 < a.n; r0 += wslots) {
    const int64_t row = r0 + slot;
    const bool valid = row < a.n;
    int64_t beg = 0, end = 0;
    float4 p1 = make_float4(0.f, 0.f, 0.f, 0.f), g = p1, own = p1;
    float vsu = 1.f, ivsu = 1.f;
    if (valid) {
      beg = __ldg(a.row_ptr + row);
      end = __ldg(a.row_ptr + row + 1);
      p1 = ldv(a.phi1 + row * w + sub * 4);
      g = ldv(a.gt + row * w + sub * 4);
      own = ldv(a.vj + row * w + sub * 4);
      vsu = __ldg(a.vs + row);
      ivsu = __ldg(a.ivs + row);
    }
    int len = (int)(end - beg);
    int maxlen = len;
    for (int off = 16; off > 0; off >>= 1) maxlen = max(maxlen, __shfl_xor_sync(kAll, maxlen, off));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    constexpr int kLines = LPR >= 8 ? LPR / 8 : 1;  // 128-byte lines per gathered row
    for (int e0 = 0; e0 < maxlen; e0 += kEdgeUnroll) {
      if (a.l2pf) {
        // the next batch's rows of both gathered blocks into L2 while this batch loads
        for (int q = sub; q < 2 * kEdgeUnroll * kLines; q += LPR) {
          const int u = q / (2 * kLines), rest = q % (2 * kLines);
          if (e0 + kEdgeUnroll + u < len) {
            const int c = __ldg(a.col + beg + e0 + kEdgeUnroll + u);
            const float* src = (rest < kLines ? a.phi1 : a.vj) + (int64_t)c * w + (rest % kLines) * 32;
            asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(src) : "memory");
          }
        }
      }
      float4 pv[kEdgeUnroll], vv[kEdgeUnroll];
      float wt[kEdgeUnroll], sv[kEdgeUnroll], dot[kEdgeUnroll];
#pragma unroll
      for (int u = 0; u < kEdgeUnroll; ++u) {
        const bool ok = e0 + u < len;
        const int c = ok ? __ldg(a.col + beg + e0 + u) : 0;
        wt[u] = ok ? (a.val != nullptr ? __ldg(a.val + beg + e0 + u) : 1.0f) : 0.0f;
        sv[u] = ok && a.j0 ? __ldg(a.vs + c) : 1.0f;
        pv[u] = ok ? ldv(a.phi1 + (int64_t)c * w + sub * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        vv[u] = ok ? ldv(a.vj + (int64_t)c * w + sub * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kEdgeUnroll; ++u) {
        acc.x = fmaf(wt[u], pv[u].x, acc.x);
        acc.y = fmaf(wt[u], pv[u].y, acc.y);
        acc.z = fmaf(wt[u], pv[u].z, acc.z);
        acc.w = fmaf(wt[u], pv[u].w, acc.w);
        dot[u] = dot4v(p1, vv[u]) * sv[u];
      }
      // reduce-scatter of the four per-edge dots over the LPR lanes of the slot: the first two
      // exchanges hand each half of the lanes half of the edges, a butterfly finishes
      const int hA = LPR / 2;
      const bool upA = (sub & hA) != 0;
      float k0 = upA ? dot[2] : dot[0], k1 = upA ? dot[3] : dot[1];
      k0 += __shfl_xor_sync(kAll, upA ? dot[0] : dot[2], hA);
      k1 += __shfl_xor_sync(kAll, upA ? dot[1] : dot[3], hA);
      if constexpr (LPR >= 4) {
        constexpr int hB = LPR / 4;
        const bool upB = (sub & hB) != 0;
        float kk = (upB ? k1 : k0) + __shfl_xor_sync(kAll, upB ? k0 : k1, hB);
#pragma unroll
        for (int off = hB / 2; off >= 1; off >>= 1) kk += __shfl_xor_sync(kAll, kk, off);
        const int u = (upA ? 2 : 0) + (upB ? 1 : 0);
        if (sub % hB == 0 && e0 + u < len) a.H[beg + e0 + u] += a.cj * kk;
      } else {
        const int u = upA ? 2 : 0;
        if (e0 + u < len) a.H[beg + e0 + u] += a.cj * k0;
        if (e0 + u + 1 < len) a.H[beg + e0 + u + 1] += a.cj * k1;
      }
    }
    // <G, T_j R> over this row's columns: T_j = V_j / vs for j >= 1, R for j == 0
    float ga = dot4v(g, own) * (a.j0 ? 1.0f : ivsu);
    for (int off = 1; off < LPR; off <<= 1) ga += __shfl_xor_sync(kAll, ga, off);
    if (valid && sub == 0) acc_a += (double)ga;
    if (valid && a.phi0 != nullptr) {
      const float4 p2 = a.phi2 != nullptr ? ldv(a.phi2 + row * w + sub * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float sg = a.aj * vsu, c2 = -2.0f * vsu * vsu;
      float4 o;
      o.x = fmaf(sg, g.x, fmaf(c2, acc.x, -p2.x));
      o.y = fmaf(sg, g.y, fmaf(c2, acc.y, -p2.y));
      o.z = fmaf(sg, g.z, fmaf(c2, acc.z, -p2.z));
      o.w = fmaf(sg, g.w, fmaf(c2, acc.w, -p2.w));
      *reinterpret_cast<float4*>(a.phi0 + row * w + sub * 4) = o;
    }
  }
  double accs[1] = {acc_a};
  block_partials<1>(accs, a.part, 0);
}

// Phi_m = a_m vs G and the partial sums of <G, T_m R> = <G, V_m / vs>.
__global__ void adjoint_init_kernel(int64_t n, int w, const float* __restrict__ gt, const float* __restrict__ vm,
                                    const float* __restrict__ vs, const float* __restrict__ ivs, float am,
                                    float* __restrict__ phi, double* __restrict__ part) {
  double acc = 0.0;
  const int64_t total = n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / w;
    const float g = gt[e];
    phi[e] = am * __ldg(vs + row) * g;
    acc += (double)(g * vm[e] * __ldg(ivs + row));
  }
  double accs[1] = {acc};
  block_partials<1>(accs, part, 0);
}

// tpos[e] = position of (v, u) for the stored entry e = (u, v); bad counts entries without one.
__global__ void transpose_index_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                       const int32_t* __restrict__ col, int32_t* __restrict__ tpos,
                                       unsigned long long* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nw) {
    const int64_t beg = row_ptr[u], end = row_ptr[u + 1];
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int v = col[e];
      int64_t lo = row_ptr[v], hi = row_ptr[v + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < u) lo = mid + 1;
        else hi = mid;
      }
      const bool found = lo < row_ptr[v + 1] && col[lo] == (int32_t)u;
      tpos[e] = found ? (int32_t)lo : -1;
      if (!found) atomicAdd(bad, 1ull);
    }
  }
}

// The same for an internally reordered graph whose rows keep the caller's neighbour order:
// internal edge (i, offset k) is caller edge urp[perm[i]] + k; its transpose is found by binary
// search in the caller's sorted row and mapped back by its offset.
__global__ void transpose_index_perm_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                            const int64_t* __restrict__ urp, const int32_t* __restrict__ ucol,
                                            const int32_t* __restrict__ perm, const int32_t* __restrict__ iperm,
                                            int32_t* __restrict__ tpos, unsigned long long* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    const int32_t u = perm[i];
    const int64_t ub = urp[u];
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int v = ucol[ub + (e - beg)];
      int64_t lo = urp[v], hi = urp[v + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ucol[mid] < u) lo = mid + 1;
        else hi = mid;
      }
      const bool found = lo < urp[v + 1] && ucol[lo] == u;
      tpos[e] = found ? (int32_t)(row_ptr[iperm[v]] + (lo - urp[v])) : -1;
      if (!found) atomicAdd(bad, 1ull);
    }
  }
}

// s_u = -sum_{b in row u} w_ub (H_ub + H_bu): one warp per row.
__global__ void weight_node_sum_kernel(int64_t n, const int64_t* __restrict__ row_ptr, const float* __restrict__ val,
                                       const float* __restrict__ H, const int32_t* __restrict__ tpos,
                                       double* __restrict__ s) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nw) {
    double acc = 0.0;
    for (int64_t e = row_ptr[u] + lane; e < row_ptr[u + 1]; e += 32) {
      const double wv = val != nullptr ? (double)val[e] : 1.0;
      acc -= wv * ((double)H[e] + (double)H[tpos[e]]);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kAll, acc, off);
    if (lane == 0) s[u] = acc;
  }
}

// dloss/dw_e = -(H_uv + H_vu) - s_u / (2 d_u) - s_v / (2 d_v): one warp per row.
__global__ void weight_grad_kernel(int64_t n, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const float* __restrict__ H, const int32_t* __restrict__ tpos,
                                   const double* __restrict__ s, const double* __restrict__ deg,
                                   float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nw) {
    const double hu = s[u] / (2.0 * deg[u]);
    for (int64_t e = row_ptr[u] + lane; e < row_ptr[u + 1]; e += 32) {
      const int v = col[e];
      out[e] = (float)(-((double)H[e] + (double)H[tpos[e]]) - hu - s[v] / (2.0 * deg[v]));
    }
  }
}

// loss = sum_i ||y_i - mu_a(i)||^2 with y_i = psi_i / ||psi_i|| and dloss/dpsi_i =
// (g_i - y_i <y_i, g_i>) / ||psi_i||, g_i = 2 (y_i - mu_a(i)); a zero row has y_i = 0 and
// no gradient.  One warp per row.
__global__ void kmeans_loss_grad_kernel(int64_t n, int c, const float* __restrict__ psi, int64_t ldp,
                                        const float* __restrict__ mu, int k, const int32_t* __restrict__ assign,
                                        float* __restrict__ grad, int64_t ldg, double* __restrict__ part,
                                        unsigned long long* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double loss = 0.0;
  for (int64_t i = warp; i < n; i += nw) {
    const int ai = assign[i];
    if (ai < 0 || ai >= k) {
      if (lane == 0) atomicAdd(bad, 1ull);
      continue;
    }
    const float* p = psi + i * ldp;
    const float* m = mu + (int64_t)ai * c;
    double s2 = 0.0;
    for (int l = lane; l < c; l += 32) s2 += (double)p[l] * p[l];
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(kAll, s2, off);
    const double nrm = sqrt(s2);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    double proj = 0.0, li = 0.0;
    for (int l = lane; l < c; l += 32) {
      const double y = (double)p[l] * inv, diff = y - (double)m[l];
      li += diff * diff;
      proj += y * 2.0 * diff;
    }
    for (int off = 16; off > 0; off >>= 1) {
      proj += __shfl_xor_sync(kAll, proj, off);
      li += __shfl_xor_sync(kAll, li, off);
    }
    for (int l = lane; l < c; l += 32) {
      const double y = (double)p[l] * inv, gl = 2.0 * (y - (double)m[l]);
      grad[i * ldg + l] = nrm > 0.0 ? (float)((gl - y * proj) * inv) : 0.0f;
    }
    if (lane == 0) loss += li;
  }
  double accs[1] = {loss};
  block_partials<1>(accs, part, 0);
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double red[kBlk / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kAll, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = t;
  }
}

// Block partials: three rows of the forward kernels' moments, or one row of the adjoint's,
// plus the reduced sums after them.
size_t part_doubles(int grid) { return (size_t)3 * grid + 64; }

csc_status gfail(csc_ctx* ctx, csc_status s, const std::string& msg) {
  ctx->err = msg;
  return s;
}

#define G_CUDA(call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return csc::gfail(ctx, CSC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define G_ALLOC(expr)                                                                    \
  do {                                                                                   \
    if (!(expr)) return csc::gfail(ctx, CSC_ENOMEM, "device allocation failed: " #expr); \
  } while (0)

cudaError_t launch_adjoint(const AdjArgs& a, int grid, cudaStream_t s) {
  switch (a.w / 4) {
    case 2: adjoint_step_kernel<2><<<grid, kBlk, 0, s>>>(a); break;
    case 4: adjoint_step_kernel<4><<<grid, kBlk, 0, s>>>(a); break;
    case 8: adjoint_step_kernel<8><<<grid, kBlk, 0, s>>>(a); break;
    case 16: adjoint_step_kernel<16><<<grid, kBlk, 0, s>>>(a); break;
    default: adjoint_step_kernel<32><<<grid, kBlk, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

// Row maps between the caller's node order and the internal one (nullptr: the same order).
const int32_t* to_caller(csc_ctx* ctx) { return ctx->g.permuted ? as<int32_t>(ctx->g.perm) : nullptr; }
const int32_t* to_internal(csc_ctx* ctx) { return ctx->g.permuted ? as<int32_t>(ctx->g.iperm) : nullptr; }

StepArgs step_args(csc_ctx* ctx, int w, double* part) {
  StepArgs sa{};
  sa.n = ctx->g.n;
  sa.row_ptr = as<int64_t>(ctx->g.row_ptr);
  sa.col = as<int32_t>(ctx->g.col);
  sa.val = ctx->g.weighted ? as<float>(ctx->g.val) : nullptr;
  sa.scale = as<float>(ctx->g.scale);
  sa.vs = as<float>(ctx->g.vs);
  sa.ivs = as<float>(ctx->g.ivs);
  sa.blk_row = as<int32_t>(ctx->g.blk_row);
  sa.nblk = edge_blocks(ctx->g.nnz);
  sa.srow = as<int32_t>(ctx->g.srow);
  sa.nsblk = row_blocks(ctx->g.n, ctx->g.nnz);
  sa.coef = as<float>(ctx->gs.coef_f);
  sa.w = w;
  sa.part = part;
  return sa;
}

// Runs steps j = j_from .. j_to - 1 of the forward recursion (step j produces V_{j+1}) with
// V_j supplied by vp(j); Psi accumulates into psi (tile base, leading dimension ldp) unless null.
template <typename VP>
csc_status forward_steps(csc_ctx* ctx, int j_from, int j_to, VP vp, float* psi, int64_t ldp, double* part,
                         int grid, cudaStream_t s) {
  GradState& gs = ctx->gs;
  for (int j = j_from; j < j_to; ++j) {
    StepArgs sa = step_args(ctx, gs.w, part);
    sa.psi = psi;
    sa.ldp = ldp;
    if (j == 0) {
      sa.tg = gs.rt.ptr;
      sa.tp = nullptr;
      sa.tn = vp(1);
      sa.j = 0;
      G_CUDA(launch_cheb_first(sa, CSC_F32, grid, s));
    } else {
      sa.tg = vp(j);
      sa.tp = j == 1 ? static_cast<const float*>(gs.rt.ptr) : vp(j - 1);
      sa.tn = vp(j + 1);
      sa.j = j;
      sa.tp_unscaled = j == 1;
      G_CUDA(launch_cheb_step(sa, CSC_F32, grid, s));
    }
    ctx->launches += 1;
  }
  return CSC_OK;
}

}  // namespace
}  // namespace csc

using csc::GradState;

extern "C" csc_status csc_filter_forward(csc_ctx* ctx, int m, const double* coef, const float* R, int c,
                                         int64_t ldr, float* psi_out, int64_t ldp, int stride) {
  if (!ctx) return CSC_EINVAL;
  if (!ctx->g.loaded) return csc::gfail(ctx, CSC_ESTATE, "csc_filter_forward: no graph loaded");
  if (m < 1 || !coef || !R || c < 1 || ldr < c || !psi_out || ldp < c || stride < 0)
    return csc::gfail(ctx, CSC_EINVAL, "csc_filter_forward: bad arguments");
  GradState& gs = ctx->gs;
  const int64_t n = ctx->g.n;
  cudaStream_t s = ctx->stream;
  gs.ready = false;
  gs.m = m;
  gs.c = c;
  gs.coef.assign(coef, coef + m + 1);
  gs.stride = stride > 0 ? std::min(stride, m) : std::max(1, (int)std::ceil(std::sqrt((double)m)));
  gs.segs = (m + gs.stride - 1) / gs.stride;
  // widest tile of at most 64 columns whose gathered block fits 128 MB (as the filter path)
  int w = 8;
  while (w < 64 && w < c) w *= 2;
  while (w > 8 && (double)n * w * 4.0 > 128.0 * (1 << 20)) w /= 2;
  gs.w = w;
  gs.ntiles = (c + w - 1) / w;
  gs.slots = gs.stride == 1 ? m : 2 * (gs.segs - 1);
  const size_t blk = (size_t)std::max<int64_t>(n, 1) * w;
  const int grid = csc::cheb_grid(w);
  G_ALLOC(csc::ensure(gs.coef_f, (size_t)(m + 1) * 4));
  G_ALLOC(csc::ensure(gs.rt, blk * 4));
  G_ALLOC(csc::ensure(gs.gt, blk * 4));
  G_ALLOC(csc::ensure(gs.part, csc::part_doubles(grid) * 8));
  G_ALLOC(csc::ensure(gs.ckpt, std::max<size_t>(1, (size_t)gs.ntiles * gs.slots * blk) * 4));
  for (auto& b : ctx->tbuf) G_ALLOC(csc::ensure(b, blk * 4));
  // own copy of R: the backward pass restarts the first segment from it
  G_ALLOC(csc::ensure(gs.rcopy, (size_t)std::max<int64_t>(n, 1) * c * 4));
  G_CUDA(cudaMemcpy2DAsync(gs.rcopy.ptr, (size_t)c * 4, R, (size_t)ldr * 4, (size_t)c * 4, n,
                           cudaMemcpyDeviceToDevice, s));
  gs.R = csc::as<float>(gs.rcopy);
  gs.ldr = c;
  std::vector<float> af(gs.coef.begin(), gs.coef.end());
  G_CUDA(cudaMemcpyAsync(gs.coef_f.ptr, af.data(), af.size() * 4, cudaMemcpyHostToDevice, s));
  float* ck = csc::as<float>(gs.ckpt);
  double* part = csc::as<double>(gs.part);
  // Psi accumulates in an aligned n x w scratch tile (the kernels use 16-byte accesses); its
  // valid columns are then copied into the caller's block
  float* psi_tile = csc::as<float>(gs.gt);
  for (int tile = 0; tile < gs.ntiles; ++tile) {
    const int c0 = tile * w, valid = std::min(w, c - c0);
    G_CUDA(csc::launch_copy_tile(gs.rt.ptr, R, CSC_F32, n, w, ldr, c0, valid, s, csc::to_caller(ctx)));
    G_CUDA(cudaMemsetAsync(psi_tile, 0, blk * 4, s));
    float* tile_ck = ck + (size_t)tile * gs.slots * blk;
    // V_j lives in tbuf[j % 3], or in its checkpoint slot j - 1 when every step is kept
    auto vp = [&](int j) {
      return gs.stride == 1 ? tile_ck + (size_t)(j - 1) * blk : csc::as<float>(ctx->tbuf[j % 3]);
    };
    for (int j = 0; j < m; ++j) {
      csc_status st = csc::forward_steps(ctx, j, j + 1, vp, psi_tile, w, part, grid, s);
      if (st != CSC_OK) return st;
      if (gs.stride == 1) continue;
      const int v = j + 1;  // V_v was just produced
      int slot = -1;
      if (v % gs.stride == 0 && v < m) slot = 2 * (v / gs.stride - 1) + 1;
      else if ((v + 1) % gs.stride == 0 && v + 1 < m) slot = 2 * ((v + 1) / gs.stride - 1);
      if (slot >= 0)
        G_CUDA(cudaMemcpyAsync(tile_ck + (size_t)slot * blk, vp(v), blk * 4, cudaMemcpyDeviceToDevice, s));
    }
    G_CUDA(csc::launch_convert(psi_tile, CSC_F32, w, psi_out + c0, CSC_F32, ldp, n, valid, s, csc::to_internal(ctx)));
  }
  gs.ready = true;
  return CSC_OK;
}

extern "C" csc_status csc_filter_vjp(csc_ctx* ctx, const float* grad_psi, int64_t ldg, double* grad_coef,
                                     float* grad_w) {
  if (!ctx) return CSC_EINVAL;
  GradState& gs = ctx->gs;
  if (!gs.ready || !ctx->g.loaded) return csc::gfail(ctx, CSC_ESTATE, "csc_filter_vjp: no csc_filter_forward to differentiate");
  if (!grad_psi || ldg < gs.c) return csc::gfail(ctx, CSC_EINVAL, "csc_filter_vjp: bad arguments");
  const int64_t n = ctx->g.n, nnz = ctx->g.nnz;
  const int m = gs.m, w = gs.w, S = gs.stride;
  cudaStream_t s = ctx->stream;
  const size_t blk = (size_t)std::max<int64_t>(n, 1) * w;
  const int grid = csc::cheb_grid(w);
  const int sms = csc::num_sms();
  const int agrid = sms * 8;
  G_ALLOC(csc::ensure(gs.gt, blk * 4));
  if (S > 1) G_ALLOC(csc::ensure(gs.seg, (size_t)(S + 2) * blk * 4));
  for (auto& b : gs.phi) G_ALLOC(csc::ensure(b, blk * 4));
  G_ALLOC(csc::ensure(gs.H, (size_t)std::max<int64_t>(nnz, 1) * 4));
  G_ALLOC(csc::ensure(gs.part, csc::part_doubles(std::max(grid, agrid)) * 8));
  std::vector<double> ga_part((size_t)(m + 1) * gs.ntiles, 0.0);
  // per-step <G, T_j R> sums land in ga[j * ntiles + tile]
  G_ALLOC(csc::ensure(gs.ga, (size_t)(m + 1) * gs.ntiles * 8));
  if (nnz > 0) G_CUDA(cudaMemsetAsync(gs.H.ptr, 0, (size_t)nnz * 4, s));
  double* part = csc::as<double>(gs.part);
  double* ga_dev = csc::as<double>(gs.ga);
  float* seg = csc::as<float>(gs.seg);
  const float* ck = csc::as<float>(gs.ckpt);
  for (int tile = 0; tile < gs.ntiles; ++tile) {
    const int c0 = tile * w, valid = std::min(w, gs.c - c0);
    G_CUDA(csc::launch_copy_tile(gs.rt.ptr, gs.R, CSC_F32, n, w, gs.ldr, c0, valid, s, csc::to_caller(ctx)));
    G_CUDA(csc::launch_copy_tile(gs.gt.ptr, grad_psi, CSC_F32, n, w, ldg, c0, valid, s, csc::to_caller(ctx)));
    const float* tile_ck = ck + (size_t)tile * gs.slots * blk;
    // V_j (j >= 1) of the current segment [lo, hi]: its checkpoint slot j - 1 when every step
    // is kept, else seg slot j - lo + 1 (slot 0 holds V_{lo-1})
    int lo = 0, hi = 0;
    auto vseg = [&](int j) -> float* {
      return S == 1 ? const_cast<float*>(tile_ck) + (size_t)(j - 1) * blk : seg + (size_t)(j - lo + 1) * blk;
    };
    auto phi = [&](int j) { return csc::as<float>(gs.phi[((j % 3) + 3) % 3]); };
    for (int k = gs.segs - 1; k >= 0; --k) {
      lo = k * S;
      hi = std::min(m, lo + S);
      // recompute V_{lo+1} .. V_hi (V_lo and V_{lo-1} from the checkpoints, or from R)
      if (S > 1) {
        if (k >= 1) {
          G_CUDA(cudaMemcpyAsync(vseg(lo - 1), tile_ck + (size_t)(2 * (k - 1)) * blk, blk * 4, cudaMemcpyDeviceToDevice, s));
          G_CUDA(cudaMemcpyAsync(vseg(lo), tile_ck + (size_t)(2 * (k - 1) + 1) * blk, blk * 4, cudaMemcpyDeviceToDevice, s));
        }
        auto vrec = [&](int j) { return vseg(j); };
        csc_status st = csc::forward_steps(ctx, lo, hi, vrec, nullptr, 0, part, grid, s);
        if (st != CSC_OK) return st;
      }
      if (k == gs.segs - 1) {
        csc::adjoint_init_kernel<<<agrid, csc::kBlk, 0, s>>>(n, w, csc::as<float>(gs.gt), vseg(m),
                                                             csc::as<float>(ctx->g.vs), csc::as<float>(ctx->g.ivs),
                                                             (float)gs.coef[m], phi(m), part);
        G_CUDA(cudaGetLastError());
        csc::sum_partials_kernel<<<1, csc::kBlk, 0, s>>>(part, agrid, ga_dev + (size_t)m * gs.ntiles + tile);
        G_CUDA(cudaGetLastError());
        ctx->launches += 2;
      }
      for (int j = hi - 1; j >= lo; --j) {
        csc::AdjArgs a{};
        a.n = n;
        a.row_ptr = csc::as<int64_t>(ctx->g.row_ptr);
        a.col = csc::as<int32_t>(ctx->g.col);
        a.val = ctx->g.weighted ? csc::as<float>(ctx->g.val) : nullptr;
        a.vs = csc::as<float>(ctx->g.vs);
        a.ivs = csc::as<float>(ctx->g.ivs);
        a.w = w;
        a.gt = csc::as<float>(gs.gt);
        a.j0 = j == 0;
        a.vj = j == 0 ? csc::as<float>(gs.rt) : vseg(j);
        a.phi1 = phi(j + 1);
        a.phi2 = j + 2 <= m ? phi(j + 2) : nullptr;
        a.phi0 = j >= 1 ? phi(j) : nullptr;
        a.aj = (float)gs.coef[j];
        a.cj = j == 0 ? 1.0f : 2.0f;
        a.H = csc::as<float>(gs.H);
        a.part = part;
        a.l2pf = (double)n * w * 8.0 > 64.0 * (1 << 20);  // two gathered blocks of n x w floats
        G_CUDA(csc::launch_adjoint(a, agrid, s));
        csc::sum_partials_kernel<<<1, csc::kBlk, 0, s>>>(part, agrid, ga_dev + (size_t)j * gs.ntiles + tile);
        G_CUDA(cudaGetLastError());
        ctx->launches += 2;
      }
    }
  }
  G_CUDA(cudaMemcpyAsync(ga_part.data(), ga_dev, ga_part.size() * 8, cudaMemcpyDeviceToHost, s));
  if (grad_w != nullptr && nnz > 0) {
    if (gs.graph_version != ctx->graph_version) {
      G_ALLOC(csc::ensure(gs.tpos, (size_t)nnz * 4));
      G_ALLOC(csc::ensure(gs.flag, 8));
      G_CUDA(cudaMemsetAsync(gs.flag.ptr, 0, 8, s));
      if (ctx->g.permuted)
        csc::transpose_index_perm_kernel<<<sms * 8, csc::kBlk, 0, s>>>(
            n, csc::as<int64_t>(ctx->g.row_ptr), csc::as<int64_t>(ctx->g.urp), csc::as<int32_t>(ctx->g.ucol),
            csc::as<int32_t>(ctx->g.perm), csc::as<int32_t>(ctx->g.iperm), csc::as<int32_t>(gs.tpos),
            csc::as<unsigned long long>(gs.flag));
      else
        csc::transpose_index_kernel<<<sms * 8, csc::kBlk, 0, s>>>(n, csc::as<int64_t>(ctx->g.row_ptr),
                                                                  csc::as<int32_t>(ctx->g.col),
                                                                  csc::as<int32_t>(gs.tpos),
                                                                  csc::as<unsigned long long>(gs.flag));
      G_CUDA(cudaGetLastError());
      unsigned long long bad = 0;
      G_CUDA(cudaMemcpyAsync(&bad, gs.flag.ptr, 8, cudaMemcpyDeviceToHost, s));
      G_CUDA(cudaStreamSynchronize(s));
      if (bad != 0) return csc::gfail(ctx, CSC_EINVAL, "csc_filter_vjp: the graph is not symmetric");
      gs.graph_version = ctx->graph_version;
      ctx->launches += 1;
    }
    G_ALLOC(csc::ensure(gs.nsum, (size_t)n * 8));
    const float* val = ctx->g.weighted ? csc::as<float>(ctx->g.val) : nullptr;
    csc::weight_node_sum_kernel<<<sms * 8, csc::kBlk, 0, s>>>(n, csc::as<int64_t>(ctx->g.row_ptr), val,
                                                              csc::as<float>(gs.H), csc::as<int32_t>(gs.tpos),
                                                              csc::as<double>(gs.nsum));
    G_CUDA(cudaGetLastError());
    // per internal edge; scattered to the caller's edge order when the graph is reordered
    float* gw = grad_w;
    if (ctx->g.permuted) {
      G_ALLOC(csc::ensure(gs.gw_stage, (size_t)nnz * 4));
      gw = csc::as<float>(gs.gw_stage);
    }
    csc::weight_grad_kernel<<<sms * 8, csc::kBlk, 0, s>>>(n, csc::as<int64_t>(ctx->g.row_ptr),
                                                          csc::as<int32_t>(ctx->g.col), csc::as<float>(gs.H),
                                                          csc::as<int32_t>(gs.tpos), csc::as<double>(gs.nsum),
                                                          csc::as<double>(ctx->g.deg), gw);
    G_CUDA(cudaGetLastError());
    ctx->launches += 2;
    if (ctx->g.permuted) {
      G_CUDA(csc::launch_scatter_edges(ctx->g, gw, grad_w, s));
      ctx->launches += 1;
    }
  }
  G_CUDA(cudaStreamSynchronize(s));
  if (grad_coef != nullptr)
    for (int j = 0; j <= m; ++j) {
      double t = 0.0;
      for (int tile = 0; tile < gs.ntiles; ++tile) t += ga_part[(size_t)j * gs.ntiles + tile];
      grad_coef[j] = t;
    }
  return CSC_OK;
}

extern "C" csc_status csc_kmeans_loss_grad(csc_ctx* ctx, const float* psi, int64_t ldp, int64_t n, int c,
                                           const float* mu, int k, const int32_t* assign, float* grad_psi,
                                           int64_t ldg, double* loss_out) {
  if (!ctx) return CSC_EINVAL;
  if (!psi || !mu || !assign || !grad_psi || n < 1 || c < 1 || k < 1 || ldp < c || ldg < c)
    return csc::gfail(ctx, CSC_EINVAL, "csc_kmeans_loss_grad: bad arguments");
  cudaStream_t s = ctx->stream;
  const int grid = csc::num_sms() * 8;
  G_ALLOC(csc::ensure(ctx->gs.part, csc::part_doubles(grid) * 8));
  G_ALLOC(csc::ensure(ctx->gs.flag, 8));
  double* part = csc::as<double>(ctx->gs.part);
  unsigned long long* bad = csc::as<unsigned long long>(ctx->gs.flag);
  G_CUDA(cudaMemsetAsync(bad, 0, 8, s));
  csc::kmeans_loss_grad_kernel<<<grid, csc::kBlk, 0, s>>>(n, c, psi, ldp, mu, k, assign, grad_psi, ldg, part, bad);
  G_CUDA(cudaGetLastError());
  csc::sum_partials_kernel<<<1, csc::kBlk, 0, s>>>(part, grid, part + grid);
  G_CUDA(cudaGetLastError());
  ctx->launches += 2;
  double loss = 0.0;
  unsigned long long nbad = 0;
  G_CUDA(cudaMemcpyAsync(&loss, part + grid, 8, cudaMemcpyDeviceToHost, s));
  G_CUDA(cudaMemcpyAsync(&nbad, bad, 8, cudaMemcpyDeviceToHost, s));
  G_CUDA(cudaStreamSynchronize(s));
  if (nbad != 0) return csc::gfail(ctx, CSC_EINVAL, "csc_kmeans_loss_grad: assignment outside [0, k)");
  if (loss_out) *loss_out = loss;
  return CSC_OK;
}
