// Tensor-core distance pass of k-means (Eq. 1; the assignment step of the clustering in
// Algorithm 1) for sm_103a: tcgen05 MMA with TMEM accumulators, operands staged by TMA.
//
// The nearest centroid of row y minimises f_j = |c_j|^2 - 2 <y, c_j>.  The inner products
// are one dense (n x d) by (d x k) product, the only GEMM of the path, so they go to the
// tensor cores in bfloat16 with float32 accumulation.  The centroids are split in two
// bfloat16 parts, c = c0 + c1 + ec (|ec| <= 2^-16 |c|); float32 features likewise,
// y = y0 + y1 + ey, and bfloat16 features are y0 exactly:
//     <y, c> ~ <y0, c0> + <y0, c1> (+ <y1, c0>)   (two or three MMAs into one accumulator).
// The dropped terms are at most 3.02 2^-16 |y| cmax (1.001 2^-16 |y0| cmax without y1), the
// accumulation at most (N_mma + 1) 2^-21 sum|products|, a bound that allows for truncating
// adders and two roundings per MMA instruction; with the roundings of |c|^2 and of the
// epilogue this gives E, a bound on |f_j - e_j| (e_j the exact value with the float64
// centroids).  A row whose second-best value exceeds best + 2E is
// decided; any other row keeps its candidate set {j : f_j <= best + 2E}, which contains every
// exact minimiser.  Those rows are refined on CUDA cores: float32 values of the candidates
// with their certified bound B32, then float64 on the candidates B32 cannot separate (lowest
// index on ties).  Every assignment therefore equals the float64 argmin of the reference
// definition.
//
// Kernel layout (one CTA per SM, persistent over 128-row tiles):
//   warp 0      TMA producer: the split centroids once, then y0 (and y1) chunks of 128 rows x
//               64 elements (16 KB contiguous each in the chunk-major layout, 128-byte
//               swizzle) through an S-stage ring;
//   warp 1      allocates TMEM (two accumulators of 128 lanes x N columns) and one thread
//               issues the MMAs (M = 128, N = k rounded up to 16, K = 16 per instruction);
//   warps 2-5   epilogue: each thread owns one TMEM lane (one row), reads its N values with
//               one tcgen05.ld, forms f_j, keeps best and second best in four independent
//               streams, and writes the assignment, the moves, or the near-tie candidate mask.
// Every mbarrier wait is bounded (about a second); a wait that runs out sets the error word,
// the CTA drains its copies and MMAs in flight, frees its TMEM and returns.
//
// Rows that cannot move are skipped (Hamerly's bounds).  A decided row leaves an upper bound
// u >= |y - c_a| (its own centroid a) and a lower bound l <= min_{j != a} |y - c_j|, from
// best + E and second - E plus |y|^2 in directed rounding; a near-tie row leaves (inf, 0).
// After the update the centroids move by at most delta_j (float64 norms rounded up), so by the
// triangle inequality u + delta_a and l - max_{j != a} delta_j are bounds for the new
// centroids.  A row with u < l keeps a (every other centroid is strictly farther, so no tie
// either) and is not evaluated; the others are listed, copied into a compact copy of the split
// rows (when they are at most a fifth of all rows), and the pass runs over that copy.  Skipping
// changes no assignment, so the sums, centroids and pass count are those of plain Lloyd.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "csc_internal.h"

namespace csc {

namespace {

constexpr int kTM = 128;                 // rows per tile (MMA M, TMEM lanes)
constexpr int kKC = 64;                  // bfloat16 elements per chunk (one 128-byte row)
constexpr int kThreads = 192;            // 6 warps
constexpr uint32_t kChunkA = kTM * 128;  // bytes of one 128 x 64 bfloat16 chunk
constexpr int kMaxDynSmem = 232448;      // 227 KB
constexpr int kMaxStages = 8;
constexpr int kCn2Slots = 256;           // |c|^2 cache in shared memory, +inf past k
constexpr int kPrefetch = 4;             // tiles of this CTA prefetched into L2 ahead of the loads
constexpr long long kWaitCycles = 2000000000LL;  // about a second at the SM clock

struct TcArgs {
  int64_t n;
  int k, npad, nk, stages, track, has_lo;
  uint32_t acc_off, tmem_cols;
  uint32_t stage_bytes, b_bytes;
  float kdot;                       // product error bound per ynorm.x * cmax
  const float2* ynorm;              // [n] (|y0|, |y - y0|) or, with y1, (|y|, 0); rounded up
  const float* cn2;                 // [npad] |c_j|^2 rounded to nearest from float64
  const unsigned int* cmax_bits;    // max_j |c_j| rounded up (float bits)
  int32_t* assign;                  // [n]
  int32_t* flagged;                 // [n] rows left for the float64 decision
  uint16_t* masks;                  // [n][npad / 16] candidate masks of those rows
  int32_t* moved;                   // [3][n]: row, old, new
  unsigned long long* counters;     // [0] moved, [1] flagged, [2] rows evaluated, [4] error word,
                                    // [6] compacted (with sel)
  const int32_t* sel;               // rows of the compacted copy (nullptr: every row, in place)
  int rowmajor;                     // tm_y0 maps the bfloat16 feature rows themselves (2-D)
  const float2* y2b;                // [n] |y|^2 rounded down and up
  float2* bnd;                      // [n] Hamerly bounds (u, l)
};

__device__ __forceinline__ float ldf_any(const float* p) { return *p; }
__device__ __forceinline__ float ldf_any(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// L2 prefetch of one box (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: bfloat16 A and B (K-major), float32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// TMEM -> registers: NV consecutive columns of this thread's lane, and the wait for them, in
// one asm statement so that no use of the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld_16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_128(uint32_t taddr, uint32_t (&r)[128]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x128.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64, %65, %66, %67, %68, %69, %70, %71, %72, %73, %74, %75, %76, %77, %78, %79, %80, %81, %82, %83, %84, %85, %86, %87, %88, %89, %90, %91, %92, %93, %94, %95, %96, %97, %98, %99, %100, %101, %102, %103, %104, %105, %106, %107, %108, %109, %110, %111, %112, %113, %114, %115, %116, %117, %118, %119, %120, %121, %122, %123, %124, %125, %126, %127}, [%128];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79]), "=r"(r[80]), "=r"(r[81]), "=r"(r[82]), "=r"(r[83]), "=r"(r[84]), "=r"(r[85]), "=r"(r[86]), "=r"(r[87]), "=r"(r[88]), "=r"(r[89]), "=r"(r[90]), "=r"(r[91]), "=r"(r[92]), "=r"(r[93]), "=r"(r[94]), "=r"(r[95]), "=r"(r[96]), "=r"(r[97]), "=r"(r[98]), "=r"(r[99]), "=r"(r[100]), "=r"(r[101]), "=r"(r[102]), "=r"(r[103]), "=r"(r[104]), "=r"(r[105]), "=r"(r[106]), "=r"(r[107]), "=r"(r[108]), "=r"(r[109]), "=r"(r[110]), "=r"(r[111]), "=r"(r[112]), "=r"(r[113]), "=r"(r[114]), "=r"(r[115]), "=r"(r[116]), "=r"(r[117]), "=r"(r[118]), "=r"(r[119]), "=r"(r[120]), "=r"(r[121]), "=r"(r[122]), "=r"(r[123]), "=r"(r[124]), "=r"(r[125]), "=r"(r[126]), "=r"(r[127])
      : "r"(taddr)
      : "memory");
}

template <int NV>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[NV]) {
  if constexpr (NV == 16) tmem_ld_16(taddr, r);
  else if constexpr (NV == 32) tmem_ld_32(taddr, r);
  else if constexpr (NV == 64) tmem_ld_64(taddr, r);
  else tmem_ld_128(taddr, r);
}

// (b, i, s) <- best, its index and second best of two candidate sets; equal values keep the
// lower index.
__device__ __forceinline__ void merge_top2(float& b, int& i, float& s, float b2, int i2, float s2) {
  if (b2 < b || (b2 == b && i2 < i)) {
    s = fminf(s2, b);
    b = b2;
    i = i2;
  } else {
    s = fminf(s, b2);
  }
}

__device__ __forceinline__ void set_error(const TcArgs& a, unsigned long long code) {
  atomicMax(a.counters + 4, code);
}

// NV: accumulator columns read into registers at once (the smallest power of two >= k_pad,
// at most 128; k_pad > 128 takes two reads).
template <int NV>
__global__ void __launch_bounds__(kThreads, 1)
    kmeans_tc_kernel(const __grid_constant__ CUtensorMap tm_y0, const __grid_constant__ CUtensorMap tm_y1,
                     const __grid_constant__ CUtensorMap tm_c, const __grid_constant__ CUtensorMap tm_y0c,
                     const __grid_constant__ CUtensorMap tm_y1c, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base (128-byte swizzle atoms)
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t sb = smem_u32(base);
  const uint32_t sB = sb;                       // [2][nk] chunks of npad x 128 B
  const uint32_t sA = sb + a.b_bytes;           // [stages] y0 chunk (+ y1 chunk)
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + a.b_bytes + (size_t)a.stages * a.stage_bytes);
  const int S = a.stages;
  // barrier indices: full[S], empty[S], bfull, acc_full[2], acc_empty[2], drain
  auto bar = [&](int i) { return smem_u32(bars + i); };
  const int kFull = 0, kEmpty = S, kBFull = 2 * S, kAccFull = 2 * S + 1, kAccEmpty = 2 * S + 3,
            kDrain = 2 * S + 5;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);
  float* cn2s = reinterpret_cast<float*>(tmem_holder + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rows of this pass: all n in place, or the selected rows (compacted, or in place when many)
  int64_t nr = a.n;
  bool cmp = false;
  if (a.sel != nullptr) {
    nr = (int64_t)a.counters[2];
    cmp = a.counters[6] != 0;
  }
  const int64_t ntiles = (nr + kTM - 1) / kTM;
  const CUtensorMap* my0 = cmp ? &tm_y0c : &tm_y0;
  const CUtensorMap* my1 = cmp ? &tm_y1c : &tm_y1;
  const bool rm = a.rowmajor && !cmp;  // 2-D boxes (x = chunk * 64, y = row), else chunk-major 3-D

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(bar(kFull + i), 1);
      mbar_init(bar(kEmpty + i), 1);
    }
    mbar_init(bar(kBFull), 1);
    mbar_init(bar(kAccFull), 1);
    mbar_init(bar(kAccFull + 1), 1);
    mbar_init(bar(kAccEmpty), 4 * 32);
    mbar_init(bar(kAccEmpty + 1), 4 * 32);
    mbar_init(bar(kDrain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int j = threadIdx.x; j < kCn2Slots; j += blockDim.x) cn2s[j] = j < a.k ? a.cn2[j] : INFINITY;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      // split centroids: rows [0, npad) hold c0, rows [npad, 2 npad) hold c1
      const uint32_t bchunk = (uint32_t)a.npad * 128u;
      mbar_expect_tx(bar(kBFull), a.b_bytes);
      for (int part = 0; part < 2; ++part)
        for (int kc = 0; kc < a.nk; ++kc)
          tma_load_2d(sB + (uint32_t)(part * a.nk + kc) * bchunk, &tm_c, kc * kKC, part * a.npad,
                      bar(kBFull));
      uint32_t q = 0;
      bool ok = true;
      // the stage loads of tile t hit L2: its boxes were prefetched kPrefetch tiles earlier
      for (int64_t tp = blockIdx.x; tp < ntiles && tp < blockIdx.x + (int64_t)kPrefetch * gridDim.x;
           tp += gridDim.x)
        for (int kc = 0; kc < a.nk; ++kc) {
          if (rm) {
            tma_prefetch_2d(my0, kc * kKC, (int)(tp * kTM));
          } else {
            tma_prefetch_3d(my0, 0, (int)(tp * kTM), kc);
            if (a.has_lo) tma_prefetch_3d(my1, 0, (int)(tp * kTM), kc);
          }
        }
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int64_t tp = t + (int64_t)kPrefetch * gridDim.x;
        if (tp < ntiles)
          for (int kc = 0; kc < a.nk; ++kc) {
            if (rm) {
              tma_prefetch_2d(my0, kc * kKC, (int)(tp * kTM));
            } else {
              tma_prefetch_3d(my0, 0, (int)(tp * kTM), kc);
              if (a.has_lo) tma_prefetch_3d(my1, 0, (int)(tp * kTM), kc);
            }
          }
        for (int kc = 0; kc < a.nk; ++kc) {
          const uint32_t s = q % S, ph = (q / S) & 1u;
          if (!mbar_wait(bar(kEmpty + s), ph ^ 1u)) {
            set_error(a, 1);
            ok = false;
            break;
          }
          mbar_expect_tx(bar(kFull + s), a.stage_bytes);
          const uint32_t dst = sA + s * a.stage_bytes;
          if (rm) {
            tma_load_2d(dst, my0, kc * kKC, (int)(t * kTM), bar(kFull + s));
          } else {
            tma_load_3d(dst, my0, 0, (int)(t * kTM), kc, bar(kFull + s));
            if (a.has_lo) tma_load_3d(dst + kChunkA, my1, 0, (int)(t * kTM), kc, bar(kFull + s));
          }
          ++q;
        }
      }
      // drain: the last loads issued have landed before the CTA exits
      for (uint32_t r = q > (uint32_t)S ? q - S : 0u; r < q; ++r) mbar_wait(bar(kFull + r % S), (r / S) & 1u);
      mbar_wait(bar(kBFull), 0);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = mma_idesc(a.npad);
      const uint32_t bchunk = (uint32_t)a.npad * 128u;
      bool ok = mbar_wait(bar(kBFull), 0);
      if (!ok) set_error(a, 2);
      tc_fence_after();
      uint32_t q = 0, i = 0;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const uint32_t acc = i & 1u, use = i >> 1;
        if (!mbar_wait(bar(kAccEmpty + acc), (use & 1u) ^ 1u)) {
          set_error(a, 3);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tbase + acc * a.acc_off;
        for (int kc = 0; kc < a.nk; ++kc) {
          const uint32_t s = q % S, ph = (q / S) & 1u;
          if (!mbar_wait(bar(kFull + s), ph)) {
            set_error(a, 4);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = sA + s * a.stage_bytes, a1 = a0 + kChunkA;
          const uint32_t b0 = sB + (uint32_t)kc * bchunk, b1 = sB + (uint32_t)(a.nk + kc) * bchunk;
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
            const uint32_t off = (uint32_t)kk * 32u;
            mma_bf16(d_tmem, sw128_desc(a0 + off), sw128_desc(b0 + off), idesc, (kc | kk) != 0);
            mma_bf16(d_tmem, sw128_desc(a0 + off), sw128_desc(b1 + off), idesc, 1u);
            if (a.has_lo) mma_bf16(d_tmem, sw128_desc(a1 + off), sw128_desc(b0 + off), idesc, 1u);
          }
          mma_commit(bar(kEmpty + s));  // frees the stage once these MMAs have read it
          ++q;
        }
        if (!ok) break;
        mma_commit(bar(kAccFull + acc));
      }
      // drain: every MMA issued has completed before TMEM is freed
      mma_commit(bar(kDrain));
      mbar_wait(bar(kDrain), 0);
    }
    __syncwarp();
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
    const int quad = warp & 3;
    const int rl = quad * 32 + lane;
    const float cmax = __uint_as_float(*a.cmax_bits);
    const float u = 5.9604644775390625e-8f;  // 2^-24
    const int words = a.npad / 16;
    uint32_t i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const uint32_t acc = i & 1u, use = i >> 1;
      const bool got = mbar_wait(bar(kAccFull + acc), use & 1u);
      if (!__all_sync(0xffffffffu, got)) {
        set_error(a, 5);
        break;
      }
      tc_fence_after();
      const int64_t slot_row = t * kTM + rl;
      const bool valid = slot_row < nr;
      const int64_t row = !valid ? 0 : (cmp ? (int64_t)a.sel[slot_row] : slot_row);
      const float2 yr = valid ? a.ynorm[row] : make_float2(0.f, 0.f);
      const float yabs = yr.x + yr.y;  // >= |y|
      const float dot_err = (yr.y + a.kdot * yr.x) * cmax;
      const float E = (2.0f * dot_err + u * (2.0f * cmax * cmax + 2.0f * yabs * cmax + 2.0f * dot_err)) *
                          1.0001f + 1e-30f;
      const uint32_t taddr = tbase + acc * a.acc_off + ((uint32_t)(quad * 32) << 16);
      const int groups = (a.npad + NV - 1) / NV;
      uint32_t r[NV];
      // four independent best / second-best streams (columns x mod 4), merged below
      float best[4], second[4];
      int bidx[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { best[q] = INFINITY; second[q] = INFINITY; bidx[q] = 0; }
      for (int g = 0; g < groups; ++g) {
        tmem_ld<NV>(taddr + (uint32_t)(g * NV), r);
        // branch-free: cn2s is +inf past k, so padded columns never win
#pragma unroll
        for (int x = 0; x < NV; ++x) {
          const int j = g * NV + x, q = x & 3;
          const float f = fmaf(-2.0f, __uint_as_float(r[x]), cn2s[j]);
          const bool lt = f < best[q];
          second[q] = lt ? best[q] : fminf(second[q], f);
          bidx[q] = lt ? j : bidx[q];
          best[q] = lt ? f : best[q];
        }
      }
      float bst = best[0], sec = second[0];
      int bi = bidx[0];
#pragma unroll
      for (int q = 1; q < 4; ++q) merge_top2(bst, bi, sec, best[q], bidx[q], second[q]);
      const float thr = __fadd_ru(bst, 2.0f * E);
      const bool flag = valid && !(thr < sec);
      // slots for the flagged rows of this warp
      const unsigned fm = __ballot_sync(0xffffffffu, flag);
      int slot = 0;
      if (fm) {
        unsigned long long fb = 0;
        if (lane == __ffs(fm) - 1) fb = atomicAdd(a.counters + 1, (unsigned long long)__popc(fm));
        fb = __shfl_sync(0xffffffffu, fb, __ffs(fm) - 1);
        slot = (int)fb + __popc(fm & ((1u << lane) - 1u));
        // candidate mask {j : f_j <= best + 2E}; same arithmetic as above
        for (int g = 0; g < groups; ++g) {
          if (groups > 1) tmem_ld<NV>(taddr + (uint32_t)(g * NV), r);
#pragma unroll
          for (int c = 0; c < NV / 16; ++c) {
            uint32_t bits = 0;
#pragma unroll
            for (int x = 0; x < 16; ++x) {
              const int j = g * NV + c * 16 + x;
              bits |= (fmaf(-2.0f, __uint_as_float(r[c * 16 + x]), cn2s[j]) <= thr ? 1u : 0u) << x;
            }
            const int wi = g * (NV / 16) + c;
            if (flag && wi < words) a.masks[(size_t)slot * words + wi] = (uint16_t)bits;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(bar(kAccEmpty + acc));
      if (flag) a.flagged[slot] = (int32_t)row;
      if (valid) {
        // Hamerly bounds against the float64 centroids: |y - c_j|^2 = e_j + |y|^2 with
        // |f_j - e_j| <= E; a near-tie row is evaluated again next pass
        float2 bd = make_float2(INFINITY, 0.f);
        if (!flag) {
          const float2 y2 = a.y2b[row];
          bd.x = __fsqrt_ru(__fadd_ru(__fadd_ru(bst, E), y2.y));
          const float l2 = __fadd_rd(__fsub_rd(sec, E), y2.x);
          bd.y = l2 > 0.f ? __fsqrt_rd(l2) : 0.f;
        }
        a.bnd[row] = bd;
      }
      bool mv = false;
      int old = 0;
      if (valid && !flag) {
        if (a.track) {
          old = a.assign[row];
          mv = old != bi;
          if (mv) a.assign[row] = bi;
        } else {
          a.assign[row] = bi;
        }
      }
      const unsigned mm = __ballot_sync(0xffffffffu, mv);
      if (mm) {
        unsigned long long mb = 0;
        if (lane == __ffs(mm) - 1) mb = atomicAdd(a.counters, (unsigned long long)__popc(mm));
        mb = __shfl_sync(0xffffffffu, mb, __ffs(mm) - 1);
        if (mv) {
          const int64_t m = (int64_t)mb + __popc(mm & ((1u << lane) - 1u));
          a.moved[m] = (int32_t)row;
          a.moved[a.n + m] = old;
          a.moved[2 * a.n + m] = bi;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(a.tmem_cols)
                 : "memory");
}

// Decision of the near-tie rows on their candidate sets, one warp per row: float32 values
// f_j = |c32_j|^2 - 2 <y, c32_j> with |f_j - e_j| <= B32 = u (3.1 cmax^2 + 2 (1.01 d + 1) |y| cmax)
// (u = 2^-24; recursive float32 summation of d products plus the rounding of the centroids
// and their norms); when B32 cannot separate the best candidate, float64 distances
// sum_l (y_l - c_jl)^2 on the candidates with f_j <= best + 2 B32, lowest index on ties.
template <typename TY>
__global__ void tc_refine_kernel(const TY* __restrict__ y, int64_t ldy, int d, const float* __restrict__ c32,
                                 const float* __restrict__ cn2_32, const unsigned int* __restrict__ cmax32_bits,
                                 const double* __restrict__ c64, TcArgs a) {
  const unsigned long long nflag = a.counters[1];
  const int lane = threadIdx.x & 31;
  const int words = a.npad / 16;
  const float u = 5.9604644775390625e-8f;
  const float cmax = __uint_as_float(*cmax32_bits);
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = warp; w < (int64_t)nflag; w += nwarps) {
    const int64_t row = a.flagged[w];
    const TY* yr = y + row * ldy;
    float yn = 0.f;
    for (int l = lane; l < d; l += 32) {
      const float v = ldf_any(yr + l);
      yn = fmaf(v, v, yn);
    }
    for (int off = 16; off > 0; off >>= 1) yn += __shfl_xor_sync(0xffffffffu, yn, off);
    const float B = u * (3.1f * cmax * cmax + 2.0f * (1.01f * d + 1.0f) * sqrtf(yn) * cmax);
    auto f32 = [&](int j) {
      float s = 0.f;
      for (int l = lane; l < d; l += 32) s = fmaf(ldf_any(yr + l), c32[(size_t)j * d + l], s);
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      return fmaf(-2.0f, s, cn2_32[j]);
    };
    float best = INFINITY, second = INFINITY;
    int bi = 0;
    for (int wi = 0; wi < words; ++wi) {
      uint32_t bits = a.masks[(size_t)w * words + wi];
      while (bits) {
        const int j = wi * 16 + __ffs(bits) - 1;
        bits &= bits - 1;
        const float f = f32(j);
        if (f < best) { second = best; best = f; bi = j; }
        else if (f < second) second = f;
      }
    }
    const float thr = __fadd_ru(best, 2.0f * B);
    if (!(thr < second)) {
      double b64 = INFINITY;
      for (int wi = 0; wi < words; ++wi) {
        uint32_t bits = a.masks[(size_t)w * words + wi];
        while (bits) {
          const int j = wi * 16 + __ffs(bits) - 1;
          bits &= bits - 1;
          if (!(f32(j) <= thr)) continue;
          double s = 0.0;
          for (int l = lane; l < d; l += 32) {
            const double diff = (double)ldf_any(yr + l) - c64[(size_t)j * d + l];
            s = fma(diff, diff, s);
          }
          for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          if (s < b64) { b64 = s; bi = j; }
        }
      }
    }
    if (lane == 0) {
      const int old = a.assign[row];
      if (!a.track) {
        a.assign[row] = bi;
      } else if (old != bi) {
        a.assign[row] = bi;
        const unsigned long long m = atomicAdd(a.counters, 1ull);
        a.moved[m] = (int32_t)row;
        a.moved[a.n + m] = old;
        a.moved[2 * a.n + m] = bi;
      }
    }
  }
}

// y -> y0 (and, for float32 features, y1 = bf16(y - y0)) in chunk-major layout
// [dp / 64][n][64] (zero padded), so that one TMA box of 128 rows x 64 elements is 16 KB of
// contiguous memory; the row norms the error bound needs, rounded up: (|y0|, |y - y0|) without
// y1, (|y|, 0) with it (float32 sums of squares inflated by their (d + 3) 2^-23 relative
// error bound); and max |y_il| for the fixed-point scale of the centroid sums.  One warp per row.
template <typename TY>
__global__ void split_rows_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d, int dp,
                                  __nv_bfloat16* __restrict__ y0, __nv_bfloat16* __restrict__ y1,
                                  float2* __restrict__ ynorm, float2* __restrict__ y2b,
                                  unsigned int* __restrict__ maxabs_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float infl = 1.0f + (float)(d + 3) * 1.1920928955078125e-7f;
  const float defl = 1.0f - (float)(d + 3) * 1.1920928955078125e-7f;
  float mx = 0.f;
  for (int64_t row = warp; row < n; row += nwarps) {
    float s0 = 0.f, s1 = 0.f;
    for (int l = 2 * lane; l < dp; l += 64) {
      const float v0 = l < d ? ldf_any(y + row * ldy + l) : 0.f;
      const float v1 = l + 1 < d ? ldf_any(y + row * ldy + l + 1) : 0.f;
      const float a0 = fabsf(v0), a1 = fabsf(v1);
      mx = (a0 <= 3.0e38f && a1 <= 3.0e38f) ? fmaxf(mx, fmaxf(a0, a1)) : INFINITY;  // NaN/inf -> inf
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      const float e0 = v0 - __low2float(h), e1 = v1 - __high2float(h);  // exact
      const size_t off = ((size_t)(l >> 6) * n + row) * kKC + (l & 63);
      *reinterpret_cast<__nv_bfloat162*>(y0 + off) = h;
      if (y1 != nullptr) {
        *reinterpret_cast<__nv_bfloat162*>(y1 + off) = __floats2bfloat162_rn(e0, e1);
        s0 = fmaf(v0, v0, fmaf(v1, v1, s0));
      } else {
        const float h0 = __low2float(h), h1 = __high2float(h);
        s0 = fmaf(h0, h0, fmaf(h1, h1, s0));
        s1 = fmaf(e0, e0, fmaf(e1, e1, s1));
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, off);
      s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if (lane == 0) {
      const float r = y1 != nullptr ? 0.0f : __fadd_ru(__fsqrt_ru(__fmul_ru(s1, infl)), 1e-30f);
      ynorm[row] = make_float2(__fsqrt_ru(__fmul_ru(s0, infl)), r);
      // |y|^2 is s0 (bfloat16 features are y0 exactly, s1 = 0), within (d + 3) 2^-23 relative
      y2b[row] = make_float2(__fmul_rd(s0, defl), __fmul_ru(s0, infl));
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) atomicMax(maxabs_bits, __float_as_uint(mx));
}

// split_rows_kernel with eight values per lane (16-byte loads and stores) and two rows in
// flight per warp, for rows_vec8 features; the same values, norms and bounds.  y0 == nullptr:
// norms and max |y| only (bfloat16 features that the distance pass reads in place).
template <typename TY>
__global__ void split_rows_vec_kernel(const TY* __restrict__ y, int64_t ldy, int64_t n, int d, int dp,
                                      __nv_bfloat16* __restrict__ y0, __nv_bfloat16* __restrict__ y1,
                                      float2* __restrict__ ynorm, float2* __restrict__ y2b,
                                      unsigned int* __restrict__ maxabs_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float infl = 1.0f + (float)(d + 3) * 1.1920928955078125e-7f;
  const float defl = 1.0f - (float)(d + 3) * 1.1920928955078125e-7f;
  const int groups = dp / 8;
  float mx = 0.f;
  for (int64_t r0 = warp; r0 < n; r0 += 2 * nwarps) {
    float s0[2] = {0.f, 0.f}, s1[2] = {0.f, 0.f};
    for (int g = lane; g < groups; g += 32) {
      const int l = 8 * g;
      float v[2][8];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t row = r0 + q * nwarps;
        if (row < n && l < d) {
          ld8(y + row * ldy + l, v[q]);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[q][e] = 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t row = r0 + q * nwarps;
        if (row >= n) continue;
        uint32_t h[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float v0 = v[q][2 * i], v1 = v[q][2 * i + 1];
          const float a0 = fabsf(v0), a1 = fabsf(v1);
          mx = (a0 <= 3.0e38f && a1 <= 3.0e38f) ? fmaxf(mx, fmaxf(a0, a1)) : INFINITY;  // NaN/inf -> inf
          const __nv_bfloat162 hb = __floats2bfloat162_rn(v0, v1);
          const float e0 = v0 - __low2float(hb), e1 = v1 - __high2float(hb);  // exact
          h[i] = *reinterpret_cast<const uint32_t*>(&hb);
          const __nv_bfloat162 lb = __floats2bfloat162_rn(e0, e1);
          lo[i] = *reinterpret_cast<const uint32_t*>(&lb);
          if (y1 != nullptr) {
            s0[q] = fmaf(v0, v0, fmaf(v1, v1, s0[q]));
          } else {
            const float h0 = __low2float(hb), h1 = __high2float(hb);
            s0[q] = fmaf(h0, h0, fmaf(h1, h1, s0[q]));
            s1[q] = fmaf(e0, e0, fmaf(e1, e1, s1[q]));
          }
        }
        const size_t off = ((size_t)(l >> 6) * n + row) * kKC + (l & 63);
        if (y0 != nullptr) *reinterpret_cast<uint4*>(y0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (y1 != nullptr) *reinterpret_cast<uint4*>(y1 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      for (int off = 16; off > 0; off >>= 1) {
        s0[q] += __shfl_xor_sync(0xffffffffu, s0[q], off);
        s1[q] += __shfl_xor_sync(0xffffffffu, s1[q], off);
      }
      const int64_t row = r0 + q * nwarps;
      if (lane == 0 && row < n) {
        const float r = y1 != nullptr ? 0.0f : __fadd_ru(__fsqrt_ru(__fmul_ru(s1[q], infl)), 1e-30f);
        ynorm[row] = make_float2(__fsqrt_ru(__fmul_ru(s0[q], infl)), r);
        y2b[row] = make_float2(__fmul_rd(s0[q], defl), __fmul_ru(s0[q], infl));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) atomicMax(maxabs_bits, __float_as_uint(mx));
}

// Row norms of bfloat16 features that the distance pass reads in place (rows_vec8, d a multiple
// of 64): ynorm = (|y|, 0) and y2b as in split_rows_kernel (y0 = y, no y1), and max |y_il| by
// integer maximum of the magnitude bits (inf or NaN give inf).  Eight values per lane, two rows
// in flight per warp.
__global__ void norms_bf16_kernel(const __nv_bfloat16* __restrict__ y, int64_t ldy, int64_t n, int d,
                                  float2* __restrict__ ynorm, float2* __restrict__ y2b,
                                  unsigned int* __restrict__ maxabs_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float infl = 1.0f + (float)(d + 3) * 1.1920928955078125e-7f;
  const float defl = 1.0f - (float)(d + 3) * 1.1920928955078125e-7f;
  const int groups = d / 8;
  uint32_t mb = 0;
  for (int64_t r0 = warp; r0 < n; r0 += 2 * nwarps) {
    float s0[2] = {0.f, 0.f};
    for (int g = lane; g < groups; g += 32) {
      uint4 raw[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t row = r0 + q * nwarps;
        raw[q] = row < n ? __ldg(reinterpret_cast<const uint4*>(y + row * ldy + 8 * g)) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint32_t w[4] = {raw[q].x, raw[q].y, raw[q].z, raw[q].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float lo = __uint_as_float(w[i] << 16), hi = __uint_as_float(w[i] & 0xFFFF0000u);
          s0[q] = fmaf(lo, lo, fmaf(hi, hi, s0[q]));
          mb = max(mb, max(w[i] & 0x7FFFu, (w[i] >> 16) & 0x7FFFu));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      for (int off = 16; off > 0; off >>= 1) s0[q] += __shfl_xor_sync(0xffffffffu, s0[q], off);
      const int64_t row = r0 + q * nwarps;
      if (lane == 0 && row < n) {
        ynorm[row] = make_float2(__fsqrt_ru(__fmul_ru(s0[q], infl)), 0.0f);
        y2b[row] = make_float2(__fmul_rd(s0[q], defl), __fmul_ru(s0[q], infl));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
  const float mx = mb >= 0x7F80u ? INFINITY : __uint_as_float(mb << 16);
  if (lane == 0) atomicMax(maxabs_bits, __float_as_uint(mx));
}

// Float64 centroids -> (c0, c1) bfloat16 rows [2][npad][dp] (zero padded), |c_j|^2 rounded to
// nearest, and max_j |c_j| rounded up.  One block per padded centroid row.
__global__ void split_centroids_kernel(const double* __restrict__ c64, int k, int d, int npad, int dp,
                                       __nv_bfloat16* __restrict__ cs, float* __restrict__ cn2,
                                       unsigned int* __restrict__ cmax_bits) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int l = threadIdx.x; l < dp; l += blockDim.x) {
    const double c = (j < k && l < d) ? c64[(size_t)j * d + l] : 0.0;
    const __nv_bfloat16 h0 = __double2bfloat16(c);
    const double r = c - (double)__bfloat162float(h0);  // exact
    cs[(size_t)j * dp + l] = h0;
    cs[((size_t)npad + j) * dp + l] = __double2bfloat16(r);
    s = fma(c, c, s);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0 && j < k) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cn2[j] = (float)t;
    atomicMax(cmax_bits, __float_as_uint(__double2float_ru(sqrt(t) * (1.0 + 1e-12))));
  }
}

// Hamerly's test after an update: u <- u + delta_a, l <- l - max_{j != a} delta_j (directed
// rounding; delta_j = st.cmove, the float64 movement of centroid j rounded up).  A row with
// u < l keeps its bounds and is skipped; the others are appended to sel (counters[3]), in row
// order within each block of kSelBlock rows (one atomic per block, not per warp: the counter
// is a single address).  k <= 256.
constexpr int kSelBlock = 1024;
__global__ void __launch_bounds__(kSelBlock)
    bounds_select_kernel(int64_t n, int k, const int32_t* __restrict__ assign, const float* __restrict__ cmove,
                         float2* __restrict__ bnd, int32_t* __restrict__ sel,
                         unsigned long long* __restrict__ counters) {
  __shared__ float mv[kCn2Slots];
  __shared__ float top2[2];
  __shared__ int top_j;
  __shared__ int wcount[kSelBlock / 32];
  __shared__ unsigned long long blk_base;
  for (int j = threadIdx.x; j < k; j += blockDim.x) mv[j] = cmove[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    float m0 = 0.f, m1 = 0.f;
    int j0 = 0;
    for (int j = 0; j < k; ++j) {
      const float v = mv[j];
      if (v > m0) { m1 = m0; m0 = v; j0 = j; }
      else if (v > m1) m1 = v;
    }
    top2[0] = m0;
    top2[1] = m1;
    top_j = j0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * kSelBlock;
  for (int64_t base = (int64_t)blockIdx.x * kSelBlock; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool eval = false;
    if (i < n) {
      const int a = assign[i];
      float2 b = bnd[i];
      b.x = __fadd_ru(b.x, mv[a]);
      b.y = __fsub_rd(b.y, a == top_j ? top2[1] : top2[0]);
      if (b.x < b.y) bnd[i] = b;
      else eval = true;
    }
    const unsigned m = __ballot_sync(0xffffffffu, eval);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    if (wid == 0) {
      // exclusive scan of the warp counts; one atomic for the block
      const int c = wcount[lane];
      int incl = c;
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
      }
      wcount[lane] = incl - c;
      if (lane == 31 && incl > 0) blk_base = atomicAdd(counters + 3, (unsigned long long)incl);
    }
    __syncthreads();
    if (eval) sel[blk_base + wcount[wid] + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    __syncthreads();
  }
}

// Rows the next pass evaluates: the selected ones, copied (y0, and y1 for float32 features; from
// the feature rows themselves when yrow is set) into
// the compact buffers in sel order when they are at most a fifth of the rows, else every row in
// place.  Writes counters[2] (rows) and counters[6] (compacted).  One warp per 128-byte chunk.
__global__ void compact_rows_kernel(int64_t n, int nk, int has_lo, const int32_t* __restrict__ sel,
                                    const __nv_bfloat16* __restrict__ ys, const __nv_bfloat16* __restrict__ yrow,
                                    int64_t ldy, __nv_bfloat16* __restrict__ yc,
                                    unsigned long long* __restrict__ counters) {
  const unsigned long long cnt = counters[3];
  const bool compact = cnt * 5 <= (unsigned long long)n;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counters[2] = compact ? cnt : (unsigned long long)n;
    counters[6] = compact ? 1ull : 0ull;
  }
  if (!compact) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int parts = 1 + has_lo;
  const int64_t total = (int64_t)cnt * nk * parts;
  const size_t half = (size_t)n * nk * kKC;  // elements of one split part
  for (int64_t w = warp; w < total; w += nwarps) {
    const int64_t s = w / (nk * parts);
    const int rem = (int)(w % (nk * parts));
    const int part = rem / nk, kc = rem % nk;
    const int64_t row = sel[s];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(
        yrow != nullptr ? yrow + row * ldy + (int64_t)kc * kKC : ys + part * half + ((size_t)kc * n + row) * kKC);
    uint32_t* dst = reinterpret_cast<uint32_t*>(yc + part * half + ((size_t)kc * n + s) * kKC);
    dst[lane] = __ldcs(src + lane);
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// 3-D bfloat16 map over the chunk-major split rows [nk][n][64], box 64 x 128 x 1, 128-byte swizzle.
bool encode_chunked(CUtensorMap* m, void* ptr, int64_t n, int nk) {
  EncodeTiled enc = encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)kKC, (cuuint64_t)n, (cuuint64_t)nk};
  const cuuint64_t strides[2] = {(cuuint64_t)kKC * 2, (cuuint64_t)n * kKC * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)kTM, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D bfloat16 map over rows x dp elements (leading dimension ld), box 64 x box_rows, 128-byte
// swizzle.
bool encode_rows(CUtensorMap* m, const void* ptr, int64_t rows, int dp, int box_rows, int64_t ld) {
  EncodeTiled enc = encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

TcPlan kmeans_tc_plan(int64_t n, int k, int d, int y_dtype) {
  TcPlan p;
  p.npad = (k + 15) / 16 * 16;
  p.dp = (d + kKC - 1) / kKC * kKC;
  p.nk = p.dp / kKC;
  // float32 features also stream y1 = bf16(y - y0): twice the bytes, but a 2^-16 instead of a
  // 2^-8 representation error, so far fewer rows need the exact decision
  p.has_lo = y_dtype == CSC_F32;
  p.stage_bytes = kChunkA * (1 + p.has_lo);
  p.b_bytes = 2u * (uint32_t)p.nk * (uint32_t)p.npad * 128u;
  const int fixed = 1024 + 8 * (2 * kMaxStages + 6) + 16 + 4 * 256;
  const int room = kMaxDynSmem - fixed - (int)p.b_bytes;
  p.stages = room > 0 ? std::min(kMaxStages, room / (int)p.stage_bytes) : 0;
  p.smem = 1024 + p.b_bytes + (size_t)p.stages * p.stage_bytes + 8 * (2 * p.stages + 6) + 16 + 4 * kCn2Slots;
  p.tmem_cols = 32;
  while (p.tmem_cols < (uint32_t)(2 * p.npad)) p.tmem_cols <<= 1;
  p.nv = 16;
  while (p.nv < p.npad && p.nv < 128) p.nv <<= 1;
  p.ok = k >= 1 && p.npad <= 256 && p.stages >= 3 && n >= 1 && encoder() != nullptr;
  const int ni = (p.dp / 16) * (2 + p.has_lo);  // MMA instructions accumulated into each output
  // dropped terms per |y| cmax (with y1: y1 c1, y0 ec, ey c; without: y0 ec, the ey term being
  // carried by |y - y0| in the kernel) plus the accumulation bound
  const double dropped = p.has_lo ? 3.02 : 1.001;
  p.kdot = (float)(dropped * std::ldexp(1.0, -16) + (ni + 1) * std::ldexp(1.0, -21) * 1.04);
  return p;
}

cudaError_t kmeans_tc_prepare(KmeansState& st, const TcPlan& p, const void* y, int y_dtype, int64_t n,
                              int d, int64_t ldy, unsigned int* maxabs_bits, cudaStream_t s) {
  // bfloat16 features whose rows are whole 64-element chunks are their own y0: the distance pass
  // reads them in place through a 2-D map, and only the norms are computed here
  const bool rowmajor = y_dtype == CSC_BF16 && d % kKC == 0 && rows_vec8(y, d, ldy);
  st.tc_rowmajor = rowmajor;
  const size_t half = (size_t)n * p.dp * 2;
  if ((!rowmajor && !ensure(st.ysplit, half * (1 + p.has_lo))) || !ensure(st.ynorm, (size_t)n * 8) ||
      !ensure(st.csplit, (size_t)2 * p.npad * p.dp * 2) || !ensure(st.cn2t, (size_t)p.npad * 4) ||
      !ensure(st.masks, (size_t)n * (p.npad / 16) * 2) || !ensure(st.y2b, (size_t)n * 8) ||
      !ensure(st.bnd, (size_t)n * 8) || !ensure(st.hsel, (size_t)n * 4) ||
      !ensure(st.ycomp, half * (1 + p.has_lo)))
    return cudaErrorMemoryAllocation;
  __nv_bfloat16* y0 = rowmajor ? nullptr : as<__nv_bfloat16>(st.ysplit);
  __nv_bfloat16* y1 = p.has_lo ? y0 + (size_t)n * p.dp : nullptr;
  const int grid = num_sms() * 8;
  if (rowmajor) {
    norms_bf16_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(y), ldy, n, d, as<float2>(st.ynorm),
                                           as<float2>(st.y2b), maxabs_bits);
  } else if (rows_vec8(y, d, ldy)) {
    if (y_dtype == CSC_BF16)
      split_rows_vec_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(y), ldy, n, d,
                                                                p.dp, y0, y1, as<float2>(st.ynorm),
                                                                as<float2>(st.y2b), maxabs_bits);
    else
      split_rows_vec_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(y), ldy, n, d, p.dp, y0, y1,
                                                        as<float2>(st.ynorm), as<float2>(st.y2b), maxabs_bits);
  } else if (y_dtype == CSC_BF16)
    split_rows_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(y), ldy, n, d,
                                                          p.dp, y0, y1, as<float2>(st.ynorm),
                                                          as<float2>(st.y2b), maxabs_bits);
  else
    split_rows_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(y), ldy, n, d, p.dp, y0, y1,
                                                  as<float2>(st.ynorm), as<float2>(st.y2b), maxabs_bits);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(st.tmaps);
  __nv_bfloat16* c0 = as<__nv_bfloat16>(st.ycomp);
  __nv_bfloat16* c1 = p.has_lo ? c0 + (size_t)n * p.dp : c0;
  const bool ymaps = rowmajor ? encode_rows(&maps[0], y, n, d, kTM, ldy) && encode_rows(&maps[1], y, n, d, kTM, ldy)
                              : encode_chunked(&maps[0], y0, n, p.nk) &&
                                    encode_chunked(&maps[1], p.has_lo ? (void*)y1 : (void*)y0, n, p.nk);
  if (!ymaps || !encode_rows(&maps[2], st.csplit.ptr, 2 * (int64_t)p.npad, p.dp, p.npad, p.dp) ||
      !encode_chunked(&maps[3], c0, n, p.nk) || !encode_chunked(&maps[4], c1, n, p.nk))
    return cudaErrorInvalidValue;
  const void* fn = p.nv == 16   ? (const void*)kmeans_tc_kernel<16>
                   : p.nv == 32 ? (const void*)kmeans_tc_kernel<32>
                   : p.nv == 64 ? (const void*)kmeans_tc_kernel<64>
                                : (const void*)kmeans_tc_kernel<128>;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
}

cudaError_t kmeans_tc_pass(KmeansState& st, const TcPlan& p, const void* y, int y_dtype, int64_t n, int d,
                           int64_t ldy, int k, int track, bool select, cudaStream_t s) {
  unsigned int* cmax_bits = as<unsigned int>(st.bits) + 3;
  cudaError_t e = cudaMemsetAsync(cmax_bits, 0, 4, s);
  if (e != cudaSuccess) return e;
  unsigned long long* counters = as<unsigned long long>(st.counters);
  if (select) {
    const int64_t blocks = std::min<int64_t>((n + kSelBlock - 1) / kSelBlock, (int64_t)num_sms() * 2);
    bounds_select_kernel<<<(int)blocks, kSelBlock, 0, s>>>(n, k, as<int32_t>(st.assign), as<float>(st.cmove),
                                                     as<float2>(st.bnd), as<int32_t>(st.hsel), counters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    compact_rows_kernel<<<num_sms() * 8, 256, 0, s>>>(
        n, p.nk, p.has_lo, as<int32_t>(st.hsel), as<__nv_bfloat16>(st.ysplit),
        st.tc_rowmajor ? static_cast<const __nv_bfloat16*>(y) : nullptr, ldy, as<__nv_bfloat16>(st.ycomp), counters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  split_centroids_kernel<<<p.npad, 128, 0, s>>>(as<double>(st.c64), k, d, p.npad, p.dp,
                                                  as<__nv_bfloat16>(st.csplit), as<float>(st.cn2t), cmax_bits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  TcArgs a{};
  a.n = n;
  a.k = k;
  a.npad = p.npad;
  a.nk = p.nk;
  a.stages = p.stages;
  a.track = track;
  a.has_lo = p.has_lo;
  a.tmem_cols = p.tmem_cols;
  a.acc_off = p.tmem_cols / 2;
  a.stage_bytes = p.stage_bytes;
  a.b_bytes = p.b_bytes;
  a.kdot = p.kdot;
  a.ynorm = as<float2>(st.ynorm);
  a.cn2 = as<float>(st.cn2t);
  a.cmax_bits = cmax_bits;
  a.assign = as<int32_t>(st.assign);
  a.flagged = as<int32_t>(st.flagged);
  a.masks = as<uint16_t>(st.masks);
  a.moved = as<int32_t>(st.moved);
  a.counters = counters;
  a.sel = select ? as<int32_t>(st.hsel) : nullptr;
  a.rowmajor = st.tc_rowmajor;
  a.y2b = as<float2>(st.y2b);
  a.bnd = as<float2>(st.bnd);
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(st.tmaps);
  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int grid = (int)std::min<int64_t>(num_sms(), ntiles);
  switch (p.nv) {
    case 16: kmeans_tc_kernel<16><<<grid, kThreads, p.smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a); break;
    case 32: kmeans_tc_kernel<32><<<grid, kThreads, p.smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a); break;
    case 64: kmeans_tc_kernel<64><<<grid, kThreads, p.smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a); break;
    default: kmeans_tc_kernel<128><<<grid, kThreads, p.smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the float32 centroids, their norms and max |c32| come from the last finalize
  const float* c32 = as<float>(st.c32);
  const float* cn2_32 = as<float>(st.cn2);
  const unsigned int* cmax32 = as<unsigned int>(st.bits);
  if (y_dtype == CSC_BF16)
    tc_refine_kernel<__nv_bfloat16><<<num_sms() * 4, 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(y), ldy, d, c32, cn2_32, cmax32, as<double>(st.c64), a);
  else
    tc_refine_kernel<float><<<num_sms() * 4, 256, 0, s>>>(static_cast<const float*>(y), ldy, d, c32, cn2_32,
                                                         cmax32, as<double>(st.c64), a);
  return cudaGetLastError();
}

void kmeans_tc_release(KmeansState& st) {
  release(st.ysplit);
  release(st.ynorm);
  release(st.csplit);
  release(st.cn2t);
  release(st.masks);
  release(st.y2b);
  release(st.bnd);
  release(st.hsel);
  release(st.ycomp);
}

}  // namespace csc
