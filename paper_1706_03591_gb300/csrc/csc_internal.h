// Internal declarations shared by the CUDA translation units of libcsc.
// Not part of the ABI (see include/csc.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/csc.h"

namespace csc {

// ------------------------------------------------------------------ device buffers

// Grow-only device allocation owned by a context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Returns false (and leaves the buffer empty) when cudaMalloc fails.
bool ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);

template <typename T>
inline T* as(DevBuf& b) { return static_cast<T*>(b.ptr); }

#ifdef __CUDACC__
// Eight consecutive feature values as float through the read-only path: one 16-byte load of
// bfloat16, two of float32.  p must be 16-byte aligned.
__device__ __forceinline__ void ld8(const __nv_bfloat16* p, float (&v)[8]) {
  const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
#endif

// Whether rows of features can be read eight values at a time (ld8): d and the leading
// dimension multiples of 8, base 16-byte aligned.
inline bool rows_vec8(const void* y, int64_t d, int64_t ldy) {
  return d % 8 == 0 && ldy % 8 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0;
}

// ------------------------------------------------------------------ graph state

struct Graph {
  int64_t n = 0, nnz = 0;
  bool weighted = false;
  DevBuf row_ptr;   // int64[n+1]
  DevBuf col;       // int32[nnz]
  DevBuf val;       // float[nnz] (weighted only)
  DevBuf scale;     // float[n], D^{-1/2} (0 for isolated nodes)
  DevBuf vs;        // float[n], row scale of the value-free recursion: D^{-1/2}, 1 if isolated
  DevBuf ivs;       // float[n], 1 / vs
  DevBuf deg;       // double[n]
  DevBuf blk_row;   // int32[nblk+1], edge-block partition of the rows (batched kernel)
  DevBuf srow;      // int32[nsblk+1], weight-balanced row blocks of the step kernels
  bool loaded = false;
  // Internal node order (csc_opts.reorder): internal row i holds caller row perm[i] (degrees
  // descending, ties by caller id), its neighbours in the caller's order with the ids mapped
  // through iperm; the caller's CSR stays on the device beside it.
  bool permuted = false;
  DevBuf perm;      // int32[n]: internal row -> caller row
  DevBuf iperm;     // int32[n]: caller row -> internal row
  DevBuf urp;       // int64[n+1]: caller row offsets
  DevBuf ucol;      // int32[nnz]: caller column indices
  DevBuf uval;      // float[nnz]: caller edge weights (weighted graphs)
  std::vector<int32_t> h_perm, h_iperm;
};

// Row blocks of the step kernels: a row weighs its stored edges plus kRowCost (its own
// streams), and block b starts at the first row whose cumulative weight reaches b * kBlockWeight.
constexpr int kRowCost = 4;
constexpr int kBlockWeight = 4096;
int row_blocks(int64_t n, int64_t nnz);

// Target number of stored edges per block of the recursion kernels (staged in shared memory).
constexpr int kEdgesPerBlock = 2048;
// Shared-memory capacity of a staged block: a block whose edge span or row count exceeds
// these is processed directly from global memory.
constexpr int kEdgeBuf = 3072;
constexpr int kRowBuf = 512;
int edge_blocks(int64_t nnz);

// ------------------------------------------------------------------ launch helpers

int num_sms();
int grid_for(const void* kernel, int block, size_t smem = 0);

// a[0..m]: Jackson-damped Chebyshev coefficients of the low-pass of cutoff lambda_c
// (Section 3.3), shared by every entry point that filters.
void filter_coeffs(int m, double lambda_c, double* a);

// ------------------------------------------------------------------ graph kernels (graph.cu)

cudaError_t launch_graph_prep(const Graph& g, cudaStream_t s);
// Internal CSR of g from its caller CSR (urp/ucol/uval) and perm/iperm (g.deg is used as
// scratch); deg_tmp: int64[n] scratch, sums: scan_sums_len(n) int64 scratch.
cudaError_t launch_permute_graph(Graph& g, long long* deg_tmp, long long* sums, cudaStream_t s);
// dst[i] = src[map[i]] for i < n (int32 vectors).
cudaError_t launch_gather_i32(int32_t* dst, const int32_t* src, const int32_t* map, int64_t n, cudaStream_t s);
// Edge values of the internal CSR scattered to the caller's edge order: dst[urp[perm[i]] + k] =
// src[row_ptr[i] + k].
cudaError_t launch_scatter_edges(const Graph& g, const float* src, float* dst, cudaStream_t s);
// Computes g.blk_row (edge_blocks(g.nnz) + 1 entries) and g.srow (row_blocks(g.n, g.nnz) + 1).
cudaError_t launch_block_rows(const Graph& g, cudaStream_t s);
// Device-side CSR validation; writes the number of violations into *bad (device int64).
cudaError_t launch_graph_check(const Graph& g, unsigned long long* bad, cudaStream_t s);

// ------------------------------------------------------------------ signals (signals.cu)

// Fills an n x w block (leading dimension w) of tile columns [col0, col0 + valid) of the
// Philox N(0, 1/d) signals; columns >= valid are zero.  dtype CSC_F32 / CSC_BF16.
// rowid (nullptr: identity): the Philox row counter of output row i is rowid[i].
cudaError_t launch_signals(void* out, int dtype, int64_t n, int w, int64_t ld, uint64_t seed,
                           int64_t col0, int valid, float inv_sqrt_d, cudaStream_t s,
                           const int32_t* rowid = nullptr);
// Copies columns [c0, c0 + valid) of a caller block (n x ld_src, dtype) into an n x w
// tile buffer of the same dtype, zero-filling columns >= valid; row i of the tile is row
// src_row[i] of the caller block (nullptr: row i).
cudaError_t launch_copy_tile(void* dst, const void* src, int dtype, int64_t n, int w,
                             int64_t ld_src, int c0, int valid, cudaStream_t s,
                             const int32_t* src_row = nullptr);

// ------------------------------------------------------------------ Chebyshev recursion (cheb.cu)

struct StepArgs {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const float* val;     // nullptr: unit weights
  const float* scale;   // D^{-1/2} (first step's per-edge weights)
  const float* vs;      // row scale of the stored blocks V_j = vs * T_j (j >= 1)
  const float* ivs;     // 1 / vs
  const int32_t* blk_row;  // edge-block partition (nblk + 1)
  int nblk;
  const int32_t* srow;  // weight-balanced row blocks of the step kernels (nsblk + 1)
  int nsblk;
  int l2pf;             // prefetch the next batch of gathered rows into L2 (set by launch_cheb_step)
  int tp_unscaled;      // 1: tp holds T_{j-1} (step 2 reads T_0 = R), 0: tp holds V_{j-1}
  const void* tg;       // gathered block T_j (n x w)
  const void* tp;       // T_{j-1} (own rows), unused on the first step
  float* tn;            // T_{j+1} (n x w)
  float* psi;           // Psi rows base (nullptr: moments only)
  int64_t ldp;          // Psi leading dimension
  const float* coef;    // device coefficients a_0..a_m (float32)
  int j;                // this step produces T_{j+1}
  double* part;         // block partial sums of this step, [nq][grid]
  int w;                // tile width (= 4 * lanes per row)
};

// First step: T_1 = L~ T_0 (stored as V_1 = vs T_1), Psi = a_0 T_0 + a_1 T_1,
// partials {<T0,T0>, <T1,T1>, <T1,T0>}.
cudaError_t launch_cheb_first(const StepArgs& a, int t0_dtype, int grid, cudaStream_t s);
// General step on the stored blocks V_j = vs T_j:
// V_{j+1} = -2 vs_i^2 sum_e w_e V_j[col_e] - V_{j-1}, Psi += a_{j+1} T_{j+1}, partials
// {<T_{j+1},T_{j+1}>, <T_{j+1},T_j>}.  tp_dtype is the storage type of tp.
cudaError_t launch_cheb_step(const StepArgs& a, int tp_dtype, int grid, cudaStream_t s);
int cheb_grid(int w);

// One column tile of one graph in a batched filtering launch.
struct BatchTile {
  StepArgs a;           // graph and tile pointers; tg/tp/tn/j/part/tp_unscaled set per step
  void* buf[3];         // rotating n x w blocks; buf[0] holds T_0 (dtype t0_dtype)
  int t0_dtype;
  int lpr;              // w / 4
  int64_t blk0;         // index of this tile's first edge block in the flat item list
  double* mom;          // [2m+1] trace sums of the graph (E/F rows), float64 atomics
  uint64_t seed;        // signal stream of the graph
  int64_t col0;         // global column id of this tile's first column
  int valid;            // real columns in this tile (the rest are zero padding)
  float inv_sqrt_d;
};

// item_tile[i] = tile of flat edge-block item i.
// Persistent cooperative launch over the item list: items [wave_end[w-1], wave_end[w]) run all
// m + 1 steps (signals, first step, m - 1 general steps); claim_end[w] is the cumulative number
// of (step, item) claims up to wave w.  work (one zeroed counter) hands out the claims; done
// ([tiles][m + 1], zeroed) counts the finished items of every tile and step; *err is set when a
// bounded dependency wait runs out.
cudaError_t launch_cheb_batched(const BatchTile* tiles, const int32_t* item_tile, const int64_t* wave_end,
                                const int64_t* claim_end, int nwaves, int m, unsigned long long* work,
                                unsigned int* done, int* err, int grid, cudaStream_t s);
int cheb_batched_grid();
// Sums partials[(q * nslots + slot) * grid + b] over b (fixed order) into out[q * nslots + slot]
// for q in 0..nq-1, accumulating across `tiles` consecutive partial blocks of stride tile_stride.
cudaError_t launch_reduce_partials(const double* part, int nrows, int grid, int tiles,
                                   int64_t tile_stride, double* out, cudaStream_t s);

// ------------------------------------------------------------------ features (features.cu)

// Splice + row normalisation: for each row, ring slot q takes psi[row*ldp + src[q]] when
// src[q] >= 0 (and is written back to theta), else keeps theta; y = theta / ||theta||.
cudaError_t launch_assemble(float* theta, int64_t ldt, const float* psi, int64_t ldp,
                            const int* src, int d, void* y, int y_dtype, int64_t ldy, int64_t n,
                            cudaStream_t s);
// Copies an n x d block (src dtype float or bf16, ld_src) to dst (dtype, ld_dst) on device.
// Row i of dst is row src_row[i] of src (nullptr: row i).
cudaError_t launch_convert(const void* src, int src_dtype, int64_t ld_src, void* dst,
                           int dst_dtype, int64_t ld_dst, int64_t n, int d, cudaStream_t s,
                           const int32_t* src_row = nullptr);

// ------------------------------------------------------------------ differentiation (grad.cu)

// State kept by csc_filter_forward for csc_filter_vjp.
struct GradState {
  bool ready = false;
  int m = 0, c = 0, w = 0, ntiles = 0, stride = 1, segs = 1;
  const float* R = nullptr;   // the context's copy of the signal block (n x c)
  int64_t ldr = 0;
  DevBuf rcopy;
  std::vector<double> coef;   // a_0 .. a_m
  DevBuf coef_f;              // float[m + 1]
  DevBuf ckpt;                // float [ntiles][slots][n][w]: V_j at the segment boundaries
  int slots = 0;              // checkpoint blocks per tile
  DevBuf seg;                 // float [stride + 2][n][w]: one recomputed segment
  DevBuf rt, gt;              // float [n][w]: tile of R, tile of dloss/dPsi
  DevBuf phi[3];              // float [n][w]: adjoint iterates Phi_j = D^-1/2 Lambda_j
  DevBuf H;                   // float [nnz]: sum_j c_j <Phi_{j+1}[u], V_j[v]> per stored entry
  DevBuf tpos;                // int32 [nnz]: position of the transposed entry
  DevBuf nsum;                // double [n]: per-node sums of the weight chain
  DevBuf part;                // double block partials of <dloss/dPsi, T_j>
  DevBuf ga;                  // double [m + 1][ntiles]: per-tile <dloss/dPsi, T_j R>
  DevBuf flag;                // int64: entries without a transposed partner
  DevBuf gw_stage;            // float [nnz]: edge gradients in the internal edge order
  int64_t graph_version = -1; // graph the transpose map was built for
};

// ------------------------------------------------------------------ compressive k-means (compressive.cu)

// Scratch of csc_compressive_cluster (Section 2.2, step 2).
struct CompressiveState {
  DevBuf s;                     // double [n]: row energies |theta_i|^2
  DevBuf q, prefix;             // int64 [n]: quantised weights and their inclusive prefix sums
  DevBuf flags, pos;            // int32 [n]: drawn-node flags and their inclusive prefix sums
  DevBuf sums;                  // chunk totals of the scans
  DevBuf omega;                 // int32 [min(n, draws)]: sampled nodes in increasing order
  DevBuf smax;                  // uint64: bits of max_i s_i
  DevBuf yo;                    // [n_omega][d]: rows of the sampled nodes
  DevBuf labels;                // int32 [restarts][n_omega]: reduced assignment of each restart
  DevBuf z, x;                  // float [n][k] right-hand side, float [n][cpad] interpolation
  DevBuf assign;                // int32 [n]
  DevBuf theta_stage, y_stage;  // caller features staged from host memory
};
// Row energies, integer weights and prefix sums, the draws and the sorted sample; the
// sample size is pos[n - 1] and the weight total prefix[n - 1] (device).
cudaError_t compressive_sample(CompressiveState& cs, const float* theta, int64_t ld, int64_t n, int d,
                               int64_t n_draws, uint64_t seed, cudaStream_t s);
// out[r] = y[omega[r]] for r < no (n_omega x d, leading dimension d, dtype of y).
cudaError_t compressive_gather(const void* y, int y_dtype, int64_t ldy, const int32_t* omega, int64_t no, int d,
                               void* out, cudaStream_t s);
// z[omega[r]][labels[r]] = T / (n q) for the sampled nodes (z zeroed by the caller).
cudaError_t compressive_rhs(const CompressiveState& cs, const int32_t* labels, int64_t no, int64_t n, float* z,
                            int64_t ldz, cudaStream_t s);
// out[i] = lowest index of the maximum of row i of x (k columns).
int64_t scan_sums_len(int64_t n);
cudaError_t inclusive_scan_i64(const long long* in, long long* out, int64_t n, long long* sums, cudaStream_t s);
cudaError_t compressive_argmax(const float* x, int64_t ldx, int64_t n, int k, int32_t* out, cudaStream_t s);
void compressive_release(CompressiveState& cs);

// ------------------------------------------------------------------ k-means (kmeans.cu)

struct KmeansState {
  DevBuf c64, c32, cn2;         // centroids float64 [k][d], float32 [k][d], |c32|^2 [k]
  DevBuf cmove;                 // float [k], movement of each centroid in the last update
  DevBuf bits;                  // uint32 [4]: max |c| and max movement (float bits), max |y|
  DevBuf sums, counts;          // fixed-point int64 [k][d], int32 [k]
  DevBuf assign;                // int32 [n]
  DevBuf ub, lbk;               // float [n], [n][k]: distance bounds (pruning)
  DevBuf vstamp;                // int32 [n]: centroid version the bounds of a row refer to
  DevBuf drift;                 // float [passes][k]: movement bound since each version
  DevBuf work, flagged, moved;  // int32 [n], [n], [3][n]
  DevBuf counters;              // unsigned long long [4]: moved, flagged, work
  DevBuf inertia_part;          // double [grid + 1]
  DevBuf init_idx;              // int64 [k]
  DevBuf perm, hist;            // int32 [n] rows bucketed by cluster, int32 [blocks][k]
  // tensor-core distance pass
  DevBuf ysplit, ynorm;         // bfloat16 [1 or 2][dp / 64][n][64] (y0, y1), float2 [n] row norms
  DevBuf csplit, cn2t;          // bfloat16 [2][npad][dp] (c0, c1), float [npad] |c|^2
  DevBuf masks;                 // uint16 [n][npad / 16] candidate masks of near-tie rows
  DevBuf y2b;                   // float2 [n]: |y|^2 rounded down and up
  DevBuf bnd;                   // float2 [n]: Hamerly bounds (upper to the own centroid, lower to the others)
  DevBuf hsel;                  // int32 [n]: rows whose bounds do not certify their centroid
  DevBuf ycomp;                 // bfloat16, the layout of ysplit: those rows, compacted
  bool tc_rowmajor = false;     // bfloat16 features read in place by the distance pass (no ysplit)
  alignas(64) unsigned char tmaps[5][128];  // TMA maps of y0, y1, (c0, c1), compacted y0, y1
  unsigned long long* hist_host = nullptr;   // pinned [passes][5]: counters of each pass
  size_t hist_cap = 0;
  cudaEvent_t pass_ev[3] = {nullptr, nullptr, nullptr};  // completion of a pass's counter copy
};

// Shape of the tensor-core distance pass for (n, k, d, dtype); ok = false when k or d
// do not fit its shared-memory plan (the bound-pruned pass is used instead).
struct TcPlan {
  int npad = 0, dp = 0, nk = 0, stages = 0, has_lo = 0, nv = 16;
  uint32_t stage_bytes = 0, b_bytes = 0, tmem_cols = 0;
  size_t smem = 0;
  float kdot = 0.f;
  bool ok = false;
};
TcPlan kmeans_tc_plan(int64_t n, int k, int d, int y_dtype);
// Splits the features into bfloat16 y0 (and y1), computes their row norms, max |y_il| (atomicMax into the
// float bits at maxabs_bits, which the caller zeroes) and the TMA maps (once per call).
cudaError_t kmeans_tc_prepare(KmeansState& st, const TcPlan& p, const void* y, int y_dtype, int64_t n,
                              int d, int64_t ldy, unsigned int* maxabs_bits, cudaStream_t s);
// One assignment pass against the float64 centroids in st.c64: counters[0] moves (recorded in
// st.moved when track), counters[1] near-tie rows, counters[2] rows the pass evaluated (when
// select), counters[4] error word (a wait expired).  Every evaluated row leaves Hamerly bounds
// in st.bnd.  select: rows whose bounds, moved by the centroid drift of the last update
// (st.cmove), certify their centroid are skipped; the pass evaluates the others (compacted
// when they are at most a fifth of the rows, else all rows).
cudaError_t kmeans_tc_pass(KmeansState& st, const TcPlan& p, const void* y, int y_dtype, int64_t n, int d,
                           int64_t ldy, int k, int track, bool select, cudaStream_t s);
void kmeans_tc_release(KmeansState& st);

struct KmeansResult {
  int iters = 0;
  bool converged = false;
  int64_t decided = 0;         // rows decided by the distance pass over all passes (pruning stats)
  double inertia = 0.0;
  int32_t* assign = nullptr;   // device pointer to the final assignment (inside the state)
  int64_t launches = 0;        // kernels launched
  int64_t near_ties = 0;       // rows re-decided exactly, summed over passes
};

// Runs Lloyd's iteration on device features y (n x d, leading dimension ldy, dtype).
// init_idx: host int64[k]; prev_assign: device int32[n] or nullptr.
csc_status kmeans_run(KmeansState& st, const void* y, int y_dtype, int64_t n, int d, int64_t ldy,
                      int k, const int64_t* init_idx, const int32_t* prev_assign, int max_iter,
                      cudaStream_t s, KmeansResult* res, std::string* err);
void kmeans_release(KmeansState& st);

}  // namespace csc

// Library context (opaque to callers; see include/csc.h).
struct csc_ctx {
  csc_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  csc::Graph g;
  int64_t graph_version = 0;  // incremented by every csc_set_graph
  // filtering
  csc::DevBuf tbuf[3];
  csc::DevBuf psi;
  csc::DevBuf part;
  csc::DevBuf ef;          // reduced E/F sums, double[2m+1]
  csc::DevBuf coef;        // float[m+1]
  csc::DevBuf rstage;      // caller signal block staged on the device
  std::vector<double> mu;
  int last_m = 0;
  // feature ring (Eq. 6)
  int64_t ring_n = 0;
  int ring_d = 0;
  csc::DevBuf theta;       // float n x d
  csc::DevBuf y;           // n x d, float or bf16 (row-normalised features)
  csc::DevBuf slot_src;    // int[d]
  std::vector<int64_t> stamp;
  int64_t t = 0;
  int64_t next_id = 0;
  bool has_lambda = false;
  double lambda = 0.0;
  double rho_since = 0.0;  // edge distance summed since the last eigencount check
  // k-means
  csc::KmeansState km;
  csc::DevBuf prev_assign;
  int prev_k = 0;
  bool has_prev = false;
  bool grouped = false;    // reorder = 2: rows grouped by an assignment
  csc::DevBuf ystage;      // caller features staged on the device
  csc::DevBuf astage;      // caller assignment staged on the device
  csc::DevBuf out_stage;   // conversions before a host copy
  csc::DevBuf bad;         // CSR violation counter
  csc::DevBuf gtmp;        // set_graph scratch: int64 [n] + scan sums
  // counters (csc_get_stats)
  int64_t launches = 0, step_launches = 0, filter_passes = 0;
  double step_ms = 0.0;
  double step_bytes = 0.0;  // algorithmic bytes of the timed step launches
  int last_tile = 0;
  std::vector<cudaEvent_t> events;  // timing event pairs, one per column tile
  // batched filtering (batched.cu)
  csc::DevBuf b_prep, b_tbuf, b_psi, b_coef, b_mom, b_tiles, b_items, b_bar, b_tune, b_part;
  csc::DevBuf b_waves;  // int64 [waves]: end of each wave in the item list
  csc::GradState gs;    // differentiation: checkpoints of the last csc_filter_forward
  csc::DevBuf sim;      // csc_laplacian_distance scratch: double [2n + 2 grid + 8]
  csc::CompressiveState cmp;  // csc_compressive_cluster scratch
  csc::DevBuf b_work;   // uint64 claim counter, int64 [waves] claim ends, uint32 [tiles][m + 1] done counts
  cudaStream_t b_cap = nullptr;
  cudaGraphExec_t b_exec = nullptr;
  std::vector<uint64_t> b_sig;              // launch signature of b_exec
  std::map<uint64_t, int> tune;             // size class -> column tile
  int64_t batched_launches = 0, graph_replays = 0, autotune_trials = 0, batched_waves = 0;
  int64_t kmeans_passes = 0, kmeans_near_ties = 0, kmeans_rows = 0;
};

