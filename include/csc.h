/*
 * csc.h -- C ABI of the GB300 (sm_103a) dynamic compressive spectral clustering library.
 *
 * Method: Martin, Loukas, Vandergheynst, "Fast Approximate Spectral Clustering for
 * Dynamic Networks" (ICML 2017, arXiv:1706.03591).  The calls follow the paper's
 * statement of the problem (Algorithm 1: a graph sequence G_t, the number of
 * signals d, the reuse fraction p and k in; assignments X_t out):
 *
 *   csc_set_graph        G_t as CSR                                  Section 2.1, Section 4
 *   csc_estimate_lambda_k  eigencount dichotomy for the cutoff       Section 3.3, Algorithm 1
 *   csc_filter           Jackson-damped Chebyshev filtering of the    Section 2.2, Section 3.3,
 *                        new signals, eigencount check, refinement,   Eq. 6, Algorithm 1, Section 4.1
 *                        splice into the feature matrix Theta_t
 *   csc_cluster          row normalisation + k-means on Theta_t       Eq. 1, Eq. 5, Algorithm 1
 *
 * plus stateless-per-call building blocks used by tests and benchmarks
 * (csc_signals, csc_cheb_filter, csc_kmeans) and host-only helpers that need
 * no GPU (coefficients, eigencount from moments, the dichotomy).
 *
 * Conventions (every entry point):
 *  - Returns a csc_status; no exception or abort crosses the ABI.  Details of the
 *    last failure on a context are in csc_last_error(ctx).
 *  - `where` arguments say where a caller pointer lives: CSC_HOST (pageable or
 *    pinned host memory) or CSC_DEVICE (device memory of the context's device).
 *  - The library owns every device buffer it allocates (graph copy, recursion
 *    blocks, feature ring, k-means state).  Caller buffers are only read or
 *    written during the call; output buffers are caller-owned.
 *  - All device work runs on the stream given to csc_create (NULL = legacy
 *    default stream).  Calls that return host values synchronise that stream.
 *  - A context is not thread-safe; use one context per host thread.
 *  - Layouts are row-major: an n x c block with leading dimension ld has
 *    element (i, v) at base[i*ld + v].
 */
#ifndef CSC_H
#define CSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSC_ABI_VERSION 9

typedef struct csc_ctx csc_ctx;

typedef enum csc_status {
  CSC_OK = 0,
  CSC_EINVAL = 1,   /* invalid argument (sizes, pointers, malformed CSR, unknown enum) */
  CSC_ENOMEM = 2,   /* a device or host allocation failed */
  CSC_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  CSC_ETIMEOUT = 4, /* a bounded device-side wait expired */
  CSC_ESTATE = 5,   /* call order: e.g. csc_filter before csc_set_graph */
  CSC_ELIMIT = 6    /* a size is beyond the fixed limit of csc_cheb_filter_noalloc */
} csc_status;

enum { CSC_HOST = 0, CSC_DEVICE = 1 };
enum { CSC_F32 = 0, CSC_BF16 = 1 };

typedef struct csc_opts {
  int precision;    /* CSC_F32: signal block and features stored in float32.
                       CSC_BF16: signal block R and row-normalised features stored in
                       bfloat16; the recursion and accumulation stay float32 and the
                       eigencount trace sums and centroid sums exact/float64. */
  double count_tol; /* eigencount acceptance half-width tau; <= 0 selects
                       max(0.5, 2 sqrt(2k/c)) for a block of c signals */
  int max_bisect;   /* cap on eigencount evaluations of the dichotomy (default 30) */
  int max_iter;     /* cap on Lloyd assignment passes (default 100) */
  int col_tile;     /* column-tile width of the recursion: 0 = automatic (tiles of 8, 16, 32
                       and 64 columns minimising sum (8 + w) over the tiles that cover the
                       columns), else one of 8, 16, 32, 64, 128 for every tile */
  int checked;      /* nonzero: validate the CSR on csc_set_graph (device input too) */
  int timing;       /* nonzero: time the Chebyshev step launches with CUDA events on the
                       context stream (read with csc_get_stats) */
  int estimator;    /* eigencount of the cutoff search: 0 = (d/c) ||h(L) R||_F^2, which
                       estimates tr h(L)^2 (default); 1 = (d/c) tr(R^T h(L) R), which
                       estimates tr h(L) (Hutchinson) */
  int reorder;      /* 1 (default): the library stores the graph in its own node order,
                       degrees descending (ties by node id), so that the rows a block of the
                       recursion handles have similar degrees and the most gathered rows are
                       contiguous; the order is fixed at the first csc_set_graph of a feature
                       ring.  2: the same, and at the first csc_set_graph after a csc_cluster
                       the rows are regrouped once by that assignment (degrees descending within
                       a cluster; the ring moves with them), so that most gathers of a block stay
                       inside one cluster's rows.  0: the caller's order.  Every row-indexed input
                       and output of the ABI stays in the caller's node order. */
  int64_t wave_bytes; /* csc_filter_batched: working-set budget (bytes) of one wave, the run of
                         consecutive column tiles whose recursion proceeds together; <= 0 selects
                         16 GiB.  Smaller waves finish tiles sooner, larger ones keep more tiles
                         in flight per recursion step. */
} csc_opts;

/* Counters of a context (csc_get_stats). */
typedef struct csc_stats {
  int64_t launches;       /* kernels this library launched on the context */
  int64_t step_launches;  /* general Chebyshev step launches bracketed by timing events */
  double step_ms;         /* device time of those launches (ms), CUDA events on the context stream */
  int64_t filter_passes;  /* recursion passes (one per column tile per filtering call) */
  int64_t tile;           /* widest column tile of the last filtering pass (a pass covers its
                             columns with tiles of 8, 16, 32 or 64; see csc_opts.col_tile) */
  int64_t batched_launches; /* persistent batched kernel launches (direct or in a graph) */
  int64_t graph_replays;    /* batched launches replayed from a captured CUDA graph */
  int64_t autotune_trials;  /* candidate tile timings run by the batched-path autotuner */
  int64_t batched_waves;    /* waves of the last batched call (csc_opts.wave_bytes) */
  int64_t kmeans_passes;    /* k-means assignment passes */
  int64_t kmeans_near_ties; /* rows whose distance-pass margin was within its error bound and
                               were re-decided exactly (summed over passes) */
  double step_bytes;        /* algorithmic bytes of the timed step launches: per launch over a
                               tile of width w, 4 nnz (col_idx; 8 nnz when weighted) + 8 (n+1)
                               (row_ptr) + 4 n (D^-1/2) + n w (s + 4 + 4 + 8) (V_{j-1} of s bytes
                               per value, V_j, V_{j+1}, Psi read and write) */
  int64_t kmeans_rows;      /* rows whose distances a k-means pass evaluated, summed over passes
                               (every row in the first pass of a call; later passes skip the rows
                               whose Hamerly bounds certify their centroid) */
} csc_stats;

/* ---------------------------------------------------------------- library */

/* Fills *opts with the defaults listed in csc_opts. */
void csc_default_opts(csc_opts* opts);
/* Static string for a status code. */
const char* csc_status_string(csc_status s);
/* CSC_ABI_VERSION of the built library. */
int csc_abi_version(void);

/* Host only.  The column tiles of a filtering pass over c columns (Section 3.3's recursion, run
 * tile by tile): widths in {8, 16, 32, 64} covering c that minimise sum (8 + w) over the tiles,
 * widest first (ties keep fewer, wider tiles); col_tile > 0 (8, 16, 32, 64 or 128) forces that
 * width.  Writes up to cap widths to widths_out and returns the number of tiles; -1 for bad
 * arguments, -(tiles + 1) when cap is too small. */
int csc_tile_plan(int c, int col_tile, int* widths_out, int cap);

/* Host only.  Algorithmic bytes of one general Chebyshev step launch over a tile of width w:
 * 4 nnz (8 nnz when weighted) + 8 (n + 1) + 4 n + n w (s_prev + 4 + 4 + 8), i.e. the column
 * indices (and weights), row offsets and D^-1/2 once, V_{j-1} (s_prev bytes per value), V_j,
 * V_{j+1}, and Psi read and written (the per-launch term of csc_stats.step_bytes). */
double csc_step_launch_bytes(int64_t n, int64_t nnz, int weighted, int w, int s_prev);

/* Creates a context on the current CUDA device.  `cuda_stream` is a cudaStream_t
 * (NULL = default stream).  opts may be NULL (defaults).  *out is owned by the
 * caller and released with csc_destroy. */
csc_status csc_create(csc_ctx** out, const csc_opts* opts, void* cuda_stream);
/* Frees every device and host buffer of the context (synchronises its stream). */
void csc_destroy(csc_ctx* ctx);
/* Message of the last failure on ctx ("" if none).  Valid until the next call. */
const char* csc_last_error(const csc_ctx* ctx);

/* Copies the context counters into *out; reset != 0 zeroes them afterwards. */
csc_status csc_get_stats(csc_ctx* ctx, csc_stats* out, int reset);

/* ---------------------------------------------------------------- graph */

/* Section 2.1: G = (V, E, W), simple, undirected, W_ij > 0, no self-loops.
 * Loads snapshot G_t as symmetric CSR: row_ptr int64[n+1] (row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz), col_idx int32[nnz] in [0, n), vals
 * float32[nnz] edge weights or NULL for unit weights.  Both directions of every
 * edge must be stored.  The data are copied (host->device or device->device);
 * the caller keeps ownership.  Computes degrees and D^{-1/2} (0 for isolated
 * nodes) of the normalized Laplacian L = I - D^{-1/2} W D^{-1/2}.
 * n must equal the n of earlier snapshots on this context (fixed vertex set,
 * Section 4) unless no snapshot has been filtered yet.
 * Errors: CSC_EINVAL on bad sizes or (host input, or checked mode) malformed
 * CSR; CSC_ENOMEM; CSC_ECUDA. */
csc_status csc_set_graph(csc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr,
                         const int32_t* col_idx, const float* vals, int where);

/* ---------------------------------------------------------------- host-only helpers (no GPU) */

/* Section 3.3: coefficients a_0..a_m (a_out double[m+1]) of the order-m
 * Jackson-damped Chebyshev approximation of 1[lambda <= lambda_c] on [0, 2],
 * h(lambda) = sum_j a_j T_j(lambda - 1).  lambda_c is clamped to [0, 2].
 * Errors: CSC_EINVAL if m < 0 or a_out is NULL. */
csc_status csc_filter_coeffs(int m, double lambda_c, double* a_out);

/* Default eigencount acceptance half-width max(0.5, 2 sqrt(2k/c)). */
double csc_count_tolerance(int k, int c);

/* Section 3.3 eigencount from the trace moments mu_l = tr(R^T T_l(L~) R),
 * l = 0..2m (mu double[2m+1]): count = (d/c) sum_{i,j} a_i a_j (mu_{i+j} + mu_{|i-j|})/2
 * = (d/c) ||h(L) R||_F^2 for c signals of variance 1/d. */
csc_status csc_count_from_moments(int m, const double* mu, double lambda_c, int d, int c,
                                  double* count_out);

/* The Hutchinson-type eigencount from the same moments: count = (d/c) sum_j a_j mu_j
 * = (d/c) tr(R^T h(L) R), an unbiased estimate of tr h(L) for c signals of variance 1/d
 * (csc_opts.estimator = 1 selects it in csc_estimate_lambda_k and csc_filter). */
csc_status csc_trace_count_from_moments(int m, const double* mu, double lambda_c, int d, int c,
                                        double* count_out);

/* Section 4.1 dichotomy of Algorithm 1 on the moment-based eigencount:
 * with lambda_prev < 0 bisect [0, 2]; else test lambda_prev, then grow a bracket
 * 0.01 * 2^i toward k until the count crosses k, then bisect.  Accept when
 * |count - k| <= tau; at most max_steps evaluations.  Outputs the cutoff, its
 * count and the number of evaluations. */
csc_status csc_lambda_search_moments(int m, const double* mu, int d, int c, int k, double tau,
                                     double lambda_prev, int max_steps, double* lambda_out,
                                     double* count_out, int* evals_out);

/* ---------------------------------------------------------------- building blocks */

/* Section 2.2 (approximate features): the n x c block of i.i.d. N(0, 1/d) signals for global column
 * ids col0 .. col0+c-1 (Philox-4x32-10 counter (row, column), key seed;
 * Box-Muller).  out: dtype CSC_F32 or CSC_BF16, leading dimension ld >= c,
 * caller-owned, host or device per `where`. */
csc_status csc_signals(csc_ctx* ctx, uint64_t seed, int64_t n, int64_t col0, int c, int d,
                       void* out, int dtype, int64_t ld, int where);

/* Sections 2.2 and 3.3: Psi~ = h(L) R for the current graph, caller's signal block
 * R (n x c, dtype CSC_F32 or CSC_BF16, leading dimension ldr, host or device per
 * r_where), Jackson-damped order-m low-pass of cutoff lambda_c in [0, 2], m >= 1.
 * psi_out: float32 n x c, leading dimension ldp >= c, host or device per
 * psi_where (NULL: moments only).  mu_out: host double[2m+1] trace moments
 * mu_l = tr(R^T T_l(L~) R) (NULL: not returned).  Does not touch the feature ring. */
csc_status csc_cheb_filter(csc_ctx* ctx, int m, double lambda_c, const void* R, int r_dtype, int c,
                           int64_t ldr, int r_where, float* psi_out, int64_t ldp, int psi_where,
                           double* mu_out);

/* Eq. 1-2 k-means (Lloyd) on caller features Y (n x d, d <= 1024, dtype CSC_F32 or CSC_BF16,
 * leading dimension ldy, host or device per y_where), used as given (no row
 * normalisation).  Initial centroids: rows init_idx (host int64[k], distinct, in
 * [0, n)) or, when prev_assign (host or device per assign_where, int32[n]) is
 * given, the means of that assignment with an empty cluster taking row
 * init_idx[j].  Assignment by squared Euclidean distance, ties to the lowest
 * index, decided exactly in float64 whenever the float32 margin is within its
 * error bound; update by means (exact fixed-point sums), an empty cluster keeps
 * its centroid; stop when the assignment repeats or after max_iter passes
 * (<= 0: the context's max_iter).  Outputs: assign_out int32[n] (host or
 * device per assign_where), centroids_out host double[k*d] or NULL,
 * inertia_out = sum_i ||y_i - c_{a(i)}||^2, iters_out = assignment passes. */
csc_status csc_kmeans(csc_ctx* ctx, const void* Y, int y_dtype, int64_t n, int d, int64_t ldy,
                      int y_where, int k, const int64_t* init_idx, const int32_t* prev_assign,
                      int max_iter, int32_t* assign_out, int assign_where, double* centroids_out,
                      double* inertia_out, int* iters_out);

/* ---------------------------------------------------------------- Algorithm 1 */

/* Initial cutoff of Algorithm 1 (Section 3.3): cutoff lambda_c whose eigencount of the d
 * signals the next csc_filter will draw (seed, the next d global column ids) is
 * within tau of k, by one moment pass of order m and the dichotomy on [0, 2].
 * Stores the cutoff on the context.  Outputs may be NULL. */
csc_status csc_estimate_lambda_k(csc_ctx* ctx, int k, int m, int d, uint64_t seed,
                                 double* lambda_out, double* count_out, int* evals_out);

/* One snapshot of Algorithm 1 up to the clustering (Eq. 6, Section 4.1).  First snapshot (or
 * p == 0): filter d new signals.  Later snapshots: keep dp = floor(p d) columns of
 * Theta_{t-1} (the ring slots filtered most recently) and filter dq = d - dp new
 * signals.  Cutoff: lambda_c >= 0 is used as given; lambda_c < 0 uses the
 * context's current cutoff (estimated first when there is none; needs k > 0).
 * With k > 0 the eigencount of the new block is checked and the cutoff refined
 * by the dichotomy when |count - k| > tau, after which the block is refiltered
 * (same signals).  The new columns overwrite the oldest ring slots; the
 * row-normalised Theta_t is prepared for csc_cluster.  d must stay the same
 * across snapshots.  Outputs (may be NULL): final cutoff, its eigencount,
 * dichotomy evaluations (0 when lambda_c was given or k <= 0), columns filtered. */
csc_status csc_filter(csc_ctx* ctx, int m, int d, double p, uint64_t seed, int k, double lambda_c,
                      double* lambda_out, double* count_out, int* evals_out, int* cols_out);

/* The splice of Eq. 6 with new columns that the caller filtered (for example one shard of the
 * columns per GPU, gathered afterwards): psi_new (float32, n x c, leading dimension ldp >= c,
 * host or device per where) holds the filtered columns of the next c global column ids, in
 * order; they overwrite the ring slots csc_filter would choose (c = d at the first snapshot or
 * when p == 0, else c = d - floor(p d)), the row-normalised Theta_t is prepared for
 * csc_cluster, and lambda_c (in [0, 2]) becomes the context's cutoff.  The global column
 * counter advances by c, as in csc_filter.  n and d must stay the same across snapshots.
 * Errors: CSC_EINVAL (bad arguments or a c that does not match), CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_splice(csc_ctx* ctx, int64_t n, int d, double p, const float* psi_new, int c, int64_t ldp,
                      int where, double lambda_c);

/* Edge-similarity policy for the dynamic scheme (Section 4: Definition 4.1, Theorem 4.1 with
 * Corollary 4.2, Section 4.1).  Given rho_t = ||L_t - L_{t-1}||_F (csc_laplacian_distance):
 *  - reuse fraction: Corollary 4.2 bounds ||H_t - H_{t-1}||_F by gamma = sqrt(2) rho_t / alpha
 *    (alpha: the caller's eigengap estimate), and the proof of Theorem 4.1 bounds the added
 *    k-means cost of reusing p d columns by 2 sqrt(p (1 + delta)) gamma; with delta = 1 and a
 *    budget eps, p_t = min(p_max, eps^2 / (8 gamma^2)) and dp = floor(p_t d) (dp = 0 refilters
 *    all d columns).  budget <= 0 or rho_t = 0 keeps p_max.
 *  - eigencount check: by Weyl's inequality no eigenvalue of L moves by more than the sum of
 *    rho since the last check, so while that sum stays <= rho_skip the previous cutoff is kept
 *    without the check; otherwise the check and refinement of Algorithm 1 run and the sum
 *    restarts at 0.  rho_skip = 0 checks at every snapshot that changed. */
typedef struct csc_similarity_policy {
  double alpha;    /* eigengap estimate (> 0 when budget > 0) */
  double budget;   /* tolerated added k-means cost eps (<= 0: no limit on the reuse) */
  double rho_skip; /* skip the check while the summed rho since the last one is <= this (>= 0) */
} csc_similarity_policy;

/* Host-only: the policy's decision for one snapshot: dp_out = reused columns, check_out = 1 when
 * the eigencount check runs, rho_since_out = the summed rho carried to the next snapshot (0 after
 * a check).  Errors: CSC_EINVAL. */
csc_status csc_reuse_policy(int d, double p_max, double rho, const csc_similarity_policy* pol, double rho_since,
                            int* dp_out, int* check_out, double* rho_since_out);

/* csc_filter with the edge-similarity policy above: at the first snapshot the same as csc_filter
 * with lambda_c < 0; afterwards dp and the check come from csc_reuse_policy with rho (this
 * snapshot's distance to the previous graph) and the sum carried on the context.  k >= 1.
 * Outputs as csc_filter (evals 0 when the check was skipped), checked_out = whether the check
 * ran (may be NULL).  Errors as csc_filter. */
csc_status csc_filter_adaptive(csc_ctx* ctx, int m, int d, double p_max, uint64_t seed, int k, double rho,
                               const csc_similarity_policy* pol, double* lambda_out, double* count_out,
                               int* evals_out, int* cols_out, int* checked_out);

/* Copies Theta_t (normalized = 0, float32 ring in slot order) or the row-normalised
 * features y_i = theta_i / ||theta_i|| (normalized = 1) into dst (n x d, dtype
 * CSC_F32 or CSC_BF16, leading dimension ld >= d, host or device per where). */
csc_status csc_get_features(csc_ctx* ctx, void* dst, int dtype, int64_t ld, int normalized,
                            int where);

/* Trace moments mu_0..mu_{2m} of the last filtering pass (host double[len], len <= 2m+1). */
csc_status csc_get_moments(csc_ctx* ctx, double* mu_out, int len);

/* The clustering of Algorithm 1: k-means on the row-normalised Theta_t.  The first
 * call on a context starts from Forgy rows init_idx (host int64[k]; NULL = draw
 * with the counter-based generator, key seed ^ (t * 0x9E3779B97F4A7C15)); later
 * calls warm-start from the previous assignment (an empty cluster takes row
 * init_idx[j]).  assign_out int32[n] host or device per where; cost_out =
 * C_Theta = sqrt(inertia) (Eq. 1 with Theta's row-normalised features);
 * iters_out = Lloyd assignment passes.  Outputs may be NULL except assign_out. */
csc_status csc_cluster(csc_ctx* ctx, int k, uint64_t seed, const int64_t* init_idx,
                       int32_t* assign_out, int where, double* cost_out, int* iters_out);

/* ---------------------------------------------------------------- batching */

/* One graph of a batched filtering call (all pointers are caller-owned device memory). */
typedef struct csc_graph_desc {
  int64_t n;              /* nodes */
  int64_t nnz;            /* stored entries (both directions of every edge) */
  const int64_t* row_ptr; /* CSR row pointers, n+1 */
  const int32_t* col_idx; /* CSR columns, nnz */
  const float* vals;      /* edge weights, nnz, or NULL for unit weights */
  int c;                  /* signals filtered for this graph (columns) */
  int d;                  /* the signals have variance 1/d (d >= c) */
  double lambda_c;        /* cutoff in [0, 2] */
  uint64_t seed;          /* signal stream: global column ids 0..c-1 under this key */
  float* psi;             /* output n x c float32, leading dimension ldp (NULL: moments only) */
  int64_t ldp;
} csc_graph_desc;

/* Filters many independent graphs (and snapshots) at once: for every graph g,
 * Psi~_g = h_g(L_g) R_g with R_g its counter-based signals (stored in bfloat16 when the
 * context precision is CSC_BF16, else float32), the order-m Jackson-damped low-pass of
 * cutoff lambda_c, and its trace moments (Sections 2.2 and 3.3).  All recursion steps of all
 * graphs run in one persistent cooperative kernel launch in which every step of a tile waits
 * (bounded) for the previous step of that tile, captured in a CUDA graph and replayed on later
 * calls with the same plan.  The
 * column tile of each graph is chosen by an autotuner that times the candidate tiles once per
 * graph size class (cached on the context).  Graphs must satisfy the CSR conditions of
 * csc_set_graph (not validated here).  mu_out: host double[n_graphs * (2m+1)] or NULL.
 * Errors: CSC_EINVAL, CSC_ENOMEM, CSC_ECUDA, CSC_ETIMEOUT (a dependency wait expired). */
csc_status csc_filter_batched(csc_ctx* ctx, int n_graphs, const csc_graph_desc* descs, int m,
                              double* mu_out);

/* ---------------------------------------------------------------- allocation-free variant */

/* The paper has no counterpart to this entry point.  It exists for callers that cannot call
 * cudaMalloc while they run: a framework whose caching allocator reserved the device memory up
 * front (a further allocation may fail, or fragment the memory that allocator manages), or a
 * latency-bound service that forbids allocation after start-up (cudaMalloc and cudaFree can
 * synchronise the whole device and stall every other stream).
 *
 * Computes the same Psi~ = h(L) R and trace moments as csc_cheb_filter, for a graph given
 * directly as caller-owned device CSR (row_ptr int64[n+1], col_idx int32[nnz], vals float[nnz]
 * or NULL; valid symmetric CSR as described at csc_set_graph, not validated here), a
 * caller-owned device signal block R (float32, n x c, leading dimension ldr >= c) and a
 * caller-owned device output psi_out (float32, n x c, leading dimension ldp >= c; NULL:
 * moments only).  mu_out: host double[2m+1] or NULL.  Work runs on cuda_stream (NULL = default
 * stream); the call copies each tile's moments to the host, synchronises that stream and
 * returns when the results are written.
 *
 * It allocates nothing: all scratch lives in one fixed static device array of about 11 MB,
 * which every GPU that loads this library holds until the process exits.  Limits: n <= 65,536,
 * nnz <= 4,194,304, 1 <= m <= 128 (any c; columns are processed 8 at a time); larger sizes
 * return CSC_ELIMIT.  The first call on a device looks up that array's device address (which
 * loads the module), so make the first call before any stream capture.  Every call shares the
 * one array, which keeps the last call's contents: calls that overlap on the GPU (other streams
 * or host threads) race on it and must be serialised by the caller.  Errors: CSC_EINVAL (bad
 * sizes, a null R, or an array that is not device memory), CSC_ELIMIT, CSC_ECUDA. */
csc_status csc_cheb_filter_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col_idx, const float* vals, int m,
                                   double lambda_c, const float* R, int c, int64_t ldr,
                                   float* psi_out, int64_t ldp, double* mu_out, void* cuda_stream);

/* ---------------------------------------------------------------- differentiation */
/* The paper has no derivative; these calls make its filter (Section 2.2 features
 * Psi = sum_j a_j T_j(L~) R, Section 3.3) a differentiable layer with respect to the
 * coefficients a_j and the edge weights W (through L~ = -D^-1/2 W D^-1/2, Section 2.1). */

/* Psi = sum_{j=0}^{m} coef[j] T_j(L~) R on the context's graph (its edge weights, unit if
 * none) for an arbitrary coefficient vector (host double[m+1]) and the caller's signal block R
 * (device float32, n x c, leading dimension ldr), written to psi_out (device float32, n x c,
 * leading dimension ldp).  The recursion state at every stride-th step (stride 0: ceil(sqrt m),
 * about 2 n c sqrt(m) floats; 1: every step, m n c floats written in place, and csc_filter_vjp
 * recomputes nothing) and a copy of R are kept in the context for csc_filter_vjp.
 * Errors: CSC_ESTATE without a graph, CSC_EINVAL, CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_filter_forward(csc_ctx* ctx, int m, const double* coef, const float* R, int c,
                              int64_t ldr, float* psi_out, int64_t ldp, int stride);

/* Vector-Jacobian product of the last csc_filter_forward: given grad_psi = dloss/dPsi (device
 * float32, n x c, leading dimension ldg), writes dloss/dcoef to grad_coef (host double[m+1],
 * may be NULL) and dloss/dw to grad_w (device float32[nnz] in CSR order, the gradient with
 * respect to the symmetric weight of each edge, equal at its two stored entries; may be NULL).
 * The graph must be symmetric.  Errors: CSC_ESTATE without a forward pass (or after a new
 * graph), CSC_EINVAL (bad arguments, asymmetric graph), CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_filter_vjp(csc_ctx* ctx, const float* grad_psi, int64_t ldg, double* grad_coef,
                          float* grad_w);

/* Feature-space k-means loss of Eq. 1 with fixed centroids and assignment:
 * loss = sum_i || psi_i / ||psi_i|| - mu_{assign[i]} ||^2 (a zero row contributes
 * ||mu_{assign[i]}||^2 and no gradient) and grad_psi = dloss/dPsi.  psi (n x c, ldp), mu
 * (k x c, contiguous), assign (int32[n]) and grad_psi (n x c, ldg) on the device; *loss_out on
 * the host.  Errors: CSC_EINVAL (bad arguments, a label outside [0, k)), CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_kmeans_loss_grad(csc_ctx* ctx, const float* psi, int64_t ldp, int64_t n, int c,
                                const float* mu, int k, const int32_t* assign, float* grad_psi,
                                int64_t ldg, double* loss_out);

/* ---------------------------------------------------------------- snapshot similarity */

/* Edge similarity of Definition 4.1: *rho_out = ||L_b - L_a||_F for the normalized
 * Laplacians L = I - D^-1/2 W D^-1/2 of two graphs a and b on the same n nodes, each a
 * device CSR (row_ptr int64[n+1], col_idx int32 with strictly increasing columns per row,
 * vals float32 or NULL for unit weights).  Corollary 4.2 bounds the change of the spectral
 * projector by sqrt(2)/alpha times rho.  Errors: CSC_EINVAL, CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_laplacian_distance(csc_ctx* ctx, int64_t n, const int64_t* rp_a, const int32_t* col_a,
                                  const float* val_a, const int64_t* rp_b, const int32_t* col_b,
                                  const float* val_b, double* rho_out);

/* ---------------------------------------------------------------- checkpoint / resume */

/* Algorithm 1 carries the feature ring Theta_{t-1}, the cutoff lambda_{t-1} and the
 * assignment X_{t-1} from one snapshot to the next.  csc_save_state writes that state to a
 * binary file at path: the ring (Theta float32 n x d and its row-normalised copy in the
 * context's precision), the ring stamps, the snapshot counter, the next signal column id,
 * the cutoff, the moments of the last filtering, the previous assignment with its k, the edge
 * distance summed since the last eigencount check (csc_filter_adaptive) and the context's node
 * order (csc_opts.reorder; the ring's rows are stored in it).  csc_load_state reads it into a
 * context created with the same precision and reorder setting, replacing that context's dynamic
 * state; the graph is not part of the state, so csc_set_graph (with the saved n) must come before
 * the next filtering.  A resumed context continues the sequence exactly as the saving one would
 * have: the same signal columns, slots, cutoff check and warm start.
 * The file is written in the machine's byte order: magic "CSCSTATE", version 2.
 * Errors: CSC_ESTATE (save before any csc_filter), CSC_EINVAL (NULL path, a file that cannot
 * be opened, written or read, not a state file, a corrupt or truncated file, a precision or
 * reorder mismatch), CSC_ENOMEM, CSC_ECUDA. */
csc_status csc_save_state(csc_ctx* ctx, const char* path);
csc_status csc_load_state(csc_ctx* ctx, const char* path);

/* ---------------------------------------------------------------- compressive k-means */

/* Compressive k-means (Section 2.2, step 2; cost counted in Section 4.2): k-means on a
 * variable-density sample of the nodes, the other assignments inferred by a Tikhonov
 * interpolation made of k graph filterings.
 *
 * 1. Sampling.  Node i is drawn with probability proportional to s_i = ||theta_i||^2 (the
 *    energy of its row of the unnormalised filtered signals), made exact in integers:
 *    s_i = float64 sum over columns in order of theta_il^2, q_i = floor(s_i 2^E) with
 *    E = 62 - ceil(log2 n) - e, 2^(e-1) <= max s < 2^e; P = inclusive prefix sums of q, T = P[n-1].
 *    Draw t (t < n_draws) uses Philox-4x32-10 with counter (t, 0, 0, 2) and key seed:
 *    u = floor((x0 2^32 + x1) T / 2^64); the node is the smallest i with P[i] > u.  The
 *    sample Omega is the set of distinct drawn nodes in increasing order.
 * 2. Reduced k-means.  Lloyd (as csc_kmeans) on the normalised rows y_i, i in Omega, from the
 *    Forgy rows of n_init restarts (restart r draws with key seed + r * 0x9E3779B97F4A7C15);
 *    the lowest inertia wins, inertias within a relative 1e-6 of it counting as equal and
 *    the lowest restart then winning.
 * 3. Interpolation.  Z (n x k) holds w_i = T / (n q_i) at (i, a_i) for every sampled node i
 *    with reduced label a_i; X = h(L) Z with the order-m Jackson-damped low pass of cutoff
 *    lambda_c, the minimiser of ||x - z_j||^2 + x^T (h(L)^-1 - I) x for every column.
 * 4. Node i is assigned the lowest j maximising X_ij.
 *
 * Features: theta == NULL and y == NULL take the context's current features (after
 * csc_filter: Theta_t, its row-normalised copy, the current cutoff when lambda_c < 0 and the
 * last filter order when m <= 0; d, ld, y_dtype and feat_where are then ignored).  Otherwise
 * theta is float32 n x d and y (y_dtype) n x d, both with leading dimension ld, in
 * feat_where memory, n being the loaded graph's size.
 * n_draws <= 0 takes max(k, ceil(2 k ln k)); n_init <= 0 takes 10; max_iter <= 0 the
 * context's.  Outputs in out_where memory: assign_out int32[n]; optional sample_out and
 * sample_labels_out int32[min(n, n_draws)] (Omega and its reduced labels; |Omega| entries
 * written) and interp_out float32 n x k (leading dimension ldx >= k); optional host
 * n_sampled_out (|Omega|) and restart_out (the restart kept).  The context's moments are
 * left as the last csc_filter set them.
 * Errors: CSC_ESTATE (no graph; context features before csc_filter), CSC_EINVAL (bad
 * arguments, all-zero features, fewer distinct sampled nodes than k, n_draws >= 2^31),
 * CSC_ENOMEM, CSC_ECUDA, CSC_ETIMEOUT (a bounded wait in the k-means pass expired). */
csc_status csc_compressive_cluster(csc_ctx* ctx, const float* theta, const void* y, int y_dtype, int d,
                                   int64_t ld, int feat_where, int k, int64_t n_draws, int n_init,
                                   double lambda_c, int m, uint64_t seed, int max_iter, int32_t* assign_out,
                                   int out_where, int32_t* sample_out, int32_t* sample_labels_out,
                                   float* interp_out, int64_t ldx, int64_t* n_sampled_out, int* restart_out);

#ifdef __cplusplus
}
#endif

#endif /* CSC_H */
