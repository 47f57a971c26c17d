// C ABI of libcsc (declarations and contracts in include/csc.h).
//
// Host-side logic of the method lives here: the Jackson-damped coefficients
// (Section 3.3), the eigencount from trace moments, the dichotomy for the cutoff
// (Algorithm 1, Section 4.1), the feature ring of Eq. 6 and the
// Lloyd driver.  Every device step runs in the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "csc_internal.h"

using csc::DevBuf;

namespace csc {

bool ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return true;
  release(b);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.ptr = p;
  b.bytes = bytes;
  return true;
}

void release(DevBuf& b) {
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int grid_for(const void* kernel, int block, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  return std::max(1, per_sm) * num_sms();
}

// Jackson-damped Chebyshev coefficients of the step 1[lambda <= lambda_c] (Section 3.3
// reading): a_j = g_j c_j with x = lambda - 1, theta = arccos(lambda_c - 1),
// c_0 = (pi - theta)/pi, c_j = -2 sin(j theta)/(j pi) and the Jackson factors g_j of order m.
void filter_coeffs(int m, double lambda_c, double* a) {
  const double x_c = std::min(1.0, std::max(-1.0, lambda_c - 1.0));
  const double theta = std::acos(x_c);
  const double mp2 = m + 2.0;
  const double alpha = M_PI / mp2;
  for (int j = 0; j <= m; ++j) {
    const double c = j == 0 ? (M_PI - theta) / M_PI : -2.0 * std::sin(j * theta) / (j * M_PI);
    const double g = ((mp2 - j) * std::sin(alpha) * std::cos(j * alpha) +
                      std::cos(alpha) * std::sin(j * alpha)) / (mp2 * std::sin(alpha));
    a[j] = g * c;
  }
}

}  // namespace csc

namespace {

using csc::filter_coeffs;

// ------------------------------------------------------------------ host math (Section 3.3)

double count_moments(int m, const double* mu, const double* a, int d, int c) {
  double s = 0.0;
  for (int i = 0; i <= m; ++i)
    for (int j = 0; j <= m; ++j) s += a[i] * a[j] * 0.5 * (mu[i + j] + mu[std::abs(i - j)]);
  return (double)d / (double)c * s;
}

// Hutchinson-type estimate (d/c) tr(R^T h(L) R) = (d/c) sum_j a_j mu_j of tr h(L).
double count_moments_trace(int m, const double* mu, const double* a, int d, int c) {
  double s = 0.0;
  for (int j = 0; j <= m; ++j) s += a[j] * mu[j];
  return (double)d / (double)c * s;
}

double tolerance(int k, int c) { return std::max(0.5, 2.0 * std::sqrt(2.0 * k / (double)c)); }

// Dichotomy used by Algorithm 1 to refine the cutoff (Section 4.1; rule in csc.h).
template <typename F>
void search(F count, int k, double tau, double lam_prev, int max_steps, double* lam_out,
            double* cnt_out, int* evals_out) {
  int evals = 0;
  double lam = 0.0, cnt = 0.0, lo = 0.0, hi = 2.0;
  auto ev = [&](double x) { ++evals; return count(x); };
  auto done = [&]() { *lam_out = lam; *cnt_out = cnt; *evals_out = evals; };
  if (lam_prev >= 0.0) {
    lam = lam_prev;
    cnt = ev(lam_prev);
    if (std::fabs(cnt - k) <= tau) return done();
    const double dir = cnt < k ? 1.0 : -1.0;
    double step = 0.01, prev = lam_prev;
    bool bracketed = false;
    while (evals < max_steps) {
      const double probe = std::min(2.0, std::max(0.0, lam_prev + dir * step));
      lam = probe;
      cnt = ev(probe);
      if (std::fabs(cnt - k) <= tau) return done();
      const bool crossed = dir > 0 ? (cnt > k) : (cnt < k);
      if (crossed || probe == 0.0 || probe == 2.0) {
        lo = std::min(prev, probe);
        hi = std::max(prev, probe);
        bracketed = true;
        break;
      }
      prev = probe;
      step *= 2.0;
    }
    if (!bracketed) return done();
  }
  while (evals < max_steps) {
    const double mid = 0.5 * (lo + hi);
    lam = mid;
    cnt = ev(mid);
    if (std::fabs(cnt - k) <= tau) return done();
    if (cnt < k) lo = mid; else hi = mid;
  }
  done();
}

// Philox-4x32-10 on the host (Forgy draws when the caller passes no indices).
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
}

std::vector<int64_t> forgy_draw(uint64_t seed, int64_t n, int k) {
  std::vector<int64_t> out;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int j = 0; j < k; ++j) {
    for (uint32_t attempt = 0;; ++attempt) {
      uint32_t c[4] = {(uint32_t)j, attempt, 0u, 1u};
      philox_host(c, k0, k1);
      const unsigned __int128 u = ((unsigned __int128)(((uint64_t)c[0] << 32) | c[1])) * (uint64_t)n;
      const int64_t idx = (int64_t)(u >> 64);
      if (std::find(out.begin(), out.end(), idx) == out.end()) {
        out.push_back(idx);
        break;
      }
    }
  }
  return out;
}

// Key of the Forgy draw of restart r of the reduced k-means.
uint64_t restart_seed(uint64_t seed, int r) { return seed + (uint64_t)r * 0x9E3779B97F4A7C15ull; }

// ------------------------------------------------------------------ context helpers

csc_status fail(csc_ctx* ctx, csc_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define CUDA_OK(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, CSC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

#define ALLOC_OK(expr) \
  do {                 \
    if (!(expr)) return fail(ctx, CSC_ENOMEM, "device allocation failed: " #expr); \
  } while (0)

// Column tiles of a filtering pass over c columns: widths in {8, 16, 32, 64} covering c, chosen to
// minimise sum_i (kTileFixed + w_i).  A step launch costs a part that does not depend on its width
// (the per-row staging, own-row loads and epilogue) plus a part proportional to it: on the
// power-law graph at n = 8e6 a launch took 2.7, 3.6, 5.3 and 8.4 ms at w = 8, 16, 32 and 64, on
// the SBM at n = 1e6 0.30, 0.53 and 0.96 ms at w = 16, 32 and 64, so wide tiles are cheaper per
// column on both, and a small remainder takes its own narrow tile.  col_tile > 0 forces one width.
constexpr int kTileFixed = 8;
std::vector<int> plan_tiles(int c, int col_tile) {
  if (c <= 0) return {};
  if (col_tile > 0) return std::vector<int>((c + col_tile - 1) / col_tile, col_tile);
  static const int widths[4] = {64, 32, 16, 8};
  std::vector<int> cost(c + 1, 0), pick(c + 1, 8);
  for (int r = 1; r <= c; ++r) {
    cost[r] = INT32_MAX;
    for (int w : widths) {  // widest first: ties keep the fewer, wider tiles
      const int v = kTileFixed + w + cost[std::max(0, r - w)];
      if (v < cost[r]) { cost[r] = v; pick[r] = w; }
    }
  }
  std::vector<int> plan;
  for (int r = c; r > 0; r -= pick[r]) plan.push_back(pick[r]);
  std::sort(plan.begin(), plan.end(), [](int x, int y) { return x > y; });
  return plan;
}
std::vector<int> tile_plan(const csc_ctx* ctx, int c) { return plan_tiles(c, ctx->opts.col_tile); }

int plan_columns(const std::vector<int>& plan) {
  int t = 0;
  for (int w : plan) t += w;
  return t;
}

// Algorithmic bytes of one general step launch over a tile of width w, each array counted
// once: col_idx (+ weights), row_ptr, D^-1/2, V_{j-1} (s_prev bytes per value), V_j, V_{j+1},
// and Psi read and write.
double step_launch_bytes(int64_t n, int64_t nnz, bool weighted, int w, int s_prev) {
  return 4.0 * nnz * (weighted ? 2 : 1) + 8.0 * (n + 1) + 4.0 * n + (double)n * w * (s_prev + 4 + 4 + 8);
}

bool valid_tile(int w) { return w == 8 || w == 16 || w == 32 || w == 64 || w == 128; }

// Signal source of a filtering pass: Philox columns or a caller block already on the device.
struct Source {
  bool philox = true;
  uint64_t seed = 0;
  int64_t col0 = 0;
  int d = 1;
  int dtype = CSC_F32;
  const void* R = nullptr;
  int64_t ldr = 0;
};

// Chebyshev recursion over c columns in tiles.  The signal source is in the caller's node order;
// psi_dst (device float, leading dim ldp; nullptr: moments only) receives Psi in the internal
// node order.  Fills ctx->mu (2m+1 trace moments).
csc_status run_filter(csc_ctx* ctx, int m, double lambda_c, int c, const Source& src, float* psi_dst,
                      int64_t ldp) {
  const int64_t n = ctx->g.n;
  cudaStream_t s = ctx->stream;
  const std::vector<int> plan = tile_plan(ctx, c);
  const int wmax = plan.empty() ? 8 : plan.front();
  if (!valid_tile(wmax)) return fail(ctx, CSC_EINVAL, "col_tile must be 8, 16, 32, 64 or 128");
  const int ntiles = (int)plan.size();
  const int grid = csc::cheb_grid(wmax);
  ctx->last_tile = wmax;
  const int rows = 2 * m + 1;
  for (auto& b : ctx->tbuf) ALLOC_OK(csc::ensure(b, (size_t)std::max<int64_t>(n, 1) * wmax * 4));
  ALLOC_OK(csc::ensure(ctx->part, (size_t)ntiles * rows * grid * 8));
  ALLOC_OK(csc::ensure(ctx->ef, (size_t)rows * 8));
  ALLOC_OK(csc::ensure(ctx->coef, (size_t)(m + 1) * 4));
  std::vector<double> a(m + 1);
  filter_coeffs(m, lambda_c, a.data());
  std::vector<float> af(a.begin(), a.end());
  CUDA_OK(cudaMemcpyAsync(ctx->coef.ptr, af.data(), af.size() * 4, cudaMemcpyHostToDevice, s));
  const int t0_dtype = src.philox ? ctx->opts.precision : src.dtype;
  const bool timed = ctx->opts.timing && m >= 2;
  if (timed) {
    while ((int)ctx->events.size() < 2 * ntiles) {
      cudaEvent_t e;
      CUDA_OK(cudaEventCreate(&e));
      ctx->events.push_back(e);
    }
  }
  const float inv_sqrt_d = (float)(1.0 / std::sqrt((double)src.d));
  double* part = csc::as<double>(ctx->part);
  int c0 = 0;
  for (int tile = 0; tile < ntiles; c0 += plan[tile], ++tile) {
    const int w = plan[tile];
    const int valid = std::min(w, c - c0);
    // signals and caller blocks are in the caller's node order; the tile in the internal order
    const int32_t* to_caller = ctx->g.permuted ? csc::as<int32_t>(ctx->g.perm) : nullptr;
    if (src.philox)
      CUDA_OK(csc::launch_signals(ctx->tbuf[0].ptr, t0_dtype, n, w, w, src.seed, src.col0 + c0, valid,
                                  inv_sqrt_d, s, to_caller));
    else
      CUDA_OK(csc::launch_copy_tile(ctx->tbuf[0].ptr, src.R, t0_dtype, n, w, src.ldr, c0, valid, s, to_caller));
    double* tile_part = part + (size_t)tile * rows * grid;
    csc::StepArgs sa{};
    sa.n = n;
    sa.row_ptr = csc::as<int64_t>(ctx->g.row_ptr);
    sa.col = csc::as<int32_t>(ctx->g.col);
    sa.val = ctx->g.weighted ? csc::as<float>(ctx->g.val) : nullptr;
    sa.scale = csc::as<float>(ctx->g.scale);
    sa.vs = csc::as<float>(ctx->g.vs);
    sa.ivs = csc::as<float>(ctx->g.ivs);
    sa.blk_row = csc::as<int32_t>(ctx->g.blk_row);
    sa.nblk = csc::edge_blocks(ctx->g.nnz);
    sa.srow = csc::as<int32_t>(ctx->g.srow);
    sa.nsblk = csc::row_blocks(ctx->g.n, ctx->g.nnz);
    sa.psi = psi_dst ? psi_dst + c0 : nullptr;
    sa.ldp = ldp;
    sa.coef = csc::as<float>(ctx->coef);
    sa.w = w;
    sa.tg = ctx->tbuf[0].ptr;
    sa.tp = nullptr;
    sa.tn = csc::as<float>(ctx->tbuf[1]);
    sa.j = 0;
    sa.part = tile_part;
    CUDA_OK(csc::launch_cheb_first(sa, t0_dtype, grid, s));
    if (timed) CUDA_OK(cudaEventRecord(ctx->events[2 * tile], s));
    for (int j = 1; j < m; ++j) {
      sa.tg = ctx->tbuf[j % 3].ptr;
      sa.tp = ctx->tbuf[(j - 1) % 3].ptr;
      sa.tn = csc::as<float>(ctx->tbuf[(j + 1) % 3]);
      sa.j = j;
      sa.part = tile_part + (size_t)(2 * (j + 1) - 1) * grid;
      sa.tp_unscaled = j == 1;
      CUDA_OK(csc::launch_cheb_step(sa, j == 1 ? t0_dtype : CSC_F32, grid, s));
    }
    if (timed) {
      CUDA_OK(cudaEventRecord(ctx->events[2 * tile + 1], s));
      for (int j = 1; j < m; ++j)
        ctx->step_bytes += step_launch_bytes(n, ctx->g.nnz, ctx->g.weighted, w,
                                             j == 1 && t0_dtype == CSC_BF16 ? 2 : 4);
    }
    ctx->launches += m + 1;
    ctx->filter_passes += 1;
  }
  ctx->launches += 1;
  CUDA_OK(csc::launch_reduce_partials(part, rows, grid, ntiles, (int64_t)rows * grid,
                                      csc::as<double>(ctx->ef), s));
  std::vector<double> ef(rows);
  CUDA_OK(cudaMemcpyAsync(ef.data(), ctx->ef.ptr, rows * 8, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (timed) {
    for (int tile = 0; tile < ntiles; ++tile) {
      float ms = 0.f;
      CUDA_OK(cudaEventElapsedTime(&ms, ctx->events[2 * tile], ctx->events[2 * tile + 1]));
      ctx->step_ms += ms;
      ctx->step_launches += m - 1;
    }
  }
  ctx->mu.assign(2 * m + 1, 0.0);
  ctx->mu[0] = ef[0];
  if (m >= 1) {
    ctx->mu[1] = ef[2];
    for (int q = 1; q <= m; ++q) {
      ctx->mu[2 * q] = 2.0 * ef[2 * q - 1] - ctx->mu[0];
      if (q >= 2) ctx->mu[2 * q - 1] = 2.0 * ef[2 * q] - ctx->mu[1];
    }
  }
  ctx->last_m = m;
  return CSC_OK;
}

double count_at(const csc_ctx* ctx, double lam, int d, int c) {
  std::vector<double> a(ctx->last_m + 1);
  filter_coeffs(ctx->last_m, lam, a.data());
  if (ctx->opts.estimator == 1) return count_moments_trace(ctx->last_m, ctx->mu.data(), a.data(), d, c);
  return count_moments(ctx->last_m, ctx->mu.data(), a.data(), d, c);
}

size_t dtype_size(int dtype) { return dtype == CSC_BF16 ? 2 : 4; }
bool valid_dtype(int dtype) { return dtype == CSC_F32 || dtype == CSC_BF16; }
bool valid_where(int where) { return where == CSC_HOST || where == CSC_DEVICE; }

// Node order of the internal graph: degrees descending, ties by caller id (a stable counting
// sort, O(n + max degree)).  perm[i] = caller row of internal row i, iperm its inverse.
// With labels (label[u] in [0, k) for caller row u): grouped by label first, degrees descending
// within a label (a stable counting sort by degree, then a stable one by label).
void degree_order(int64_t n, const int64_t* rp, const int32_t* label, int k, std::vector<int32_t>& perm,
                  std::vector<int32_t>& iperm) {
  int64_t maxdeg = 0;
  for (int64_t u = 0; u < n; ++u) maxdeg = std::max(maxdeg, rp[u + 1] - rp[u]);
  std::vector<int64_t> start(maxdeg + 2, 0);
  for (int64_t u = 0; u < n; ++u) start[maxdeg - (rp[u + 1] - rp[u]) + 1] += 1;
  for (int64_t b = 1; b <= maxdeg + 1; ++b) start[b] += start[b - 1];
  std::vector<int32_t> by_degree(n);
  for (int64_t u = 0; u < n; ++u) by_degree[start[maxdeg - (rp[u + 1] - rp[u])]++] = (int32_t)u;
  perm.assign(n, 0);
  iperm.assign(n, 0);
  if (label == nullptr) {
    perm = by_degree;
  } else {
    std::vector<int64_t> lstart(k + 1, 0);
    for (int64_t u = 0; u < n; ++u) lstart[label[u] + 1] += 1;
    for (int b = 1; b <= k; ++b) lstart[b] += lstart[b - 1];
    for (int64_t i = 0; i < n; ++i) {
      const int32_t u = by_degree[i];
      perm[lstart[label[u]]++] = u;
    }
  }
  for (int64_t i = 0; i < n; ++i) iperm[perm[i]] = (int32_t)i;
}

csc_status validate_host_csr(csc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* rp,
                             const int32_t* ci, const float* vals) {
  if (rp[0] != 0 || rp[n] != nnz) return fail(ctx, CSC_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] = nnz");
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return fail(ctx, CSC_EINVAL, "row_ptr must be non-decreasing");
    int64_t prev = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t c = ci[p];
      if (c < 0 || c >= n) return fail(ctx, CSC_EINVAL, "col_idx out of range");
      if (c == i) return fail(ctx, CSC_EINVAL, "self-loops are not allowed (simple graph)");
      if (c <= prev) return fail(ctx, CSC_EINVAL, "columns of a row must be strictly increasing");
      if (vals && !(vals[p] > 0.0f)) return fail(ctx, CSC_EINVAL, "edge weights must be positive");
      prev = c;
    }
  }
  return CSC_OK;
}

// Copies an n x d device block (dtype src_dtype, ld_src) to a caller destination.
// Caller row u -> internal row (nullptr when the graph is in the caller's order).
const int32_t* to_internal(csc_ctx* ctx) { return ctx->g.permuted ? csc::as<int32_t>(ctx->g.iperm) : nullptr; }

// Row i of dst is row src_row[i] of src (src_row nullptr: row i).
csc_status copy_out(csc_ctx* ctx, const void* src, int src_dtype, int64_t ld_src, int64_t n, int d,
                    void* dst, int dst_dtype, int64_t ld_dst, int where, const int32_t* src_row = nullptr) {
  cudaStream_t s = ctx->stream;
  const size_t esz = dtype_size(dst_dtype);
  ctx->launches += 1;
  if (where == CSC_DEVICE) {
    CUDA_OK(csc::launch_convert(src, src_dtype, ld_src, dst, dst_dtype, ld_dst, n, d, s, src_row));
    return CSC_OK;
  }
  ALLOC_OK(csc::ensure(ctx->out_stage, (size_t)std::max<int64_t>(n, 1) * d * esz));
  CUDA_OK(csc::launch_convert(src, src_dtype, ld_src, ctx->out_stage.ptr, dst_dtype, d, n, d, s, src_row));
  if (n > 0 && d > 0)
    CUDA_OK(cudaMemcpy2DAsync(dst, ld_dst * esz, ctx->out_stage.ptr, d * esz, d * esz, n,
                              cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  return CSC_OK;
}

// New internal order grouped by the previous assignment (reorder = 2); permutes the feature ring,
// its row-normalised copy and the previous assignment into it.  The caller's CSR of the snapshot
// being loaded (host or device row_ptr) gives the degrees.
csc_status regroup_by_clusters(csc_ctx* ctx, int64_t n, const int64_t* row_ptr, int where) {
  csc::Graph& g = ctx->g;
  cudaStream_t s = ctx->stream;
  std::vector<int64_t> rp_host;
  const int64_t* rp = row_ptr;
  if (where == CSC_DEVICE) {
    rp_host.resize(n + 1);
    CUDA_OK(cudaMemcpyAsync(rp_host.data(), row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, s));
  }
  std::vector<int32_t> lab_int(n), lab(n);
  CUDA_OK(cudaMemcpyAsync(lab_int.data(), ctx->prev_assign.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (where == CSC_DEVICE) rp = rp_host.data();
  for (int64_t u = 0; u < n; ++u) lab[u] = lab_int[g.h_iperm[u]];
  std::vector<int32_t> perm, iperm;
  degree_order(n, rp, lab.data(), ctx->prev_k, perm, iperm);
  // old internal row of each new internal row
  std::vector<int32_t> from(n);
  for (int64_t i = 0; i < n; ++i) from[i] = g.h_iperm[perm[i]];
  const int d = ctx->ring_d;
  const size_t ysz = dtype_size(ctx->opts.precision);
  ALLOC_OK(csc::ensure(ctx->out_stage, (size_t)n * d * 4));
  ALLOC_OK(csc::ensure(ctx->astage, (size_t)n * 4));
  ALLOC_OK(csc::ensure(g.perm, (size_t)n * 4));
  ALLOC_OK(csc::ensure(g.iperm, (size_t)n * 4));
  CUDA_OK(cudaMemcpyAsync(g.iperm.ptr, from.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));  // map (scratch)
  const int32_t* map = csc::as<int32_t>(g.iperm);
  // the ring, its normalised copy and the previous assignment move with the rows
  CUDA_OK(csc::launch_convert(ctx->theta.ptr, CSC_F32, d, ctx->out_stage.ptr, CSC_F32, d, n, d, s, map));
  CUDA_OK(cudaMemcpyAsync(ctx->theta.ptr, ctx->out_stage.ptr, (size_t)n * d * 4, cudaMemcpyDeviceToDevice, s));
  CUDA_OK(csc::launch_convert(ctx->y.ptr, ctx->opts.precision, d, ctx->out_stage.ptr, ctx->opts.precision, d, n, d,
                              s, map));
  CUDA_OK(cudaMemcpyAsync(ctx->y.ptr, ctx->out_stage.ptr, (size_t)n * d * ysz, cudaMemcpyDeviceToDevice, s));
  CUDA_OK(csc::launch_gather_i32(csc::as<int32_t>(ctx->astage), csc::as<int32_t>(ctx->prev_assign), map, n, s));
  CUDA_OK(cudaMemcpyAsync(ctx->prev_assign.ptr, ctx->astage.ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  CUDA_OK(cudaMemcpyAsync(g.perm.ptr, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(g.iperm.ptr, iperm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaStreamSynchronize(s));
  g.h_perm = std::move(perm);
  g.h_iperm = std::move(iperm);
  ctx->launches += 3;
  ctx->grouped = true;
  return CSC_OK;
}

}  // namespace

// ------------------------------------------------------------------ checkpoint / resume file

namespace {

constexpr char kStateMagic[8] = {'C', 'S', 'C', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kStateVersion = 2;

struct StateFile {
  FILE* f = nullptr;
  ~StateFile() {
    if (f) fclose(f);
  }
};

bool put(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

}  // namespace

extern "C" {

void csc_default_opts(csc_opts* o) {
  if (!o) return;
  o->precision = CSC_F32;
  o->count_tol = 0.0;
  o->max_bisect = 30;
  o->max_iter = 100;
  o->col_tile = 0;
  o->checked = 0;
  o->timing = 0;
  o->estimator = 0;
  o->reorder = 1;
  o->wave_bytes = 0;
}

const char* csc_status_string(csc_status s) {
  switch (s) {
    case CSC_OK: return "ok";
    case CSC_EINVAL: return "invalid argument";
    case CSC_ENOMEM: return "out of memory";
    case CSC_ECUDA: return "CUDA error";
    case CSC_ETIMEOUT: return "device wait timed out";
    case CSC_ESTATE: return "invalid call order";
    case CSC_ELIMIT: return "size beyond the fixed limit of the allocation-free entry point";
  }
  return "unknown status";
}

int csc_abi_version(void) { return CSC_ABI_VERSION; }

int csc_tile_plan(int c, int col_tile, int* widths_out, int cap) {
  if (c < 0 || (col_tile != 0 && !valid_tile(col_tile)) || (cap > 0 && !widths_out)) return -1;
  const std::vector<int> plan = plan_tiles(c, col_tile);
  if ((int)plan.size() > cap) return -(int)plan.size() - 1;
  for (size_t i = 0; i < plan.size(); ++i) widths_out[i] = plan[i];
  return (int)plan.size();
}

double csc_step_launch_bytes(int64_t n, int64_t nnz, int weighted, int w, int s_prev) {
  return step_launch_bytes(n, nnz, weighted != 0, w, s_prev);
}

csc_status csc_create(csc_ctx** out, const csc_opts* opts, void* cuda_stream) {
  if (!out) return CSC_EINVAL;
  *out = nullptr;
  csc_opts o;
  csc_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_dtype(o.precision) || o.max_bisect < 1 || o.max_iter < 1 ||
      (o.col_tile != 0 && !valid_tile(o.col_tile)) || (o.estimator != 0 && o.estimator != 1) ||
      (o.reorder < 0 || o.reorder > 2))
    return CSC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return CSC_ECUDA;
  }
  csc_ctx* ctx = new (std::nothrow) csc_ctx();
  if (!ctx) return CSC_ENOMEM;
  ctx->opts = o;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->device = dev;
  *out = ctx;
  return CSC_OK;
}

void csc_destroy(csc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  if (ctx->b_exec) cudaGraphExecDestroy(ctx->b_exec);
  if (ctx->b_cap) cudaStreamDestroy(ctx->b_cap);
  DevBuf* bufs[] = {&ctx->g.row_ptr, &ctx->g.col, &ctx->g.val, &ctx->g.scale, &ctx->g.deg,
                    &ctx->g.blk_row, &ctx->g.srow, &ctx->g.vs, &ctx->g.ivs,
                    &ctx->g.perm, &ctx->g.iperm, &ctx->g.urp, &ctx->g.ucol, &ctx->g.uval, &ctx->gtmp,
                    &ctx->tbuf[0], &ctx->tbuf[1], &ctx->tbuf[2], &ctx->psi, &ctx->part, &ctx->ef,
                    &ctx->coef, &ctx->rstage, &ctx->theta, &ctx->y, &ctx->slot_src,
                    &ctx->prev_assign, &ctx->ystage, &ctx->astage, &ctx->out_stage, &ctx->bad,
                    &ctx->b_prep, &ctx->b_tbuf, &ctx->b_psi, &ctx->b_coef, &ctx->b_mom,
                    &ctx->b_tiles, &ctx->b_items, &ctx->b_bar, &ctx->b_tune, &ctx->b_part,
                    &ctx->b_waves, &ctx->b_work,
                    &ctx->gs.coef_f, &ctx->gs.ckpt, &ctx->gs.seg, &ctx->gs.rt, &ctx->gs.gt,
                    &ctx->gs.phi[0], &ctx->gs.phi[1], &ctx->gs.phi[2], &ctx->gs.H, &ctx->gs.tpos,
                    &ctx->gs.nsum, &ctx->gs.part, &ctx->gs.flag, &ctx->gs.ga, &ctx->gs.rcopy, &ctx->gs.gw_stage,
                    &ctx->sim};
  for (DevBuf* b : bufs) csc::release(*b);
  csc::kmeans_release(ctx->km);
  csc::compressive_release(ctx->cmp);
  delete ctx;
}

const char* csc_last_error(const csc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

csc_status csc_get_stats(csc_ctx* ctx, csc_stats* out, int reset) {
  if (!ctx || !out) return CSC_EINVAL;
  out->launches = ctx->launches;
  out->step_launches = ctx->step_launches;
  out->step_ms = ctx->step_ms;
  out->filter_passes = ctx->filter_passes;
  out->tile = ctx->last_tile;
  out->batched_launches = ctx->batched_launches;
  out->graph_replays = ctx->graph_replays;
  out->autotune_trials = ctx->autotune_trials;
  out->batched_waves = ctx->batched_waves;
  out->kmeans_passes = ctx->kmeans_passes;
  out->kmeans_near_ties = ctx->kmeans_near_ties;
  out->kmeans_rows = ctx->kmeans_rows;
  out->step_bytes = ctx->step_bytes;
  if (reset) {
    ctx->launches = ctx->step_launches = ctx->filter_passes = 0;
    ctx->batched_launches = ctx->graph_replays = ctx->autotune_trials = 0;
    ctx->kmeans_passes = ctx->kmeans_near_ties = ctx->kmeans_rows = 0;
    ctx->step_ms = 0.0;
    ctx->step_bytes = 0.0;
  }
  return CSC_OK;
}

csc_status csc_set_graph(csc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr,
                         const int32_t* col_idx, const float* vals, int where) {
  if (!ctx) return CSC_EINVAL;
  if (n < 1 || nnz < 0 || n > INT32_MAX || !row_ptr || (nnz > 0 && !col_idx) || !valid_where(where))
    return fail(ctx, CSC_EINVAL, "csc_set_graph: bad sizes or pointers");
  if (ctx->t > 0 && n != ctx->ring_n)
    return fail(ctx, CSC_EINVAL, "csc_set_graph: the vertex set is fixed across snapshots");
  cudaStream_t s = ctx->stream;
  csc::Graph& g = ctx->g;
  const bool reorder = ctx->opts.reorder != 0;
  // caller CSR: uploaded into the caller-order buffers when the library reorders, else in place
  csc::DevBuf& rp_b = reorder ? g.urp : g.row_ptr;
  csc::DevBuf& col_b = reorder ? g.ucol : g.col;
  csc::DevBuf& val_b = reorder ? g.uval : g.val;
  ALLOC_OK(csc::ensure(g.row_ptr, (size_t)(n + 1) * 8));
  ALLOC_OK(csc::ensure(g.col, (size_t)nnz * 4));
  ALLOC_OK(csc::ensure(rp_b, (size_t)(n + 1) * 8));
  ALLOC_OK(csc::ensure(col_b, (size_t)nnz * 4));
  ALLOC_OK(csc::ensure(g.scale, (size_t)n * 4));
  ALLOC_OK(csc::ensure(g.vs, (size_t)n * 4));
  ALLOC_OK(csc::ensure(g.ivs, (size_t)n * 4));
  ALLOC_OK(csc::ensure(g.deg, (size_t)n * 8));
  ALLOC_OK(csc::ensure(g.blk_row, ((size_t)csc::edge_blocks(nnz) + 1) * 4));
  ALLOC_OK(csc::ensure(g.srow, ((size_t)csc::row_blocks(n, nnz) + 1) * 4));
  const cudaMemcpyKind kind = where == CSC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CUDA_OK(cudaMemcpyAsync(rp_b.ptr, row_ptr, (size_t)(n + 1) * 8, kind, s));
  if (nnz > 0) CUDA_OK(cudaMemcpyAsync(col_b.ptr, col_idx, (size_t)nnz * 4, kind, s));
  g.weighted = vals != nullptr;
  if (g.weighted) {
    ALLOC_OK(csc::ensure(g.val, (size_t)nnz * 4));
    ALLOC_OK(csc::ensure(val_b, (size_t)nnz * 4));
    if (nnz > 0) CUDA_OK(cudaMemcpyAsync(val_b.ptr, vals, (size_t)nnz * 4, kind, s));
  }
  g.n = n;
  g.nnz = nnz;
  // host input is always validated, on the device after the upload (an O(nnz) pass on the host
  // would cost more than the copy); the host validator runs only to name a failure
  if (where == CSC_HOST || ctx->opts.checked) {
    csc::Graph view;  // the caller's CSR
    view.n = n;
    view.nnz = nnz;
    view.weighted = g.weighted;
    view.row_ptr.ptr = rp_b.ptr;
    view.col.ptr = col_b.ptr;
    view.val.ptr = g.weighted ? val_b.ptr : nullptr;
    ALLOC_OK(csc::ensure(ctx->bad, 16));
    CUDA_OK(cudaMemsetAsync(ctx->bad.ptr, 0, 8, s));
    CUDA_OK(csc::launch_graph_check(view, csc::as<unsigned long long>(ctx->bad), s));
    view.row_ptr.ptr = view.col.ptr = view.val.ptr = nullptr;  // not owned
    ctx->launches += 1;
    unsigned long long bad = 0;
    int64_t ends[2] = {0, 0};
    CUDA_OK(cudaMemcpyAsync(&bad, ctx->bad.ptr, 8, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(&ends[0], rp_b.ptr, 8, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(&ends[1], csc::as<int64_t>(rp_b) + n, 8, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    if (bad != 0 || ends[0] != 0 || ends[1] != nnz) {
      g.loaded = false;
      if (where == CSC_HOST) {
        csc_status st = validate_host_csr(ctx, n, nnz, row_ptr, col_idx, vals);
        if (st != CSC_OK) return st;
      }
      return fail(ctx, CSC_EINVAL, "csc_set_graph: malformed CSR (" + std::to_string(bad) +
                                       " violations)");
    }
  }
  if (reorder) {
    // the node order: fixed while a feature ring exists (its rows are stored in that order)
    if (!(ctx->t > 0 && g.permuted && (int64_t)g.h_perm.size() == n)) {
      std::vector<int64_t> rp_host;
      const int64_t* rp = row_ptr;
      if (where == CSC_DEVICE) {
        rp_host.resize(n + 1);
        CUDA_OK(cudaMemcpyAsync(rp_host.data(), row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        rp = rp_host.data();
      }
      degree_order(n, rp, nullptr, 0, g.h_perm, g.h_iperm);
      ALLOC_OK(csc::ensure(g.perm, (size_t)n * 4));
      ALLOC_OK(csc::ensure(g.iperm, (size_t)n * 4));
      CUDA_OK(cudaMemcpyAsync(g.perm.ptr, g.h_perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaMemcpyAsync(g.iperm.ptr, g.h_iperm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaStreamSynchronize(s));  // the host vectors may be reallocated later
      ctx->grouped = false;
    } else if (ctx->opts.reorder == 2 && !ctx->grouped && ctx->has_prev && ctx->prev_k > 0) {
      // once, after the first clustering: rows grouped by the previous assignment (degrees
      // descending within a cluster), so that a block's gathers mostly stay inside one cluster's
      // rows; the ring and the previous assignment move with the rows
      csc_status st = regroup_by_clusters(ctx, n, row_ptr, where);
      if (st != CSC_OK) return st;
    }
    ALLOC_OK(csc::ensure(ctx->gtmp, ((size_t)n + (size_t)csc::scan_sums_len(n)) * 8));
    long long* tmp = csc::as<long long>(ctx->gtmp);
    CUDA_OK(csc::launch_permute_graph(g, tmp, tmp + n, s));
    ctx->launches += 4;
    g.permuted = true;
  } else {
    g.permuted = false;
  }
  CUDA_OK(csc::launch_graph_prep(g, s));
  CUDA_OK(csc::launch_block_rows(g, s));
  ctx->launches += 2;
  g.loaded = true;
  ctx->graph_version += 1;
  ctx->gs.ready = false;
  return CSC_OK;
}

csc_status csc_filter_coeffs(int m, double lambda_c, double* a_out) {
  if (m < 0 || !a_out || !(lambda_c == lambda_c)) return CSC_EINVAL;
  filter_coeffs(m, lambda_c, a_out);
  return CSC_OK;
}

double csc_count_tolerance(int k, int c) { return c > 0 ? tolerance(k, c) : 0.0; }

csc_status csc_count_from_moments(int m, const double* mu, double lambda_c, int d, int c,
                                  double* count_out) {
  if (m < 0 || !mu || d < 1 || c < 1 || !count_out) return CSC_EINVAL;
  std::vector<double> a(m + 1);
  filter_coeffs(m, lambda_c, a.data());
  *count_out = count_moments(m, mu, a.data(), d, c);
  return CSC_OK;
}

csc_status csc_trace_count_from_moments(int m, const double* mu, double lambda_c, int d, int c,
                                       double* count_out) {
  if (m < 0 || !mu || d < 1 || c < 1 || !count_out) return CSC_EINVAL;
  std::vector<double> a(m + 1);
  filter_coeffs(m, lambda_c, a.data());
  *count_out = count_moments_trace(m, mu, a.data(), d, c);
  return CSC_OK;
}

csc_status csc_lambda_search_moments(int m, const double* mu, int d, int c, int k, double tau,
                                     double lambda_prev, int max_steps, double* lambda_out,
                                     double* count_out, int* evals_out) {
  if (m < 0 || !mu || d < 1 || c < 1 || k < 1 || !(tau >= 0.0) || max_steps < 1 || !lambda_out ||
      !count_out || !evals_out)
    return CSC_EINVAL;
  std::vector<double> a(m + 1);
  auto count = [&](double lam) {
    filter_coeffs(m, lam, a.data());
    return count_moments(m, mu, a.data(), d, c);
  };
  search(count, k, tau, lambda_prev, max_steps, lambda_out, count_out, evals_out);
  return CSC_OK;
}

csc_status csc_signals(csc_ctx* ctx, uint64_t seed, int64_t n, int64_t col0, int c, int d, void* out,
                       int dtype, int64_t ld, int where) {
  if (!ctx) return CSC_EINVAL;
  if (n < 0 || col0 < 0 || c < 0 || d < 1 || ld < c || !out || !valid_dtype(dtype) || !valid_where(where))
    return fail(ctx, CSC_EINVAL, "csc_signals: bad arguments");
  const float inv_sqrt_d = (float)(1.0 / std::sqrt((double)d));
  cudaStream_t s = ctx->stream;
  ctx->launches += 1;
  if (where == CSC_DEVICE) {
    CUDA_OK(csc::launch_signals(out, dtype, n, c, ld, seed, col0, c, inv_sqrt_d, s));
    return CSC_OK;
  }
  const size_t esz = dtype_size(dtype);
  ALLOC_OK(csc::ensure(ctx->out_stage, (size_t)std::max<int64_t>(n, 1) * std::max(c, 1) * esz));
  CUDA_OK(csc::launch_signals(ctx->out_stage.ptr, dtype, n, c, c, seed, col0, c, inv_sqrt_d, s));
  if (n > 0 && c > 0)
    CUDA_OK(cudaMemcpy2DAsync(out, ld * esz, ctx->out_stage.ptr, c * esz, c * esz, n,
                              cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  return CSC_OK;
}

csc_status csc_cheb_filter(csc_ctx* ctx, int m, double lambda_c, const void* R, int r_dtype, int c,
                           int64_t ldr, int r_where, float* psi_out, int64_t ldp, int psi_where,
                           double* mu_out) {
  if (!ctx) return CSC_EINVAL;
  if (!ctx->g.loaded) return fail(ctx, CSC_ESTATE, "csc_cheb_filter: no graph loaded");
  if (m < 1 || c < 1 || !R || ldr < c || !valid_dtype(r_dtype) || !valid_where(r_where) ||
      !(lambda_c >= 0.0 && lambda_c <= 2.0) || (psi_out && (ldp < c || !valid_where(psi_where))))
    return fail(ctx, CSC_EINVAL, "csc_cheb_filter: bad arguments");
  const int64_t n = ctx->g.n;
  cudaStream_t s = ctx->stream;
  Source src;
  src.philox = false;
  src.dtype = r_dtype;
  src.d = 1;
  if (r_where == CSC_HOST) {
    const size_t esz = dtype_size(r_dtype);
    ALLOC_OK(csc::ensure(ctx->rstage, (size_t)n * c * esz));
    CUDA_OK(cudaMemcpy2DAsync(ctx->rstage.ptr, c * esz, R, ldr * esz, c * esz, n,
                              cudaMemcpyHostToDevice, s));
    src.R = ctx->rstage.ptr;
    src.ldr = c;
  } else {
    src.R = R;
    src.ldr = ldr;
  }
  const int cpad = plan_columns(tile_plan(ctx, c));
  float* psi = nullptr;
  if (psi_out) {
    ALLOC_OK(csc::ensure(ctx->psi, (size_t)n * cpad * 4));
    psi = csc::as<float>(ctx->psi);
  }
  csc_status st = run_filter(ctx, m, lambda_c, c, src, psi, cpad);
  if (st != CSC_OK) return st;
  if (psi_out) {
    st = copy_out(ctx, psi, CSC_F32, cpad, n, c, psi_out, CSC_F32, ldp, psi_where, to_internal(ctx));
    if (st != CSC_OK) return st;
    CUDA_OK(cudaStreamSynchronize(s));
  }
  if (mu_out) std::copy(ctx->mu.begin(), ctx->mu.end(), mu_out);
  return CSC_OK;
}

csc_status csc_estimate_lambda_k(csc_ctx* ctx, int k, int m, int d, uint64_t seed,
                                 double* lambda_out, double* count_out, int* evals_out) {
  if (!ctx) return CSC_EINVAL;
  if (!ctx->g.loaded) return fail(ctx, CSC_ESTATE, "csc_estimate_lambda_k: no graph loaded");
  if (k < 1 || m < 1 || d < 1) return fail(ctx, CSC_EINVAL, "csc_estimate_lambda_k: bad arguments");
  Source src;
  src.seed = seed;
  src.col0 = ctx->next_id;
  src.d = d;
  csc_status st = run_filter(ctx, m, 1.0, d, src, nullptr, 0);
  if (st != CSC_OK) return st;
  const double tau = ctx->opts.count_tol > 0 ? ctx->opts.count_tol : tolerance(k, d);
  double lam, cnt;
  int evals;
  search([&](double x) { return count_at(ctx, x, d, d); }, k, tau, -1.0, ctx->opts.max_bisect, &lam,
         &cnt, &evals);
  ctx->lambda = lam;
  ctx->has_lambda = true;
  if (lambda_out) *lambda_out = lam;
  if (count_out) *count_out = cnt;
  if (evals_out) *evals_out = evals;
  return CSC_OK;
}

}  // extern "C"

namespace {

// Ring slots that the new columns of this snapshot overwrite (Eq. 6 reading): all d at the
// first snapshot or when dp == 0, else the dq = d - dp slots with the oldest stamp, ties to the
// lowest slot, in ascending slot order.
std::vector<int> new_slots(const csc_ctx* ctx, int d, int dp) {
  std::vector<int> slots;
  if (ctx->t == 0 || dp <= 0) {
    for (int q = 0; q < d; ++q) slots.push_back(q);
    return slots;
  }
  const int c = d - dp;
  std::vector<int> order(d);
  for (int q = 0; q < d; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ctx->stamp[x] < ctx->stamp[y]; });
  slots.assign(order.begin(), order.begin() + c);
  std::sort(slots.begin(), slots.end());
  return slots;
}

// Writes the new columns psi (device float32, n x c, leading dimension ldp; column v goes to
// slots[v]) into Theta_t, row-normalises it into Y and advances the ring (Eq. 6, Algorithm 1).
csc_status splice_columns(csc_ctx* ctx, int64_t n, int d, const std::vector<int>& slots, const float* psi,
                          int64_t ldp, double lam) {
  cudaStream_t s = ctx->stream;
  const int c = (int)slots.size();
  if (ctx->t == 0) {
    ALLOC_OK(csc::ensure(ctx->theta, (size_t)n * d * 4));
    ALLOC_OK(csc::ensure(ctx->y, (size_t)n * d * 4));
    ALLOC_OK(csc::ensure(ctx->slot_src, (size_t)d * 4));
    ctx->stamp.assign(d, 0);
    ctx->ring_n = n;
    ctx->ring_d = d;
  }
  std::vector<int> src_of(d, -1);
  for (int v = 0; v < c; ++v) src_of[slots[v]] = v;
  CUDA_OK(cudaMemcpyAsync(ctx->slot_src.ptr, src_of.data(), d * 4, cudaMemcpyHostToDevice, s));
  CUDA_OK(csc::launch_assemble(csc::as<float>(ctx->theta), d, psi, ldp, csc::as<int>(ctx->slot_src), d,
                               ctx->y.ptr, ctx->opts.precision, d, n, s));
  ctx->launches += 1;
  CUDA_OK(cudaStreamSynchronize(s));
  ctx->t += 1;
  for (int q : slots) ctx->stamp[q] = ctx->t;
  ctx->next_id += c;
  ctx->lambda = lam;
  ctx->has_lambda = true;
  return CSC_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// One snapshot of Algorithm 1 up to the clustering with dp reused columns; check = false keeps
// the current cutoff without the eigencount check.
csc_status filter_snapshot(csc_ctx* ctx, int m, int d, int dp, uint64_t seed, int k, double lambda_c,
                           bool check, double* lambda_out, double* count_out, int* evals_out,
                           int* cols_out) {
  const int64_t n = ctx->g.n;
  if (!check && ctx->has_lambda && lambda_c < 0) lambda_c = ctx->lambda;
  const std::vector<int> slots = new_slots(ctx, d, dp);
  const int c = (int)slots.size();
  Source src;
  src.seed = seed;
  src.col0 = ctx->next_id;
  src.d = d;
  double lam = lambda_c;
  int evals = 0;
  bool searched = false;
  const double tau = ctx->opts.count_tol > 0 ? ctx->opts.count_tol : (k >= 1 ? tolerance(k, c) : 0.0);
  if (lam < 0 && !ctx->has_lambda) {
    csc_status st = run_filter(ctx, m, 1.0, c, src, nullptr, 0);
    if (st != CSC_OK) return st;
    double cnt;
    search([&](double x) { return count_at(ctx, x, d, c); }, k, tau, -1.0, ctx->opts.max_bisect,
           &lam, &cnt, &evals);
    searched = true;
  } else if (lam < 0) {
    lam = ctx->lambda;
  }
  const int cpad = plan_columns(tile_plan(ctx, c));
  ALLOC_OK(csc::ensure(ctx->psi, (size_t)n * cpad * 4));
  csc_status st = run_filter(ctx, m, lam, c, src, csc::as<float>(ctx->psi), cpad);
  if (st != CSC_OK) return st;
  double cnt = count_at(ctx, lam, d, c);
  if (lambda_c < 0 && k >= 1 && !searched) {
    double lam2, cnt2;
    search([&](double x) { return count_at(ctx, x, d, c); }, k, tau, lam, ctx->opts.max_bisect, &lam2,
           &cnt2, &evals);
    if (lam2 != lam) {
      st = run_filter(ctx, m, lam2, c, src, csc::as<float>(ctx->psi), cpad);
      if (st != CSC_OK) return st;
      lam = lam2;
    }
    cnt = cnt2;
  }
  // splice the new columns into the oldest slots and row-normalise (Eq. 6)
  st = splice_columns(ctx, n, d, slots, csc::as<float>(ctx->psi), cpad, lam);
  if (st != CSC_OK) return st;
  if (lambda_out) *lambda_out = lam;
  if (count_out) *count_out = cnt;
  if (evals_out) *evals_out = evals;
  if (cols_out) *cols_out = c;
  return CSC_OK;
}

csc_status filter_args(csc_ctx* ctx, int m, int d, double p, int k, double lambda_c, const char* who) {
  if (!ctx->g.loaded) return fail(ctx, CSC_ESTATE, std::string(who) + ": no graph loaded");
  if (m < 1 || d < 1 || d > 1024 || !(p >= 0.0 && p < 1.0) || lambda_c > 2.0)
    return fail(ctx, CSC_EINVAL, std::string(who) + ": need m >= 1, 1 <= d <= 1024, 0 <= p < 1, lambda_c <= 2");
  if (ctx->t > 0 && d != ctx->ring_d)
    return fail(ctx, CSC_EINVAL, std::string(who) + ": d must stay the same across snapshots");
  if (ctx->t > 0 && ctx->g.n != ctx->ring_n)
    return fail(ctx, CSC_ESTATE, std::string(who) + ": the graph's n differs from the feature ring's");
  if (lambda_c < 0 && !ctx->has_lambda && k < 1)
    return fail(ctx, CSC_ESTATE, std::string(who) + ": no cutoff yet; pass lambda_c >= 0 or k >= 1");
  return CSC_OK;
}

// Edge-similarity policy (Definition 4.1, Theorem 4.1 with Corollary 4.2; rule in csc.h).
void reuse_policy(int d, double p_max, double rho, const csc_similarity_policy& pol, double rho_since, int* dp,
                  int* check, double* rho_after) {
  const double acc = rho_since + rho;
  double p = p_max;
  if (pol.budget > 0.0 && rho > 0.0) {
    const double gamma = std::sqrt(2.0) * rho / pol.alpha;
    p = std::min(p_max, pol.budget * pol.budget / (8.0 * gamma * gamma));
  }
  *dp = (int)std::floor(p * d);
  *check = !(acc <= pol.rho_skip);
  *rho_after = *check ? 0.0 : acc;
}

bool valid_policy(const csc_similarity_policy* pol) {
  return pol && pol->budget == pol->budget && pol->rho_skip >= 0.0 && (pol->budget <= 0.0 || pol->alpha > 0.0);
}

}  // namespace

extern "C" {

csc_status csc_filter(csc_ctx* ctx, int m, int d, double p, uint64_t seed, int k, double lambda_c,
                      double* lambda_out, double* count_out, int* evals_out, int* cols_out) {
  if (!ctx) return CSC_EINVAL;
  csc_status st = filter_args(ctx, m, d, p, k, lambda_c, "csc_filter");
  if (st != CSC_OK) return st;
  const int dp = p > 0.0 ? (int)std::floor(p * d) : 0;
  return filter_snapshot(ctx, m, d, dp, seed, k, lambda_c, true, lambda_out, count_out, evals_out, cols_out);
}

csc_status csc_reuse_policy(int d, double p_max, double rho, const csc_similarity_policy* pol, double rho_since,
                            int* dp_out, int* check_out, double* rho_since_out) {
  if (d < 1 || !(p_max >= 0.0 && p_max < 1.0) || !(rho >= 0.0) || !(rho_since >= 0.0) || !valid_policy(pol) ||
      !dp_out || !check_out || !rho_since_out)
    return CSC_EINVAL;
  reuse_policy(d, p_max, rho, *pol, rho_since, dp_out, check_out, rho_since_out);
  return CSC_OK;
}

csc_status csc_filter_adaptive(csc_ctx* ctx, int m, int d, double p_max, uint64_t seed, int k, double rho,
                               const csc_similarity_policy* pol, double* lambda_out, double* count_out,
                               int* evals_out, int* cols_out, int* checked_out) {
  if (!ctx) return CSC_EINVAL;
  if (!valid_policy(pol) || !(rho >= 0.0) || k < 1)
    return fail(ctx, CSC_EINVAL, "csc_filter_adaptive: need k >= 1, rho >= 0 and a valid policy");
  csc_status st = filter_args(ctx, m, d, p_max, k, -1.0, "csc_filter_adaptive");
  if (st != CSC_OK) return st;
  int dp = p_max > 0.0 ? (int)std::floor(p_max * d) : 0, check = 1;
  double after = 0.0;
  if (ctx->t > 0) reuse_policy(d, p_max, rho, *pol, ctx->rho_since, &dp, &check, &after);
  st = filter_snapshot(ctx, m, d, dp, seed, k, -1.0, check != 0, lambda_out, count_out, evals_out, cols_out);
  if (st != CSC_OK) return st;
  ctx->rho_since = after;
  if (checked_out) *checked_out = check;
  return CSC_OK;
}

csc_status csc_splice(csc_ctx* ctx, int64_t n, int d, double p, const float* psi_new, int c, int64_t ldp,
                      int where, double lambda_c) {
  if (!ctx) return CSC_EINVAL;
  if (n < 1 || d < 1 || d > 1024 || !(p >= 0.0 && p < 1.0) || c < 1 || !psi_new || ldp < c ||
      !valid_where(where) || !(lambda_c >= 0.0 && lambda_c <= 2.0))
    return fail(ctx, CSC_EINVAL, "csc_splice: bad arguments");
  if (ctx->t > 0 && (d != ctx->ring_d || n != ctx->ring_n))
    return fail(ctx, CSC_EINVAL, "csc_splice: n and d must stay the same across snapshots");
  const std::vector<int> slots = new_slots(ctx, d, p > 0.0 ? (int)std::floor(p * d) : 0);
  if ((int)slots.size() != c)
    return fail(ctx, CSC_EINVAL, "csc_splice: c must be d at the first snapshot (or p = 0), else d - floor(p d)");
  const float* src = psi_new;
  int64_t ld = ldp;
  if (where == CSC_HOST) {
    ALLOC_OK(csc::ensure(ctx->rstage, (size_t)n * c * 4));
    CUDA_OK(cudaMemcpy2DAsync(ctx->rstage.ptr, (size_t)c * 4, psi_new, (size_t)ldp * 4, (size_t)c * 4, n,
                              cudaMemcpyHostToDevice, ctx->stream));
    src = csc::as<float>(ctx->rstage);
    ld = c;
  }
  if (ctx->g.permuted) {
    // the caller's rows into the internal node order of the ring
    if (!ctx->g.loaded || ctx->g.n != n) return fail(ctx, CSC_ESTATE, "csc_splice: load the snapshot's graph first");
    ALLOC_OK(csc::ensure(ctx->psi, (size_t)n * c * 4));
    CUDA_OK(csc::launch_convert(src, CSC_F32, ld, ctx->psi.ptr, CSC_F32, c, n, c, ctx->stream,
                                csc::as<int32_t>(ctx->g.perm)));
    ctx->launches += 1;
    src = csc::as<float>(ctx->psi);
    ld = c;
  }
  return splice_columns(ctx, n, d, slots, src, ld, lambda_c);
}

csc_status csc_get_features(csc_ctx* ctx, void* dst, int dtype, int64_t ld, int normalized, int where) {
  if (!ctx) return CSC_EINVAL;
  if (ctx->t == 0) return fail(ctx, CSC_ESTATE, "csc_get_features: nothing filtered yet");
  if (!dst || !valid_dtype(dtype) || ld < ctx->ring_d || !valid_where(where))
    return fail(ctx, CSC_EINVAL, "csc_get_features: bad arguments");
  if (normalized)
    return copy_out(ctx, ctx->y.ptr, ctx->opts.precision, ctx->ring_d, ctx->ring_n, ctx->ring_d, dst,
                    dtype, ld, where, to_internal(ctx));
  return copy_out(ctx, ctx->theta.ptr, CSC_F32, ctx->ring_d, ctx->ring_n, ctx->ring_d, dst, dtype, ld,
                  where, to_internal(ctx));
}

csc_status csc_get_moments(csc_ctx* ctx, double* mu_out, int len) {
  if (!ctx) return CSC_EINVAL;
  if (ctx->mu.empty()) return fail(ctx, CSC_ESTATE, "csc_get_moments: no filtering pass yet");
  if (!mu_out || len < 0 || len > (int)ctx->mu.size())
    return fail(ctx, CSC_EINVAL, "csc_get_moments: len must be <= 2m+1");
  std::copy(ctx->mu.begin(), ctx->mu.begin() + len, mu_out);
  return CSC_OK;
}

csc_status csc_kmeans(csc_ctx* ctx, const void* Y, int y_dtype, int64_t n, int d, int64_t ldy,
                      int y_where, int k, const int64_t* init_idx, const int32_t* prev_assign,
                      int max_iter, int32_t* assign_out, int assign_where, double* centroids_out,
                      double* inertia_out, int* iters_out) {
  if (!ctx) return CSC_EINVAL;
  if (!Y || n < 1 || d < 1 || d > 1024 || ldy < d || k < 1 || k > n || !init_idx || !assign_out ||
      !valid_dtype(y_dtype) || !valid_where(y_where) || !valid_where(assign_where))
    return fail(ctx, CSC_EINVAL, "csc_kmeans: bad arguments");
  for (int j = 0; j < k; ++j)
    if (init_idx[j] < 0 || init_idx[j] >= n) return fail(ctx, CSC_EINVAL, "csc_kmeans: init_idx out of range");
  cudaStream_t s = ctx->stream;
  const size_t esz = dtype_size(y_dtype);
  const void* ydev = Y;
  int64_t ld = ldy;
  if (y_where == CSC_HOST) {
    ALLOC_OK(csc::ensure(ctx->ystage, (size_t)n * d * esz));
    CUDA_OK(cudaMemcpy2DAsync(ctx->ystage.ptr, d * esz, Y, ldy * esz, d * esz, n,
                              cudaMemcpyHostToDevice, s));
    ydev = ctx->ystage.ptr;
    ld = d;
  }
  const int32_t* prev = nullptr;
  if (prev_assign) {
    if (assign_where == CSC_HOST) {
      for (int64_t i = 0; i < n; ++i)
        if (prev_assign[i] < 0 || prev_assign[i] >= k)
          return fail(ctx, CSC_EINVAL, "csc_kmeans: prev_assign out of range");
      ALLOC_OK(csc::ensure(ctx->astage, (size_t)n * 4));
      CUDA_OK(cudaMemcpyAsync(ctx->astage.ptr, prev_assign, (size_t)n * 4, cudaMemcpyHostToDevice, s));
      prev = csc::as<int32_t>(ctx->astage);
    } else {
      prev = prev_assign;
    }
  }
  csc::KmeansResult res;
  csc_status st = csc::kmeans_run(ctx->km, ydev, y_dtype, n, d, ld, k, init_idx, prev,
                                  max_iter > 0 ? max_iter : ctx->opts.max_iter, s, &res, &ctx->err);
  ctx->launches += res.launches;
  ctx->kmeans_passes += res.iters;
  ctx->kmeans_near_ties += res.near_ties;
  ctx->kmeans_rows += res.decided;
  if (st != CSC_OK) return st;
  const cudaMemcpyKind kind = assign_where == CSC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CUDA_OK(cudaMemcpyAsync(assign_out, res.assign, (size_t)n * 4, kind, s));
  if (centroids_out)
    CUDA_OK(cudaMemcpyAsync(centroids_out, ctx->km.c64.ptr, (size_t)k * d * 8, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (inertia_out) *inertia_out = res.inertia;
  if (iters_out) *iters_out = res.iters;
  return CSC_OK;
}

csc_status csc_cluster(csc_ctx* ctx, int k, uint64_t seed, const int64_t* init_idx, int32_t* assign_out,
                       int where, double* cost_out, int* iters_out) {
  if (!ctx) return CSC_EINVAL;
  if (ctx->t == 0) return fail(ctx, CSC_ESTATE, "csc_cluster: call csc_filter first");
  const int64_t n = ctx->ring_n;
  const int d = ctx->ring_d;
  if (k < 1 || k > n || !assign_out || !valid_where(where))
    return fail(ctx, CSC_EINVAL, "csc_cluster: bad arguments");
  std::vector<int64_t> idx;
  if (init_idx) {
    idx.assign(init_idx, init_idx + k);
    for (int64_t v : idx)
      if (v < 0 || v >= n) return fail(ctx, CSC_EINVAL, "csc_cluster: init_idx out of range");
  } else {
    idx = forgy_draw(seed ^ ((uint64_t)ctx->t * 0x9E3779B97F4A7C15ull), n, k);
  }
  cudaStream_t s = ctx->stream;
  // the ring is in the internal node order; Forgy rows and the assignment are in the caller's
  const bool perm = ctx->g.permuted;
  if (perm)
    for (int64_t& v : idx) v = ctx->g.h_iperm[v];
  const bool warm = ctx->has_prev && ctx->prev_k == k;
  csc::KmeansResult res;
  csc_status st = csc::kmeans_run(ctx->km, ctx->y.ptr, ctx->opts.precision, n, d, d, k, idx.data(),
                                  warm ? csc::as<int32_t>(ctx->prev_assign) : nullptr,
                                  ctx->opts.max_iter, s, &res, &ctx->err);
  ctx->launches += res.launches;
  ctx->kmeans_passes += res.iters;
  ctx->kmeans_near_ties += res.near_ties;
  ctx->kmeans_rows += res.decided;
  if (st != CSC_OK) return st;
  ALLOC_OK(csc::ensure(ctx->prev_assign, (size_t)n * 4));
  CUDA_OK(cudaMemcpyAsync(ctx->prev_assign.ptr, res.assign, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  const int32_t* out = res.assign;
  if (perm) {
    ALLOC_OK(csc::ensure(ctx->astage, (size_t)n * 4));
    CUDA_OK(csc::launch_gather_i32(csc::as<int32_t>(ctx->astage), res.assign, csc::as<int32_t>(ctx->g.iperm), n, s));
    out = csc::as<int32_t>(ctx->astage);
  }
  const cudaMemcpyKind kind = where == CSC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CUDA_OK(cudaMemcpyAsync(assign_out, out, (size_t)n * 4, kind, s));
  CUDA_OK(cudaStreamSynchronize(s));
  ctx->has_prev = true;
  ctx->prev_k = k;
  if (cost_out) *cost_out = std::sqrt(std::max(0.0, res.inertia));
  if (iters_out) *iters_out = res.iters;
  return CSC_OK;
}


csc_status csc_compressive_cluster(csc_ctx* ctx, const float* theta, const void* y, int y_dtype, int d,
                                   int64_t ld, int feat_where, int k, int64_t n_draws, int n_init,
                                   double lambda_c, int m, uint64_t seed, int max_iter, int32_t* assign_out,
                                   int out_where, int32_t* sample_out, int32_t* sample_labels_out,
                                   float* interp_out, int64_t ldx, int64_t* n_sampled_out, int* restart_out) {
  if (!ctx) return CSC_EINVAL;
  if (!ctx->g.loaded) return fail(ctx, CSC_ESTATE, "csc_compressive_cluster: no graph loaded");
  const int64_t n = ctx->g.n;
  if (k < 1 || !assign_out || !valid_where(out_where) || (theta == nullptr) != (y == nullptr) ||
      n_draws >= ((int64_t)1 << 31) || (interp_out && ldx < k))
    return fail(ctx, CSC_EINVAL, "csc_compressive_cluster: bad arguments");
  cudaStream_t s = ctx->stream;
  csc::CompressiveState& cs = ctx->cmp;
  const float* th = theta;
  const void* yy = y;
  if (theta == nullptr) {
    if (ctx->t == 0 || ctx->ring_n != n)
      return fail(ctx, CSC_ESTATE, "csc_compressive_cluster: call csc_filter first");
    th = csc::as<float>(ctx->theta);
    yy = ctx->y.ptr;
    y_dtype = ctx->opts.precision;
    d = ctx->ring_d;
    ld = d;
    if (ctx->g.permuted) {
      // the draws are defined in the caller's node order: the ring's rows in that order first
      const size_t esz = dtype_size(y_dtype);
      ALLOC_OK(csc::ensure(cs.theta_stage, (size_t)n * d * 4));
      ALLOC_OK(csc::ensure(cs.y_stage, (size_t)n * d * esz));
      CUDA_OK(csc::launch_convert(th, CSC_F32, d, cs.theta_stage.ptr, CSC_F32, d, n, d, s, to_internal(ctx)));
      CUDA_OK(csc::launch_convert(yy, y_dtype, d, cs.y_stage.ptr, y_dtype, d, n, d, s, to_internal(ctx)));
      ctx->launches += 2;
      th = csc::as<float>(cs.theta_stage);
      yy = cs.y_stage.ptr;
    }
    if (lambda_c < 0.0) {
      if (!ctx->has_lambda) return fail(ctx, CSC_ESTATE, "csc_compressive_cluster: no cutoff yet");
      lambda_c = ctx->lambda;
    }
    if (m <= 0) m = ctx->last_m;
  } else {
    if (d < 1 || d > 1024 || ld < d || !valid_dtype(y_dtype) || !valid_where(feat_where))
      return fail(ctx, CSC_EINVAL, "csc_compressive_cluster: bad feature arguments");
    if (feat_where == CSC_HOST) {
      const size_t esz = dtype_size(y_dtype);
      ALLOC_OK(csc::ensure(cs.theta_stage, (size_t)n * d * 4));
      ALLOC_OK(csc::ensure(cs.y_stage, (size_t)n * d * esz));
      CUDA_OK(cudaMemcpy2DAsync(cs.theta_stage.ptr, (size_t)d * 4, theta, (size_t)ld * 4, (size_t)d * 4, n,
                                cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaMemcpy2DAsync(cs.y_stage.ptr, d * esz, y, ld * esz, d * esz, n, cudaMemcpyHostToDevice, s));
      th = csc::as<float>(cs.theta_stage);
      yy = cs.y_stage.ptr;
      ld = d;
    }
  }
  if (m < 1 || !(lambda_c >= 0.0 && lambda_c <= 2.0))
    return fail(ctx, CSC_EINVAL, "csc_compressive_cluster: the interpolation needs m >= 1 and a cutoff in [0, 2]");
  if (n_draws <= 0) n_draws = std::max<int64_t>(k, (int64_t)std::ceil(2.0 * k * std::log((double)k)));
  if (n_init <= 0) n_init = 10;
  if (max_iter <= 0) max_iter = ctx->opts.max_iter;

  // 1. variable-density draws and the sorted sample
  CUDA_OK(csc::compressive_sample(cs, th, ld, n, d, n_draws, seed, s));
  ctx->launches += 9;
  long long total = 0;
  int n_omega = 0;
  CUDA_OK(cudaMemcpyAsync(&total, csc::as<long long>(cs.prefix) + (n - 1), 8, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaMemcpyAsync(&n_omega, csc::as<int>(cs.pos) + (n - 1), 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (total <= 0) return fail(ctx, CSC_EINVAL, "csc_compressive_cluster: the features are all zero");
  if (n_omega < k)
    return fail(ctx, CSC_EINVAL, "csc_compressive_cluster: " + std::to_string(n_omega) +
                                     " distinct sampled nodes for k = " + std::to_string(k) + "; raise n_draws");
  const int32_t* omega = csc::as<int32_t>(cs.omega);

  // 2. reduced k-means: n_init Forgy restarts on the sampled rows, lowest inertia kept
  ALLOC_OK(csc::ensure(cs.yo, (size_t)n_omega * d * dtype_size(y_dtype)));
  ALLOC_OK(csc::ensure(cs.labels, (size_t)n_init * n_omega * 4));
  CUDA_OK(csc::compressive_gather(yy, y_dtype, ld, omega, n_omega, d, cs.yo.ptr, s));
  ctx->launches += 1;
  std::vector<double> inertia(n_init);
  for (int r = 0; r < n_init; ++r) {
    const std::vector<int64_t> idx = forgy_draw(restart_seed(seed, r), n_omega, k);
    csc::KmeansResult res;
    csc_status st = csc::kmeans_run(ctx->km, cs.yo.ptr, y_dtype, n_omega, d, d, k, idx.data(), nullptr,
                                    max_iter, s, &res, &ctx->err);
    ctx->launches += res.launches;
    ctx->kmeans_passes += res.iters;
    ctx->kmeans_near_ties += res.near_ties;
    ctx->kmeans_rows += res.decided;
    if (st != CSC_OK) return st;
    inertia[r] = res.inertia;
    CUDA_OK(cudaMemcpyAsync(csc::as<int32_t>(cs.labels) + (size_t)r * n_omega, res.assign, (size_t)n_omega * 4,
                            cudaMemcpyDeviceToDevice, s));
  }
  const double best = *std::min_element(inertia.begin(), inertia.end());
  int pick = 0;
  while (!(inertia[pick] <= best * (1.0 + 1e-6))) ++pick;
  const int32_t* labels = csc::as<int32_t>(cs.labels) + (size_t)pick * n_omega;

  // 3. interpolation: X = h(L) Z, one filtering of each cluster's weighted indicator
  const int cpad = plan_columns(tile_plan(ctx, k));
  ALLOC_OK(csc::ensure(cs.z, (size_t)n * k * 4));
  ALLOC_OK(csc::ensure(cs.x, (size_t)n * cpad * 4));
  ALLOC_OK(csc::ensure(cs.assign, (size_t)n * 4));
  CUDA_OK(cudaMemsetAsync(cs.z.ptr, 0, (size_t)n * k * 4, s));
  CUDA_OK(csc::compressive_rhs(cs, labels, n_omega, n, csc::as<float>(cs.z), k, s));
  ctx->launches += 1;
  Source src;
  src.philox = false;
  src.dtype = CSC_F32;
  src.R = cs.z.ptr;
  src.ldr = k;
  const std::vector<double> mu_keep = ctx->mu;
  const int m_keep = ctx->last_m;
  csc_status st = run_filter(ctx, m, lambda_c, k, src, csc::as<float>(cs.x), cpad);
  ctx->mu = mu_keep;
  ctx->last_m = m_keep;
  if (st != CSC_OK) return st;
  CUDA_OK(csc::compressive_argmax(csc::as<float>(cs.x), cpad, n, k, csc::as<int32_t>(cs.assign), s));
  ctx->launches += 1;
  // X and its argmax are in the internal node order
  const int32_t* assign = csc::as<int32_t>(cs.assign);
  if (ctx->g.permuted) {
    ALLOC_OK(csc::ensure(ctx->astage, (size_t)n * 4));
    CUDA_OK(csc::launch_gather_i32(csc::as<int32_t>(ctx->astage), assign, to_internal(ctx), n, s));
    assign = csc::as<int32_t>(ctx->astage);
  }
  const cudaMemcpyKind kind = out_where == CSC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CUDA_OK(cudaMemcpyAsync(assign_out, assign, (size_t)n * 4, kind, s));
  if (sample_out) CUDA_OK(cudaMemcpyAsync(sample_out, omega, (size_t)n_omega * 4, kind, s));
  if (sample_labels_out) CUDA_OK(cudaMemcpyAsync(sample_labels_out, labels, (size_t)n_omega * 4, kind, s));
  if (interp_out) {
    st = copy_out(ctx, cs.x.ptr, CSC_F32, cpad, n, k, interp_out, CSC_F32, ldx, out_where, to_internal(ctx));
    if (st != CSC_OK) return st;
  }
  CUDA_OK(cudaStreamSynchronize(s));
  if (n_sampled_out) *n_sampled_out = n_omega;
  if (restart_out) *restart_out = pick;
  return CSC_OK;
}


csc_status csc_save_state(csc_ctx* ctx, const char* path) {
  if (!ctx) return CSC_EINVAL;
  if (!path) return fail(ctx, CSC_EINVAL, "csc_save_state: null path");
  if (ctx->t == 0) return fail(ctx, CSC_ESTATE, "csc_save_state: nothing filtered yet");
  const int64_t n = ctx->ring_n;
  const int d = ctx->ring_d;
  const size_t cells = (size_t)n * d;
  const size_t ysz = dtype_size(ctx->opts.precision);
  std::vector<float> theta(cells);
  std::vector<unsigned char> y(cells * ysz);
  std::vector<int32_t> prev;
  cudaStream_t s = ctx->stream;
  CUDA_OK(cudaMemcpyAsync(theta.data(), ctx->theta.ptr, cells * 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaMemcpyAsync(y.data(), ctx->y.ptr, cells * ysz, cudaMemcpyDeviceToHost, s));
  if (ctx->has_prev) {
    prev.resize((size_t)n);
    CUDA_OK(cudaMemcpyAsync(prev.data(), ctx->prev_assign.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  }
  CUDA_OK(cudaStreamSynchronize(s));
  StateFile sf;
  sf.f = fopen(path, "wb");
  if (!sf.f) return fail(ctx, CSC_EINVAL, std::string("csc_save_state: cannot open ") + path);
  const int32_t precision = ctx->opts.precision, ring_d = d, has_lambda = ctx->has_lambda ? 1 : 0;
  const int32_t last_m = ctx->last_m, n_mu = (int32_t)ctx->mu.size();
  const int32_t has_prev = ctx->has_prev ? 1 : 0, prev_k = ctx->prev_k;
  const int64_t t = ctx->t, next_id = ctx->next_id;
  // the ring's rows are stored in the context's node order, which is saved with them
  const int32_t permuted = ctx->g.permuted && (int64_t)ctx->g.h_perm.size() == n ? 1 : 0;
  const int32_t grouped = ctx->grouped ? 1 : 0;
  const bool ok = put(sf.f, kStateMagic, 8) && put(sf.f, &kStateVersion, 4) && put(sf.f, &precision, 4) &&
                  put(sf.f, &n, 8) && put(sf.f, &ring_d, 4) && put(sf.f, &t, 8) && put(sf.f, &next_id, 8) &&
                  put(sf.f, &has_lambda, 4) && put(sf.f, &ctx->lambda, 8) && put(sf.f, &last_m, 4) &&
                  put(sf.f, &n_mu, 4) && put(sf.f, ctx->mu.data(), ctx->mu.size() * 8) &&
                  put(sf.f, ctx->stamp.data(), ctx->stamp.size() * 8) && put(sf.f, &has_prev, 4) &&
                  put(sf.f, &prev_k, 4) && put(sf.f, theta.data(), cells * 4) && put(sf.f, y.data(), y.size()) &&
                  put(sf.f, prev.data(), prev.size() * 4) && put(sf.f, &ctx->rho_since, 8) &&
                  put(sf.f, &permuted, 4) && put(sf.f, &grouped, 4) &&
                  put(sf.f, ctx->g.h_perm.data(), permuted ? (size_t)n * 4 : 0);
  const bool closed = fclose(sf.f) == 0;
  sf.f = nullptr;
  if (!ok || !closed) return fail(ctx, CSC_EINVAL, std::string("csc_save_state: write failed for ") + path);
  return CSC_OK;
}

csc_status csc_load_state(csc_ctx* ctx, const char* path) {
  if (!ctx) return CSC_EINVAL;
  if (!path) return fail(ctx, CSC_EINVAL, "csc_load_state: null path");
  StateFile sf;
  sf.f = fopen(path, "rb");
  if (!sf.f) return fail(ctx, CSC_EINVAL, std::string("csc_load_state: cannot open ") + path);
  char magic[8];
  uint32_t version = 0;
  int32_t precision = 0, ring_d = 0, has_lambda = 0, last_m = 0, n_mu = 0, has_prev = 0, prev_k = 0;
  int64_t n = 0, t = 0, next_id = 0;
  double lambda = 0.0;
  if (!get(sf.f, magic, 8) || std::memcmp(magic, kStateMagic, 8) != 0 || !get(sf.f, &version, 4) ||
      version != kStateVersion)
    return fail(ctx, CSC_EINVAL, std::string("csc_load_state: not a state file: ") + path);
  bool ok = get(sf.f, &precision, 4) && get(sf.f, &n, 8) && get(sf.f, &ring_d, 4) && get(sf.f, &t, 8) &&
            get(sf.f, &next_id, 8) && get(sf.f, &has_lambda, 4) && get(sf.f, &lambda, 8) &&
            get(sf.f, &last_m, 4) && get(sf.f, &n_mu, 4);
  if (!ok || n < 1 || ring_d < 1 || ring_d > 1024 || t < 1 || next_id < 0 || n_mu < 0 || n_mu > (1 << 20) ||
      !valid_dtype(precision))
    return fail(ctx, CSC_EINVAL, "csc_load_state: corrupt header");
  if (precision != ctx->opts.precision)
    return fail(ctx, CSC_EINVAL, "csc_load_state: the state was saved with another precision");
  std::vector<double> mu((size_t)n_mu);
  std::vector<int64_t> stamp((size_t)ring_d);
  ok = get(sf.f, mu.data(), mu.size() * 8) && get(sf.f, stamp.data(), stamp.size() * 8) &&
       get(sf.f, &has_prev, 4) && get(sf.f, &prev_k, 4);
  if (!ok || (has_prev != 0 && has_prev != 1) || (has_prev && prev_k < 1))
    return fail(ctx, CSC_EINVAL, "csc_load_state: corrupt header");
  const size_t cells = (size_t)n * ring_d;
  const size_t ysz = dtype_size(precision);
  std::vector<float> theta(cells);
  std::vector<unsigned char> y(cells * ysz);
  std::vector<int32_t> prev(has_prev ? (size_t)n : 0);
  double rho_since = 0.0;
  int32_t permuted = 0, grouped = 0;
  ok = get(sf.f, theta.data(), cells * 4) && get(sf.f, y.data(), y.size()) && get(sf.f, prev.data(), prev.size() * 4) &&
       get(sf.f, &rho_since, 8) && get(sf.f, &permuted, 4) && get(sf.f, &grouped, 4);
  if (!ok || (permuted != 0 && permuted != 1) || (grouped != 0 && grouped != 1) || !(rho_since >= 0.0))
    return fail(ctx, CSC_EINVAL, "csc_load_state: truncated file");
  if ((permuted != 0) != (ctx->opts.reorder != 0))
    return fail(ctx, CSC_EINVAL, "csc_load_state: the state was saved with another reorder setting");
  std::vector<int32_t> perm(permuted ? (size_t)n : 0), iperm(perm.size(), -1);
  if (!get(sf.f, perm.data(), perm.size() * 4)) return fail(ctx, CSC_EINVAL, "csc_load_state: truncated file");
  for (size_t i = 0; i < perm.size(); ++i) {
    const int32_t u = perm[i];
    if (u < 0 || u >= n || iperm[u] != -1) return fail(ctx, CSC_EINVAL, "csc_load_state: corrupt node order");
    iperm[u] = (int32_t)i;
  }
  for (int32_t v : prev)
    if (v < 0 || v >= prev_k) return fail(ctx, CSC_EINVAL, "csc_load_state: assignment label out of range");
  cudaStream_t s = ctx->stream;
  ALLOC_OK(csc::ensure(ctx->theta, cells * 4));
  ALLOC_OK(csc::ensure(ctx->y, cells * 4));
  ALLOC_OK(csc::ensure(ctx->slot_src, (size_t)ring_d * 4));
  if (has_prev) ALLOC_OK(csc::ensure(ctx->prev_assign, (size_t)n * 4));
  CUDA_OK(cudaMemcpyAsync(ctx->theta.ptr, theta.data(), cells * 4, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(ctx->y.ptr, y.data(), y.size(), cudaMemcpyHostToDevice, s));
  if (has_prev) CUDA_OK(cudaMemcpyAsync(ctx->prev_assign.ptr, prev.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  if (permuted) {
    ALLOC_OK(csc::ensure(ctx->g.perm, (size_t)n * 4));
    ALLOC_OK(csc::ensure(ctx->g.iperm, (size_t)n * 4));
    CUDA_OK(cudaMemcpyAsync(ctx->g.perm.ptr, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(ctx->g.iperm.ptr, iperm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
  }
  CUDA_OK(cudaStreamSynchronize(s));
  // the graph is not part of the state: load the next snapshot before filtering
  ctx->g.loaded = false;
  ctx->g.permuted = permuted != 0;
  ctx->g.h_perm = std::move(perm);
  ctx->g.h_iperm = std::move(iperm);
  ctx->rho_since = rho_since;
  ctx->grouped = grouped != 0;
  ctx->ring_n = n;
  ctx->ring_d = ring_d;
  ctx->t = t;
  ctx->next_id = next_id;
  ctx->has_lambda = has_lambda != 0;
  ctx->lambda = lambda;
  ctx->last_m = last_m;
  ctx->mu = mu;
  ctx->stamp = stamp;
  ctx->has_prev = has_prev != 0;
  ctx->prev_k = prev_k;
  return CSC_OK;
}

}  // extern "C"
