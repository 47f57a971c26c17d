"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: features within 1e-5 relative Frobenius error (float32 storage)
and 3e-3 against the float64-signal oracle for bfloat16 signal storage;
moments within 1e-5 of mu_0; k-means assignments exactly equal given identical
features and initial rows.
"""
import math

import numpy as np
import pytest

import workloads as W
from conftest import fp32_floor
from oracle import chebyshev as cb
from oracle import kmeans as km
from oracle import laplacian as lp
from oracle import similarity as sm
from oracle.dynamic import DynamicCSC, row_normalize
from oracle.philox import gaussian_columns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 3e-3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def upload_graph(ctx, g, vals=None):
    ctx.set_graph(g.n, dev(g.row_ptr), dev(g.col_idx), None if vals is None else dev(vals))


@pytest.fixture(scope="module")
def cfg1_graph():
    return W.sbm_graph(2000, 10, 20, 10, seed=1)


def test_signals_match_oracle_generator(gpu_lib):
    n, c, d, col0, seed = 5003, 13, 64, 7, 0xDEADBEEF12345
    with gpu_lib.Context() as ctx:
        out = torch.zeros((n, c), dtype=torch.float32, device="cuda")
        ctx.signals(seed, n, col0, c, d, out)
        ref = gaussian_columns(seed, n, np.arange(col0, col0 + c), d)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
        outb = torch.zeros((n, 16), dtype=torch.bfloat16, device="cuda")
        ctx.signals(seed, n, col0, c, d, outb[:, :c])
        gb = outb[:, :c].float().cpu().numpy()
        # bf16 rounding of the float32 draws: within one bf16 ulp of the float64 draw
        assert np.all(np.abs(gb - ref) <= 2.0**-7 * np.abs(ref) + 1e-30)
        assert np.all(outb[:, c:].float().cpu().numpy() == 0)


@pytest.mark.parametrize("reorder", [1, 0])
@pytest.mark.parametrize("tile", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("c", [64, 13, 1])
def test_cheb_filter_parity_tiles(gpu_lib, cfg1_graph, tile, c, reorder):
    g = cfg1_graph
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(g.n, c, 64, seed=c * 7 + tile)
    m, lam = 50, 0.53
    with gpu_lib.Context({"col_tile": tile, "reorder": reorder}) as ctx:
        upload_graph(ctx, g)
        psi = torch.zeros((g.n, c), dtype=torch.float32, device="cuda")
        mu = ctx.cheb_filter(m, lam, dev(r), psi)
    ref = cb.cheb_filter(lt, r.astype(np.float64), m, lam)
    assert rel(psi.cpu().numpy(), ref) < FP32_TOL
    mu_ref = cb.moments(lt, r.astype(np.float64), 2 * m)
    assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0]


@pytest.mark.parametrize("m", [1, 2, 3, 100])
def test_cheb_filter_orders(gpu_lib, cfg1_graph, m):
    g = cfg1_graph
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(g.n, 24, 24, seed=m)
    with gpu_lib.Context() as ctx:
        upload_graph(ctx, g)
        psi = np.zeros((g.n, 24), dtype=np.float32)     # host output buffer
        mu = ctx.cheb_filter(m, 1.1, r, psi)           # host input block
    assert rel(psi, cb.cheb_filter(lt, r.astype(np.float64), m, 1.1)) < FP32_TOL
    mu_ref = cb.moments(lt, r.astype(np.float64), 2 * m)
    assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0]


@pytest.mark.parametrize("reorder", [1, 0])
def test_cheb_filter_weighted_and_isolated(gpu_lib, reorder):
    g = W.random_csr(3001, 9, seed=4, isolated=40)
    rng = np.random.default_rng(0)
    upper_w = rng.uniform(0.1, 3.0, g.nnz)
    # symmetric weights: weight of (u,v) equals weight of (v,u)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key_lo = np.minimum(rows, g.col_idx) * g.n + np.maximum(rows, g.col_idx)
    _, inv = np.unique(key_lo, return_inverse=True)
    vals = upper_w[inv].astype(np.float32)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, vals)
    r = W.gaussian_block(g.n, 20, 32, seed=2)
    with gpu_lib.Context({"col_tile": 16, "reorder": reorder}) as ctx:
        upload_graph(ctx, g, vals)
        psi = torch.zeros((g.n, 20), device="cuda")
        ctx.cheb_filter(40, 0.8, dev(r), psi)
    assert rel(psi.cpu().numpy(), cb.cheb_filter(lt, r.astype(np.float64), 40, 0.8)) < FP32_TOL


def _hub_graph(n=20000, deg=10, hubs=3, hub_degree=7000, seed=8):
    """Sparse random graph plus a few hubs of very high degree (CSR, symmetric, no self-loops):
    every row block holding a hub has more edges than the step kernel stages in shared memory."""
    rng = np.random.default_rng(seed)
    m = n * deg // 2
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    hub_ids = rng.choice(n, hubs, replace=False)
    hu = np.repeat(hub_ids, hub_degree)
    hv = rng.integers(0, n, hubs * hub_degree)
    u, v = np.concatenate([u, hu]), np.concatenate([v, hv])
    keep = u != v
    u, v = u[keep], v[keep]
    keys = np.unique(np.concatenate([u * n + v, v * n + u]))
    rows, cols = keys // n, keys % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return n, np.cumsum(row_ptr), cols.astype(np.int32)


@pytest.mark.parametrize("reorder", [1, 0])
@pytest.mark.parametrize("tile", [8, 32, 64])
def test_cheb_filter_hub_rows_beyond_the_staging_buffer(gpu_lib, tile, reorder):
    n, rp, ci = _hub_graph()
    assert np.diff(rp).max() > 5632  # one hub row alone exceeds the staged edge buffer
    lt = lp.shifted_laplacian(n, rp, ci)
    r = W.gaussian_block(n, 40, 64, seed=9)
    with gpu_lib.Context({"col_tile": tile, "reorder": reorder}) as ctx:
        ctx.set_graph(n, dev(rp), dev(ci))
        psi = torch.zeros((n, 40), device="cuda")
        mu = ctx.cheb_filter(50, 0.7, dev(r), psi)
    ref = cb.cheb_filter(lt, r.astype(np.float64), 50, 0.7)
    assert rel(psi.cpu().numpy(), ref) < FP32_TOL
    mu_ref = cb.moments(lt, r.astype(np.float64), 100)
    assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0]


@pytest.mark.parametrize("reorder", [1, 0])
@pytest.mark.parametrize("tile", [8, 32])
def test_cheb_filter_power_law_graph(gpu_lib, tile, reorder):
    """Chung-Lu graph with power-law degrees (exponent 2.5) and planted communities, the graph
    class of the large workload: rows from degree 0 to about a thousand in one graph, so chunks
    run from one slot per row to a whole warp per row (rows too long to stage are the hub
    test's)."""
    g = W.chung_lu_graph_torch(60000, 2.5, 25.0, 16, 0.2, seed=12).to_numpy()
    deg = np.diff(g.row_ptr)
    assert deg.max() > 512 and (deg == 0).any()
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(g.n, 24, 64, seed=3)
    with gpu_lib.Context({"col_tile": tile, "reorder": reorder}) as ctx:
        upload_graph(ctx, g)
        psi = torch.zeros((g.n, 24), device="cuda")
        mu = ctx.cheb_filter(40, 0.3, dev(r), psi)
    ref = cb.cheb_filter(lt, r.astype(np.float64), 40, 0.3)
    assert rel(psi.cpu().numpy(), ref) < FP32_TOL
    mu_ref = cb.moments(lt, r.astype(np.float64), 80)
    assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0]


def test_cheb_filter_edgeless_graph(gpu_lib):
    n = 257
    g_rp = np.zeros(n + 1, dtype=np.int64)
    g_ci = np.zeros(0, dtype=np.int32)
    r = W.gaussian_block(n, 5, 5, seed=1)
    m, lam = 7, 0.9
    with gpu_lib.Context() as ctx:
        ctx.set_graph(n, g_rp, g_ci)
        psi = np.zeros((n, 5), dtype=np.float32)
        ctx.cheb_filter(m, lam, r, psi)
    a = cb.filter_coefficients(m, lam)
    # every node isolated: T_j(0) = cos(j pi / 2) -> h(1) = a0 - a2 + a4 - a6
    expect = (a[0] - a[2] + a[4] - a[6]) * r.astype(np.float64)
    np.testing.assert_allclose(psi, expect, rtol=2e-6, atol=1e-7)


def test_cheb_filter_bf16_signals(gpu_lib, cfg1_graph):
    g = cfg1_graph
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(g.n, 64, 64, seed=5)
    rb = torch.from_numpy(r).to(torch.bfloat16)
    r_widened = rb.float().numpy().astype(np.float64)   # the exact stored values
    with gpu_lib.Context() as ctx:
        upload_graph(ctx, g)
        psi = torch.zeros((g.n, 64), device="cuda")
        ctx.cheb_filter(50, 0.53, rb.cuda(), psi)
    got = psi.cpu().numpy()
    assert rel(got, cb.cheb_filter(lt, r_widened, 50, 0.53)) < FP32_TOL
    err_fp64_signals = rel(got, cb.cheb_filter(lt, r.astype(np.float64), 50, 0.53))
    assert err_fp64_signals < BF16_TOL


def test_estimate_lambda_matches_oracle_dichotomy(gpu_lib, cfg1_graph):
    g = cfg1_graph
    k, m, d, seed = 10, 50, 64, 99
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    basis = cb.cheb_basis(lt, gaussian_columns(seed, g.n, np.arange(d), d), m)

    def count(lam):
        return cb.eigencount(cb.combine(basis, cb.filter_coefficients(m, lam)), d)

    lam_ref, cnt_ref, ev_ref = cb.lambda_search(count, k, cb.count_tolerance(k, d), None, 30)
    with gpu_lib.Context() as ctx:
        upload_graph(ctx, g)
        lam, cnt, ev = ctx.estimate_lambda_k(k, m, d, seed)
    assert (lam, ev) == (lam_ref, ev_ref)
    assert cnt == pytest.approx(cnt_ref, rel=1e-4)


def test_estimate_lambda_with_the_trace_estimator(gpu_lib, cfg1_graph):
    """csc_opts.estimator = 1: the dichotomy on the Hutchinson count (d/c) tr(R^T h(L) R)."""
    g = cfg1_graph
    k, m, d, seed = 10, 50, 64, 99
    r = gaussian_columns(seed, g.n, np.arange(d), d)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    basis = cb.cheb_basis(lt, r, m)

    def count(lam):
        return cb.trace_count(r, cb.combine(basis, cb.filter_coefficients(m, lam)), d)

    lam_ref, cnt_ref, ev_ref = cb.lambda_search(count, k, cb.count_tolerance(k, d), None, 30)
    with gpu_lib.Context({"estimator": 1}) as ctx:
        upload_graph(ctx, g)
        lam, cnt, ev = ctx.estimate_lambda_k(k, m, d, seed)
    assert (lam, ev) == (lam_ref, ev_ref)
    assert cnt == pytest.approx(cnt_ref, rel=1e-4)
    with gpu_lib.Context() as ctx:
        upload_graph(ctx, g)
        lam0, _, _ = ctx.estimate_lambda_k(k, m, d, seed)
    assert lam0 != lam        # the two estimators target different traces


def _kmeans_case(n, d, k, seed, dtype=np.float32):
    y, _ = W.clustered_points(n, d, k, seed=seed, spread=0.6)
    return y.astype(dtype), W.forgy_indices(n, k, seed=seed + 1)


# (5000, 256, 200) does not fit the tensor-core pass's shared-memory plan and takes the
# bound-pruned pass; (5000, 1024, 16) runs the tensor-core pass over 16 K chunks.
@pytest.mark.parametrize("n,d,k", [(20000, 64, 10), (20011, 37, 100), (5000, 256, 100), (777, 8, 3),
                                   (5000, 256, 200), (5000, 1024, 16)])
def test_kmeans_exact_assignments(gpu_lib, n, d, k):
    y, idx = _kmeans_case(n, d, k, seed=n + d)
    lab_ref, c_ref, it_ref, conv_ref = km.lloyd(y, km.forgy_centroids(y, idx), max_iter=100)
    with gpu_lib.Context() as ctx:
        out = ctx.kmeans(dev(y), k, idx, max_iter=100, assign_out=torch.zeros(n, dtype=torch.int32,
                                                                               device="cuda"))
    assign = out["assign"].cpu().numpy()
    np.testing.assert_array_equal(assign, lab_ref)
    assert out["iters"] == it_ref
    np.testing.assert_allclose(out["centroids"], c_ref, rtol=0, atol=1e-12)
    assert out["inertia"] == pytest.approx(km.inertia(y, lab_ref, c_ref), rel=1e-5)


def test_kmeans_warm_start_and_bf16(gpu_lib):
    n, d, k = 9000, 48, 12
    y, idx = _kmeans_case(n, d, k, seed=3)
    prev = np.random.default_rng(1).integers(0, k, n).astype(np.int32)
    prev[:k] = np.arange(k)
    prev[prev == 5] = 4                       # cluster 5 empty -> takes row idx[5]
    lab_ref, c_ref, it_ref, _ = km.lloyd(y, km.warm_centroids(y, prev, idx), max_iter=100)
    with gpu_lib.Context() as ctx:
        out = ctx.kmeans(y, k, idx, prev_assign=prev, max_iter=100)
    np.testing.assert_array_equal(out["assign"], lab_ref)
    assert out["iters"] == it_ref
    yb = torch.from_numpy(y).to(torch.bfloat16)
    yw = yb.float().numpy()
    lab_b, _, it_b, _ = km.lloyd(yw, km.forgy_centroids(yw, idx), max_iter=100)
    with gpu_lib.Context() as ctx:
        out = ctx.kmeans(yb.cuda(), k, idx, max_iter=100)
    np.testing.assert_array_equal(out["assign"], lab_b)
    assert out["iters"] == it_b


def test_full_size_kmeans_update_and_sampled_rows(gpu_lib):
    """n = 1e6 float32 rows, d = 256, k = 100 (the clustering size of the dynamic workload).

    Runs of 2 and 3 passes from the same Forgy rows: the oracle recomputes the update between
    them on all rows (the centroids of the 3-pass run are the float64 means of the 2-pass
    assignment), and the assignment of sampled rows against the centroids each run used."""
    n, d, k = 1_000_000, 256, 100
    y, _ = W.clustered_points(n, d, k, seed=11, spread=0.6)
    idx = W.forgy_indices(n, k, seed=12)
    yd = dev(y)
    runs = []
    for passes in (2, 3):
        with gpu_lib.Context() as ctx:
            out = ctx.kmeans(yd, k, idx, max_iter=passes,
                             assign_out=torch.zeros(n, dtype=torch.int32, device="cuda"))
        runs.append((out["assign"].cpu().numpy(), out["centroids"], out["iters"]))
    (la, ca, ia), (lb, cb3, ib) = runs
    assert (ia, ib) == (2, 3)
    np.testing.assert_allclose(cb3, km.update(y, la, ca), rtol=0, atol=1e-12)
    sample = np.random.default_rng(5).choice(n, 20000, replace=False)
    for lab, c in ((la, ca), (lb, cb3)):
        ref, _ = km.assign(y[sample], c)
        np.testing.assert_array_equal(lab[sample], ref)


@pytest.mark.parametrize("k", [16, 200])
def test_kmeans_rejects_bad_inputs(gpu_lib, k):
    """Non-finite features and (device) previous labels outside [0, k) are argument errors,
    on the tensor-core path (k = 16) and the bound-pruned path (k = 200)."""
    y, idx = _kmeans_case(3000, 256, k, seed=9)
    bad = y.copy()
    bad[17, 3] = np.nan
    with gpu_lib.Context() as ctx:
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.kmeans(dev(bad), k, idx, max_iter=5)
        assert e.value.status == 1
        prev = torch.zeros(3000, dtype=torch.int32, device="cuda")
        prev[5] = k
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.kmeans(dev(y), k, idx, prev_assign=prev, max_iter=5,
                       assign_out=torch.zeros(3000, dtype=torch.int32, device="cuda"))
        assert e.value.status == 1
        out = ctx.kmeans(dev(y), k, idx, max_iter=5)   # the context stays usable
        assert out["iters"] >= 1


def test_kmeans_exact_ties_lowest_index(gpu_lib):
    # duplicated centroid rows make every distance to centroids 0 and 1 exactly equal
    y, _ = W.clustered_points(3000, 16, 4, seed=6)
    y[1] = y[0]
    idx = np.array([0, 1, 2, 3])
    lab_ref, _, it_ref, _ = km.lloyd(y, km.forgy_centroids(y, idx), max_iter=3)
    with gpu_lib.Context() as ctx:
        out = ctx.kmeans(y, 4, idx, max_iter=3)
    np.testing.assert_array_equal(out["assign"], lab_ref)


@pytest.mark.parametrize("bf16", [False, True])
def test_kmeans_bound_skipping_is_exact(gpu_lib, bf16):
    """Hamerly skipping on the tensor-core pass, on overlapping clusters that take many Lloyd
    passes: the assignment, the pass count and the centroids equal the oracle's plain Lloyd
    (Section 2.1, Eq. 1), and the passes after the first evaluate fewer than all rows
    (csc_stats.kmeans_rows)."""
    n, d, k = 60000, 64, 40
    y, _ = W.clustered_points(n, d, k, seed=21, spread=1.2)
    idx = W.forgy_indices(n, k, seed=22)
    if bf16:
        yt = torch.from_numpy(y).to(torch.bfloat16)
        y = yt.float().numpy()
    else:
        yt = torch.from_numpy(y)
    lab_ref, c_ref, it_ref, _ = km.lloyd(y.astype(np.float64), km.forgy_centroids(y, idx), max_iter=100)
    with gpu_lib.Context() as ctx:
        out = ctx.kmeans(yt.cuda(), k, idx, max_iter=100,
                         assign_out=torch.zeros(n, dtype=torch.int32, device="cuda"))
        st = ctx.stats()
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab_ref)
    assert out["iters"] == it_ref and it_ref >= 10
    np.testing.assert_allclose(out["centroids"], c_ref, rtol=0, atol=1e-12)
    assert st["kmeans_passes"] == it_ref
    print(f"passes {it_ref}, rows evaluated {st['kmeans_rows']} of {it_ref * n}")
    assert n <= st["kmeans_rows"] < 0.6 * it_ref * n


@pytest.mark.parametrize("reorder", [1, 0, 2])
def test_algorithm1_dynamic_parity_cfg1(gpu_lib, cfg1_graph, reorder):
    """SBM n=2000, k=10, degree 20, d=64, m=50, 1% rewiring per step, p=0.5: 1 + 5 snapshots."""
    n, k, d, m, p, seed = 2000, 10, 64, 50, 0.5, 2024
    graphs = [cfg1_graph]
    for t in range(5):
        graphs.append(W.edge_redraw(graphs[-1], 0.01, seed=100 + t))
    oracle = DynamicCSC(n, k, d, p, m, seed)
    with gpu_lib.Context({"reorder": reorder}) as ctx:
        assign = torch.zeros(n, dtype=torch.int32, device="cuda")
        for t, g in enumerate(graphs):
            idx = W.forgy_indices(n, k, seed=500 + t)
            lab_ref = oracle.step(g.row_ptr, g.col_idx, init_idx=idx)
            h = oracle.history[-1]
            upload_graph(ctx, g)
            lam, cnt, ev, cols = ctx.filter(m, d, p, seed, k)
            cost, iters = ctx.cluster(k, seed, idx, assign)
            assert cols == h["c"]
            assert lam == h["lam"], (t, lam, h)
            assert ev == h["evals"], (t, ev, h)
            assert cnt == pytest.approx(h["count"], rel=1e-4)
            theta = np.zeros((n, d), dtype=np.float32)
            ctx.get_features(theta)
            assert rel(theta, oracle.features()) < FP32_TOL
            y = np.zeros((n, d), dtype=np.float32)
            ctx.get_features(y, normalized=True)
            assert rel(y, row_normalize(oracle.features())) < FP32_TOL
            np.testing.assert_array_equal(assign.cpu().numpy(), lab_ref)
            assert iters == h["passes"]
            assert cost == pytest.approx(math.sqrt(h["inertia"]), rel=1e-5)


def test_algorithm1_dynamic_bf16_storage(gpu_lib, cfg1_graph):
    """The same dynamic sequence with bfloat16 signal and feature storage (float32 recursion,
    float64 moments): features within 3e-3 of the float64-signal oracle, the same cutoffs, and
    k-means assignments equal to the oracle's Lloyd iteration run on the GPU's own bfloat16
    features (Forgy at t = 1, warm start from the previous assignment after)."""
    n, k, d, m, p, seed = 2000, 10, 64, 50, 0.5, 2024
    graphs = [cfg1_graph]
    for t in range(5):
        graphs.append(W.edge_redraw(graphs[-1], 0.01, seed=100 + t))
    oracle = DynamicCSC(n, k, d, p, m, seed)
    prev = None
    with gpu_lib.Context({"precision": 1}) as ctx:
        assign = torch.zeros(n, dtype=torch.int32, device="cuda")
        for t, g in enumerate(graphs):
            idx = W.forgy_indices(n, k, seed=500 + t)
            oracle.step(g.row_ptr, g.col_idx, init_idx=idx)
            h = oracle.history[-1]
            upload_graph(ctx, g)
            lam, cnt, ev, cols = ctx.filter(m, d, p, seed, k)
            ctx.cluster(k, seed, idx, assign)
            assert cols == h["c"]
            assert lam == h["lam"], (t, lam, h)
            assert cnt == pytest.approx(h["count"], rel=1e-2)
            theta = np.zeros((n, d), dtype=np.float32)
            ctx.get_features(theta)
            err = rel(theta, oracle.features())
            assert err < BF16_TOL, (t, err)
            y = np.zeros((n, d), dtype=np.float32)
            ctx.get_features(y, normalized=True)  # the bfloat16 values, widened exactly
            assert np.array_equal(y, torch.from_numpy(y).to(torch.bfloat16).float().numpy())
            c0 = km.forgy_centroids(y, idx) if prev is None else km.warm_centroids(y, prev, idx)
            lab, _, _, _ = km.lloyd(y, c0, max_iter=100)
            np.testing.assert_array_equal(assign.cpu().numpy(), lab)
            prev = lab


def test_full_size_sampled_columns(gpu_lib):
    """n = 1e6 Zipf SBM (degree 30), 64 columns, m = 100 in the bench's tile configuration;
    the oracle recomputes two sampled columns in float64 (columns are independent).

    At this size the float32 rounding noise of the recursion, which the low-pass does not
    damp, is amplified by about sqrt(n/k) relative to the filtered signal; the tolerance is
    max(1e-5, 2 x the measured float32 floor of the same recursion)."""
    sizes = W.zipf_block_sizes(1_000_000, 100, 0.8)
    g = W.sbm_graph(1_000_000, sizes, 30, 10, seed=2)
    c, d, m, lam = 64, 256, 100, 0.06
    r = W.gaussian_block(g.n, c, d, seed=77)
    with gpu_lib.Context() as ctx:
        upload_graph(ctx, g)
        psi = torch.zeros((g.n, c), device="cuda")
        mu = ctx.cheb_filter(m, lam, dev(r), psi)
        got = psi.cpu().numpy()
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    cols = [0, 37]
    ref = cb.cheb_filter(lt, r[:, cols].astype(np.float64), m, lam)
    floor = fp32_floor(lt, r[:, cols], cb.filter_coefficients(m, lam), ref)
    err = rel(got[:, cols], ref)
    print(f"full-size sampled columns: GPU error {err:.3e}, float32 floor {floor:.3e}")
    assert err < max(FP32_TOL, 2.0 * floor)
    # moment identity at full size: ||Psi||_F^2 from the moments equals the direct norm
    a = cb.filter_coefficients(m, lam)
    i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    via = float(np.sum(a[i] * a[j] * (mu[i + j] + mu[np.abs(i - j)]) / 2.0))
    assert abs(via - float(np.sum(got.astype(np.float64) ** 2))) < 1e-5 * mu[0]


def test_errors_and_call_order(gpu_lib):
    with gpu_lib.Context() as ctx:
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.filter(10, 8, 0.0, 1, 2)
        assert e.value.status == 5  # CSC_ESTATE: no graph
        with pytest.raises(gpu_lib.CscError):
            ctx.set_graph(3, np.array([0, 1, 2, 2], dtype=np.int64), np.array([0, 0], dtype=np.int32))
        assert "self-loop" in ctx.last_error
        with pytest.raises(gpu_lib.CscError):
            ctx.set_graph(3, np.array([0, 1, 2, 2], dtype=np.int64), np.array([5, 0], dtype=np.int32))
        ctx.set_graph(3, np.array([0, 1, 2, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32))
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.cluster(2, 1, None, np.zeros(3, dtype=np.int32))
        assert e.value.status == 5
    with gpu_lib.Context({"checked": 1}) as ctx:
        with pytest.raises(gpu_lib.CscError):
            ctx.set_graph(3, dev(np.array([0, 1, 2, 2], dtype=np.int64)),
                          dev(np.array([5, 0], dtype=np.int32)))  # column out of range
        assert "malformed" in ctx.last_error


def test_algorithm1_similarity_policy_parity(gpu_lib):
    """Algorithm 1 under the edge-similarity policy (csc_filter_adaptive, Theorem 4.1 with
    Corollary 4.2 and Weyl's inequality) over a sequence that alternates node reassignment plus
    edge redrawing (Section 5.2) with light edge redrawing.  The GPU computes rho_t itself
    (csc_laplacian_distance); reuse counts, skipped checks and cutoffs equal the oracle's,
    features within the float32 tolerance, assignments exact."""
    n, k, d, m, p_max, seed = 2000, 10, 64, 50, 0.75, 77
    policy = dict(alpha=0.1, budget=100.0, rho_skip=2.0)
    graphs = [W.sbm_graph(n, k, 20, 10, seed=1)]
    for t in range(6):
        graphs.append(W.sbm_perturb(graphs[-1], 0.01, 0.03, seed=400 + t) if t % 2 == 0
                      else W.edge_redraw(graphs[-1], 0.005, seed=400 + t))
    oracle = DynamicCSC(n, k, d, p_max, m, seed)
    cols_seen, checks_seen = set(), set()
    with gpu_lib.Context() as ctx:
        assign = torch.zeros(n, dtype=torch.int32, device="cuda")
        prev = None
        for t, g in enumerate(graphs):
            cur = (dev(g.row_ptr), dev(g.col_idx), None)
            rho = 0.0 if prev is None else ctx.laplacian_distance(n, prev, cur)
            rho_ref = 0.0 if t == 0 else sm.laplacian_distance(
                n, (graphs[t - 1].row_ptr, graphs[t - 1].col_idx, None), (g.row_ptr, g.col_idx, None))
            assert rho == pytest.approx(rho_ref, rel=1e-10)
            idx = W.forgy_indices(n, k, seed=600 + t)
            lab_ref = oracle.step(g.row_ptr, g.col_idx, init_idx=idx, rho=rho_ref, policy=policy)
            h = oracle.history[-1]
            ctx.set_graph(n, cur[0], cur[1])
            lam, cnt, ev, cols, checked = ctx.filter_adaptive(m, d, p_max, seed, k, rho, **policy)
            ctx.cluster(k, seed, idx, assign)
            assert cols == h["c"] and checked == h["checked"], (t, cols, checked, h)
            assert lam == h["lam"] and ev == h["evals"], (t, lam, ev, h)
            theta = np.zeros((n, d), dtype=np.float32)
            ctx.get_features(theta)
            assert rel(theta, oracle.features()) < FP32_TOL
            np.testing.assert_array_equal(assign.cpu().numpy(), lab_ref)
            cols_seen.add(cols)
            checks_seen.add(checked)
            prev = cur
    # the sequence exercised a reduced reuse, full reuse and both check outcomes
    assert len(cols_seen) >= 3 and checks_seen == {True, False}


@pytest.mark.parametrize("c,tiles", [(39, [32, 8]), (64, [64]), (13, [16]), (192, [64, 64, 64])])
def test_tile_plan_and_step_byte_accounting(gpu_lib, cfg1_graph, c, tiles):
    """The automatic plan covers c columns with tiles of 8..64 minimising sum (8 + w), and the
    library's step_bytes count every timed step launch at its own width."""
    g = cfg1_graph
    m = 6
    r = W.gaussian_block(g.n, c, 64, seed=c)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    with gpu_lib.Context({"timing": 1}) as ctx:
        upload_graph(ctx, g)
        psi = torch.zeros((g.n, c), device="cuda")
        ctx.stats(reset=True)
        ctx.cheb_filter(m, 0.5, dev(r), psi)
        st = ctx.stats()
    assert rel(psi.cpu().numpy(), cb.cheb_filter(lt, r.astype(np.float64), m, 0.5)) < FP32_TOL
    assert st["tile"] == max(tiles) and st["filter_passes"] == len(tiles)
    assert st["step_launches"] == len(tiles) * (m - 1)
    per = lambda w: 4.0 * g.nnz + 8.0 * (g.n + 1) + 4.0 * g.n + g.n * w * (4 + 4 + 4 + 8)
    assert st["step_bytes"] == pytest.approx((m - 1) * sum(per(w) for w in tiles), rel=1e-12)
