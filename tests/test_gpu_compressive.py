"""Compressive k-means on the GPU against oracle/compressive.py (Section 2.2, step 2).

Both sides receive the same seeded features (theta from the float64 oracle filter, cast to
float32, and its float32 row normalisation).  The sample and the reduced labels are integer
or exactly decided work and must be equal; the interpolation is a float32 Chebyshev
filtering compared with the float64 one; the final argmax must agree wherever the oracle's
top-2 gap exceeds the float32 error of the interpolation.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import chebyshev as cb
from oracle import compressive as ck
from oracle import laplacian as lp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _features(g, k, d, m, seed):
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    ev = np.sort(spla.eigsh(lt, k=k + 1, which="SA", return_eigenvectors=False)) + 1.0
    lam = float(0.5 * (ev[k - 1] + ev[k]))
    r = W.gaussian_block(g.n, d, d, seed=seed).astype(np.float64)
    theta = cb.cheb_filter(lt, r, m, lam).astype(np.float32)
    y = (theta / np.linalg.norm(theta, axis=1, keepdims=True)).astype(np.float32)
    return theta, y, lam


def _check_assign(got, x_ref, tol_rel=1e-4):
    """Equal labels where the oracle's top-2 gap exceeds tol; elsewhere a near-maximiser."""
    xs = np.sort(x_ref, axis=1)
    scale = float(np.max(np.abs(x_ref)))
    gap = xs[:, -1] - xs[:, -2]
    ref = ck.argmax_assign(x_ref)
    clear = gap > tol_rel * scale
    np.testing.assert_array_equal(got[clear], ref[clear])
    rows = np.nonzero(~clear)[0]
    assert rows.size <= 0.01 * got.size
    assert np.all(x_ref[rows, got[rows]] >= xs[rows, -1] - tol_rel * scale)


@pytest.mark.parametrize("y_dtype", ["f32", "bf16"])
def test_compressive_parity_small(gpu_lib, y_dtype):
    n, k, d, m = 3000, 6, 48, 50
    g = W.sbm_graph(n, W.zipf_block_sizes(n, k, 0.8), 30, 10, seed=4)
    theta, y, lam = _features(g, k, d, m, seed=31)
    yt = dev(y) if y_dtype == "f32" else dev(y, torch.bfloat16)
    y_ref = yt.float().cpu().numpy()
    n_draws, seed = 60, 0x5EED
    assign = np.zeros(n, dtype=np.int32)
    x = np.zeros((n, k), dtype=np.float32)
    with gpu_lib.Context() as ctx:
        ctx.set_graph(n, dev(g.row_ptr), dev(g.col_idx))
        res = ctx.compressive_cluster(k, dev(theta), yt, n_draws=n_draws, n_init=10, lambda_c=lam, m=m,
                                      seed=seed, assign_out=assign, want_sample=True, interp_out=x)
    ref = ck.compressive_kmeans(n, g.row_ptr, g.col_idx, None, theta, y_ref, k, n_draws, m, lam, seed,
                                max_iter=100, n_init=10)
    np.testing.assert_array_equal(res["sample"], ref["omega"])
    assert res["n_sampled"] == ref["omega"].size
    assert res["restart"] == ref["restart"]
    np.testing.assert_array_equal(res["sample_labels"], ref["labels"])
    err = rel(x, ref["x"])
    print(f"compressive interpolation ({y_dtype}): float32 error {err:.3e}, |Omega| {res['n_sampled']}")
    assert err < FP32_TOL
    _check_assign(assign, ref["x"])


def test_compressive_parity_weighted_with_isolated_nodes(gpu_lib):
    """Symmetric random weights and three isolated nodes (their L~ rows are zero, so the
    interpolation there is h(1) z): same sample, restart, labels and interpolation."""
    n, k, d, m = 2500, 5, 40, 40
    g = W.sbm_graph(n, k, 25, 20, seed=9)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    iso = np.array([3, 700, 2499])
    keep = ~np.isin(rows, iso) & ~np.isin(g.col_idx, iso)
    rows, cols = rows[keep], g.col_idx[keep].astype(np.int32)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    key = np.minimum(rows, cols).astype(np.int64) * n + np.maximum(rows, cols)
    _, inv = np.unique(key, return_inverse=True)
    vals = np.random.default_rng(2).uniform(0.5, 2.0, inv.max() + 1)[inv].astype(np.float32)
    lt = lp.shifted_laplacian(n, rp, cols, vals)
    lam = 0.35
    r = W.gaussian_block(n, d, d, seed=12).astype(np.float64)
    theta = cb.cheb_filter(lt, r, m, lam).astype(np.float32)
    y = (theta / np.linalg.norm(theta, axis=1, keepdims=True)).astype(np.float32)
    assign = np.zeros(n, dtype=np.int32)
    x = np.zeros((n, k), dtype=np.float32)
    with gpu_lib.Context() as ctx:
        ctx.set_graph(n, dev(rp), dev(cols), dev(vals))
        res = ctx.compressive_cluster(k, dev(theta), dev(y), n_draws=80, n_init=5, lambda_c=lam, m=m,
                                      seed=21, assign_out=assign, want_sample=True, interp_out=x)
    ref = ck.compressive_kmeans(n, rp, cols, vals, theta, y, k, 80, m, lam, 21, n_init=5)
    np.testing.assert_array_equal(res["sample"], ref["omega"])
    assert res["restart"] == ref["restart"]
    np.testing.assert_array_equal(res["sample_labels"], ref["labels"])
    err = rel(x, ref["x"])
    print(f"weighted compressive interpolation: float32 error {err:.3e}")
    assert err < FP32_TOL
    _check_assign(assign, ref["x"])


def test_compressive_on_context_features(gpu_lib):
    """After csc_filter, the call on the context's own features: same moments afterwards,
    and an assignment close to the full k-means of the same features."""
    g = W.sbm_graph(2000, 10, 20, 10, seed=1)
    k, m, d = 10, 50, 64
    with gpu_lib.Context() as ctx:
        ctx.set_graph(g.n, dev(g.row_ptr), dev(g.col_idx))
        ctx.filter(m, d, 0.5, 7, k)
        mu_before = gpu_lib.csc_get_moments(ctx.h, 2 * m + 1)
        full = np.zeros(g.n, dtype=np.int32)
        gpu_lib.csc_cluster(ctx.h, k, 3, None, full)
        comp = np.zeros(g.n, dtype=np.int32)
        res = ctx.compressive_cluster(k, n_draws=200, seed=9, assign_out=comp, want_sample=True)
        mu_after = gpu_lib.csc_get_moments(ctx.h, 2 * m + 1)
    np.testing.assert_array_equal(mu_before, mu_after)
    assert 0 < res["n_sampled"] <= 200 and np.all(np.diff(res["sample"]) > 0)
    c = np.zeros((k, k))
    np.add.at(c, (comp, full), 1)
    from scipy.optimize import linear_sum_assignment
    r, cc = linear_sum_assignment(-c)
    agree = c[r, cc].sum() / g.n
    print(f"compressive vs full k-means on the context features: {agree:.3f}")
    assert agree > 0.9


def test_compressive_errors(gpu_lib):
    n, d = 500, 8
    g = W.sbm_graph(n, 4, 10, 10, seed=3)
    out = np.zeros(n, dtype=np.int32)
    with gpu_lib.Context() as ctx:
        with pytest.raises(gpu_lib.CscError):        # no graph
            ctx.compressive_cluster(4, assign_out=out)
        ctx.set_graph(n, dev(g.row_ptr), dev(g.col_idx))
        with pytest.raises(gpu_lib.CscError):        # context features before csc_filter
            ctx.compressive_cluster(4, assign_out=out)
        zero = np.zeros((n, d), dtype=np.float32)
        with pytest.raises(gpu_lib.CscError, match="all zero"):
            ctx.compressive_cluster(4, dev(zero), dev(zero), lambda_c=0.5, m=10, assign_out=out)
        theta = W.gaussian_block(n, d, d, seed=5).astype(np.float32)
        y = theta / np.linalg.norm(theta, axis=1, keepdims=True)
        with pytest.raises(gpu_lib.CscError, match="raise n_draws"):
            ctx.compressive_cluster(6, dev(theta), dev(y), n_draws=3, lambda_c=0.5, m=10, assign_out=out)
        with pytest.raises(gpu_lib.CscError):        # cutoff outside [0, 2]
            ctx.compressive_cluster(4, dev(theta), dev(y), lambda_c=2.5, m=10, assign_out=out)
        # host features are staged; the context stays usable after the errors
        res = ctx.compressive_cluster(4, theta, y, n_draws=40, lambda_c=0.5, m=10, seed=1, assign_out=out,
                                      want_sample=True)
        ref = ck.sample(theta, 40, 1)[0]
        np.testing.assert_array_equal(res["sample"], ref)
        assert out.min() >= 0 and out.max() < 4


def test_compressive_full_size(gpu_lib):
    """n = 1e6 Zipf SBM (degree 30), k = 100, d = 256, the default 2 k ln k draws: exact sample,
    restart and reduced labels; two interpolated columns recomputed by the oracle in float64."""
    n, k, d, m, lam = 1_000_000, 100, 256, 30, 0.06
    g = W.sbm_graph(n, W.zipf_block_sizes(n, k, 0.8), 30, 10, seed=2)
    theta = W.gaussian_block(n, d, d, seed=91)
    y = (theta / np.linalg.norm(theta, axis=1, keepdims=True)).astype(np.float32)
    seed, n_init = 77, 3
    assign = np.zeros(n, dtype=np.int32)
    x = np.zeros((n, k), dtype=np.float32)
    with gpu_lib.Context() as ctx:
        ctx.set_graph(n, dev(g.row_ptr), dev(g.col_idx))
        res = ctx.compressive_cluster(k, dev(theta), dev(y), n_init=n_init, lambda_c=lam, m=m, seed=seed,
                                      assign_out=assign, want_sample=True, interp_out=x)
    omega, q, total = ck.sample(theta, int(np.ceil(2 * k * np.log(k))), seed)
    np.testing.assert_array_equal(res["sample"], omega)
    labels, _, restart = ck.reduced_kmeans(y, omega, k, seed, 100, n_init)
    assert res["restart"] == restart
    np.testing.assert_array_equal(res["sample_labels"], labels)
    z = ck.tikhonov_rhs(n, k, omega, labels, ck.sample_weights(q, total, omega))
    lt = lp.shifted_laplacian(n, g.row_ptr, g.col_idx)
    cols = sorted({int(labels[0]), int(labels[-1])})
    ref = cb.cheb_filter(lt, z[:, cols], m, lam)
    err = rel(x[:, cols], ref)
    print(f"full-size compressive interpolation: float32 error {err:.3e}, |Omega| {omega.size}")
    assert err < FP32_TOL
    # the assignment is the row argmax (lowest index on ties) of the returned interpolation
    np.testing.assert_array_equal(assign, ck.argmax_assign(x))
