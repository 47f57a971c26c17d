"""Differentiation through the filter (csc_filter_forward, csc_filter_vjp, csc_kmeans_loss_grad,
the torch.autograd layer) against the float64 gradient oracle.

Loss: the k-means cost of the row-normalised features against fixed centroids and a fixed
assignment.  Checks: features and dloss/dPsi against the oracle; the vector-Jacobian product
(coefficients and every edge weight) against the oracle's adjoint; central finite differences
(h = 1e-3) of the float64 loss on 64 random coordinates; at the size of the differentiation
workload (SBM n = 2e5, k = 20, degree 25, d = 128, m = 60) the product restricted to sampled
columns (it is linear in dloss/dPsi and separates by column) and Euler's relation.
"""
import numpy as np
import pytest

import workloads as W
from conftest import fp32_floor
from oracle import chebyshev as cb
from oracle import grad as gr
from oracle import laplacian as lp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sym_weights(g, seed):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = np.minimum(rows, g.col_idx).astype(np.int64) * g.n + np.maximum(rows, g.col_idx)
    _, inv = np.unique(key, return_inverse=True)
    return np.random.default_rng(seed).uniform(0.5, 2.0, inv.max() + 1)[inv].astype(np.float32)


def small_case(c, seed=7):
    g = W.sbm_graph(2000, 10, 20, 10, seed=seed)
    w = sym_weights(g, seed)
    rng = np.random.default_rng(seed)
    r = (rng.standard_normal((g.n, c)) / np.sqrt(c)).astype(np.float32)
    a = cb.filter_coefficients(60, 0.5)
    mu = rng.standard_normal((10, c))
    mu = (mu / np.linalg.norm(mu, axis=1, keepdims=True)).astype(np.float32)
    assign = rng.integers(0, 10, g.n).astype(np.int32)
    return g, w, r, a, mu, assign


def gpu_grads(gpu_lib, g, w, r, a, mu, assign, stride, reorder=1):
    with gpu_lib.Context({"reorder": reorder}) as ctx:
        ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(),
                      None if w is None else torch.from_numpy(w).cuda())
        rt = torch.from_numpy(r).cuda()
        psi = torch.zeros((g.n, r.shape[1]), device="cuda")
        ctx.filter_forward(a.size - 1, a, rt, psi, stride)
        gpsi = torch.zeros_like(psi)
        loss = ctx.kmeans_loss_grad(psi, torch.from_numpy(mu).cuda(), torch.from_numpy(assign).cuda(), gpsi)
        gw = torch.zeros(g.col_idx.size, device="cuda")
        ga = ctx.filter_vjp(gpsi, gw)
        return psi.cpu().numpy(), loss, gpsi.cpu().numpy(), ga, gw.cpu().numpy()


@pytest.mark.parametrize("c,stride,reorder", [(16, 0, 1), (16, 1, 1), (130, 7, 1), (16, 0, 0), (40, 16, 1), (64, 1, 0)])
def test_gradients_match_oracle_and_finite_differences(gpu_lib, c, stride, reorder):
    g, w, r, a, mu, assign = small_case(c)
    psi, loss, gpsi, ga, gw = gpu_grads(gpu_lib, g, w, r, a, mu, assign, stride, reorder)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, w)
    psi_ref = gr.filter_psi(lt, r, a)
    assert rel(psi, psi_ref) < 1e-5
    loss_ref, gpsi_ref = gr.kmeans_loss_grad(psi, mu, assign)  # same (GPU) features
    assert loss == pytest.approx(loss_ref, rel=1e-9)
    assert rel(gpsi, gpsi_ref) < 1e-5
    ga_ref, gl_ref = gr.filter_vjp(lt, r, a, gpsi.astype(np.float64))
    gw_ref = gr.edge_weight_grad(g.n, g.row_ptr, g.col_idx, w, gl_ref)
    assert rel(ga, ga_ref) < 1e-4
    assert rel(gw, gw_ref) < 1e-4
    # central differences of the float64 loss on 64 random coordinates (coefficients and edges)
    rng = np.random.default_rng(c + stride + 100 * reorder)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    w64 = w.astype(np.float64)

    def loss64(a_, w_):
        return gr.kmeans_loss(gr.filter_psi(lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, w_), r, a_), mu, assign)

    h = 1e-3
    coords = [("a", j) for j in rng.choice(a.size, 8, replace=False)]
    coords += [("w", e) for e in rng.choice(np.flatnonzero(rows < g.col_idx), 56, replace=False)]
    for kind, idx in coords:
        if kind == "a":
            e = np.zeros_like(a)
            e[idx] = h
            fd = (loss64(a + e, w64) - loss64(a - e, w64)) / (2 * h)
            got = ga[idx]
        else:
            u, v = rows[idx], g.col_idx[idx]
            both = (rows == u) & (g.col_idx == v) | (rows == v) & (g.col_idx == u)
            wp, wm = w64.copy(), w64.copy()
            wp[both] += h
            wm[both] -= h
            fd = (loss64(a, wp) - loss64(a, wm)) / (2 * h)
            got = gw[idx]
        # h = 1e-3 central differences carry an O(h^2) truncation error (a few 1e-3 here);
        # a wrong factor, sign or term shows up as an O(1) mismatch
        scale = float(np.max(np.abs(ga))) if kind == "a" else float(np.max(np.abs(gw)))
        assert abs(got - fd) <= 1e-2 * abs(fd) + 1e-5 * scale, (kind, idx, got, fd)


def test_autograd_layer(gpu_lib):
    g, w, r, a, mu, assign = small_case(16, seed=11)
    with gpu_lib.Context() as ctx:
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        wt = torch.from_numpy(w).cuda().requires_grad_(True)
        at = torch.from_numpy(a).requires_grad_(True)
        psi = gpu_lib.cheb_filter_layer(ctx, g.n, rp, ci, wt, at, torch.from_numpy(r).cuda())
        y = psi / psi.norm(dim=1, keepdim=True)
        mut = torch.from_numpy(mu).cuda()
        loss = ((y - mut[torch.from_numpy(assign).long().cuda()]) ** 2).sum()
        loss.backward()
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, w)
    loss_ref, ga_ref, gw_ref = gr.loss_and_grads(g.n, g.row_ptr, g.col_idx, w.astype(np.float64), r, a, mu, assign)
    assert float(loss.detach()) == pytest.approx(loss_ref, rel=1e-5)
    assert rel(at.grad.numpy(), ga_ref) < 1e-4
    assert rel(wt.grad.cpu().numpy(), gw_ref) < 1e-4
    assert lt.nnz == g.col_idx.size


def test_gradient_at_differentiation_workload_size(gpu_lib):
    """SBM n = 2e5, k = 20, degree 25, d = 128, m = 60, unit weights, checkpoints every 8 steps."""
    g = W.sbm_graph(200_000, 20, 25, 10, seed=4)
    c, m, k = 128, 60, 20
    rng = np.random.default_rng(4)
    r = (rng.standard_normal((g.n, c)) / np.sqrt(c)).astype(np.float32)
    a = cb.filter_coefficients(m, 0.3)
    mu = rng.standard_normal((k, c))
    mu = (mu / np.linalg.norm(mu, axis=1, keepdims=True)).astype(np.float32)
    assign = rng.integers(0, k, g.n).astype(np.int32)
    cols = [3, 100]
    with gpu_lib.Context() as ctx:
        ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
        rt = torch.from_numpy(r).cuda()
        psi = torch.zeros((g.n, c), device="cuda")
        ctx.filter_forward(m, a, rt, psi, 0)
        gpsi = torch.zeros_like(psi)
        ctx.kmeans_loss_grad(psi, torch.from_numpy(mu).cuda(), torch.from_numpy(assign).cuda(), gpsi)
        gw_full = torch.zeros(g.col_idx.size, device="cuda")
        ctx.filter_vjp(gpsi, gw_full)
        # the product restricted to two columns of dloss/dPsi
        gmask = torch.zeros_like(gpsi)
        gmask[:, cols] = gpsi[:, cols]
        gw_cols = torch.zeros(g.col_idx.size, device="cuda")
        ga_cols = ctx.filter_vjp(gmask, gw_cols)
        psi_h, gpsi_h = psi.cpu().numpy(), gpsi.cpu().numpy()
        gw_full, gw_cols = gw_full.cpu().numpy(), gw_cols.cpu().numpy()
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    ref_cols = gr.filter_psi(lt, r[:, cols], a)
    floor = fp32_floor(lt, r[:, cols], a, ref_cols)
    err_psi = rel(psi_h[:, cols], ref_cols)
    _, gpsi_ref = gr.kmeans_loss_grad(psi_h, mu, assign)
    ga_ref, gl_ref = gr.filter_vjp(lt, r[:, cols], a, gpsi_h[:, cols].astype(np.float64))
    gw_ref = gr.edge_weight_grad(g.n, g.row_ptr, g.col_idx, None, gl_ref)
    err_a, err_w = rel(ga_cols, ga_ref), rel(gw_cols, gw_ref)
    print(f"n=2e5: psi error {err_psi:.3e} (float32 floor {floor:.3e}), dloss/da {err_a:.3e}, dloss/dw {err_w:.3e}")
    assert err_psi < max(1e-5, 2.0 * floor)
    assert rel(gpsi_h, gpsi_ref) < 1e-5
    assert err_a < max(1e-4, 10.0 * floor)
    assert err_w < max(1e-4, 10.0 * floor)
    # Euler's relation on the full product (unit weights): sum_e dloss/dw_e = 0
    assert abs(float(np.sum(gw_full.astype(np.float64)))) < 1e-4 * float(np.sum(np.abs(gw_full)))


def test_gradient_call_order_and_errors(gpu_lib):
    g, w, r, a, mu, assign = small_case(8)
    with gpu_lib.Context() as ctx:
        gpsi = torch.zeros((g.n, 8), device="cuda")
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.filter_vjp(gpsi)
        assert e.value.status == 5  # no forward pass yet
        ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
        psi = torch.zeros((g.n, 8), device="cuda")
        ctx.filter_forward(60, a, torch.from_numpy(r).cuda(), psi)
        ctx.set_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.filter_vjp(gpsi)
        assert e.value.status == 5  # a new graph invalidates the forward state
        bad = torch.from_numpy(assign).cuda()
        bad[3] = 10
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.kmeans_loss_grad(psi, torch.from_numpy(mu).cuda(), bad, gpsi)
        assert e.value.status == 1
