"""Pins of the gradient oracle (oracle/grad.py) against the plain forward evaluation.

The analytic gradients come from the adjoint of the Chebyshev recursion and the chain rule
through the normalized Laplacian; here they are compared with central finite differences of
the loss computed by the forward recursion alone, for every coefficient and every edge of a
small weighted graph with an isolated node, and with Euler's relation for the weights.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grad as gr
from oracle import laplacian as lp


def _case(seed=3, n=48, k=3, d=5, m=7):
    g = W.sbm_graph(n, k, 6, 10, seed=seed)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = np.minimum(rows, g.col_idx) * g.n + np.maximum(rows, g.col_idx)
    _, inv = np.unique(key, return_inverse=True)
    w = rng.uniform(0.5, 2.0, inv.max() + 1)[inv]
    # one isolated node: drop every edge of node 0
    keep = (rows != 0) & (g.col_idx != 0)
    rows2, cols2, w2 = rows[keep], g.col_idx[keep], w[keep]
    row_ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows2 + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    r = rng.standard_normal((g.n, d)) / np.sqrt(d)
    a = rng.standard_normal(m + 1) * 0.5
    mu = rng.standard_normal((k, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    assign = rng.integers(0, k, g.n)
    return g.n, row_ptr, cols2.astype(np.int64), w2, r, a, mu, assign


def _loss(n, row_ptr, col_idx, w, r, a, mu, assign):
    lt = lp.shifted_laplacian(n, row_ptr, col_idx, w)
    return gr.kmeans_loss(gr.filter_psi(lt, r, a), mu, assign)


def test_coefficient_gradient_matches_central_differences():
    n, rp, ci, w, r, a, mu, asg = _case()
    loss, ga, _ = gr.loss_and_grads(n, rp, ci, w, r, a, mu, asg)
    assert loss == pytest.approx(_loss(n, rp, ci, w, r, a, mu, asg), rel=1e-14)
    h = 1e-6
    for j in range(a.size):
        e = np.zeros_like(a)
        e[j] = h
        fd = (_loss(n, rp, ci, w, r, a + e, mu, asg) - _loss(n, rp, ci, w, r, a - e, mu, asg)) / (2 * h)
        assert ga[j] == pytest.approx(fd, rel=1e-6, abs=1e-8), j


def test_edge_weight_gradient_matches_central_differences():
    n, rp, ci, w, r, a, mu, asg = _case()
    _, _, gw = gr.loss_and_grads(n, rp, ci, w, r, a, mu, asg)
    rows = np.repeat(np.arange(n), np.diff(rp))
    h = 1e-6
    checked = 0
    for e in range(ci.size):
        u, v = rows[e], ci[e]
        if u > v:
            continue
        both = (rows == u) & (ci == v) | (rows == v) & (ci == u)
        wp, wm = w.copy(), w.copy()
        wp[both] += h
        wm[both] -= h
        fd = (_loss(n, rp, ci, wp, r, a, mu, asg) - _loss(n, rp, ci, wm, r, a, mu, asg)) / (2 * h)
        assert gw[e] == pytest.approx(fd, rel=1e-5, abs=1e-8), (u, v)
        # both stored copies of the edge carry the same gradient
        np.testing.assert_allclose(gw[both], gw[e], rtol=1e-12)
        checked += 1
    assert checked > 50


def test_weight_gradient_is_orthogonal_to_the_weights():
    """L~ = -D^{-1/2} W D^{-1/2} is unchanged when every weight is scaled, so the loss is
    homogeneous of degree 0 in w: sum_e w_e dloss/dw_e = 0 (each edge stored twice)."""
    n, rp, ci, w, r, a, mu, asg = _case(seed=8)
    _, _, gw = gr.loss_and_grads(n, rp, ci, w, r, a, mu, asg)
    assert abs(float(np.sum(w * gw))) < 1e-10 * float(np.sum(np.abs(w * gw)))


def test_coefficient_gradient_of_a_linear_combination():
    """The features are linear in a: with the loss replaced by <G, Psi> for a fixed G the
    coefficient gradient is (<G, T_j R>)_j, the same vector filter_vjp returns for gbar = G;
    and Psi(a) scaled by c equals Psi(c a)."""
    n, rp, ci, w, r, a, _, _ = _case(seed=5)
    lt = lp.shifted_laplacian(n, rp, ci, w)
    g = np.random.default_rng(1).standard_normal(r.shape)
    ga, _ = gr.filter_vjp(lt, r, a, g)
    for j in range(a.size):
        e = np.zeros_like(a)
        e[j] = 1.0
        assert ga[j] == pytest.approx(float(np.sum(g * gr.filter_psi(lt, r, e))), rel=1e-12)
    np.testing.assert_allclose(gr.filter_psi(lt, r, 2.5 * a), 2.5 * gr.filter_psi(lt, r, a), rtol=1e-12)
