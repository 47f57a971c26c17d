"""The paper's theorems as checks on the oracle (CPU only).

Thm 3.3 is an exact equality; Cor 3.5 / Thm 3.1 / Thm 4.1 / Cor 4.2 are
probabilistic or deterministic bounds checked over seeds on small SBMs with
dense eigendecomposition.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import chebyshev as cb
from oracle import kmeans as km
from oracle import laplacian as lp
from oracle import spectral as sp_
from oracle.dynamic import DynamicCSC


def _sbm(n=400, k=4, deg=16, ratio=12, seed=21):
    g = W.sbm_graph(n, k, deg, ratio, seed)
    return g, lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx)


def test_thm33_equality_exact():
    g, lap = _sbm()
    k = 4
    phi = sp_.features(lap, k)
    for d in (4, 8, 32):
        r = W.gaussian_block(g.n, d, d, seed=d).astype(np.float64)
        psi = phi @ (phi.T @ r)                       # H_k R, Eq. 3
        lhs, rhs = sp_.thm33_gap(phi, psi, r)
        assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-12)


def test_cor35_feature_bound_over_seeds():
    # ||Psi - Phi I Q||_F <= sqrt(k/d)(sqrt(k) + t) with probability >= 1 - exp(-t^2/2)
    g, lap = _sbm()
    k, d, t = 4, 24, 1.5
    phi = sp_.features(lap, k)
    bound = math.sqrt(k / d) * (math.sqrt(k) + t)
    fails = 0
    trials = 200
    for s in range(trials):
        r = W.gaussian_block(g.n, d, d, seed=5000 + s).astype(np.float64)
        _, rhs = sp_.thm33_gap(phi, phi @ (phi.T @ r), r)
        fails += rhs > bound
    # allowed failure rate exp(-t^2/2) = 0.325; binomial 3-sigma slack
    p = math.exp(-t * t / 2)
    assert fails <= trials * p + 3 * math.sqrt(trials * p * (1 - p))


def test_thm31_cost_bound_with_chebyshev_features():
    # C_Psi <= C_Phi + 2 sqrt(k/d)(sqrt(k) + t), C_Phi taken as the best Lloyd cost over restarts
    g, lap = _sbm(n=600, k=5, deg=20, ratio=15, seed=3)
    k, d, t, m = 5, 40, 2.0, 60
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    lam = np.linalg.eigvalsh(lap)
    phi = sp_.features(lap, k)
    c_phi = min(km.cost(phi, km.lloyd(phi, km.forgy_centroids(phi, W.forgy_indices(g.n, k, s)))[0], k)
                for s in range(20))
    c_phi = min(c_phi, km.cost(phi, g.labels, k))
    bound = c_phi + 2 * math.sqrt(k / d) * (math.sqrt(k) + t)
    lam_c = 0.5 * (lam[k - 1] + lam[k])
    fails = 0
    for s in range(20):
        r = W.gaussian_block(g.n, d, d, seed=900 + s).astype(np.float64)
        psi = cb.cheb_filter(lt, r, m, lam_c)
        best = min(km.cost(phi, km.lloyd(psi, km.forgy_centroids(psi, W.forgy_indices(g.n, k, 77 * s + q)))[0], k)
                   for q in range(5))
        fails += best > bound
    assert fails <= 1


def test_cor42_subspace_perturbation_bound():
    # ||H_t - H_{t-1}||_F <= sqrt(2)/alpha ||L_t - L_{t-1}||_F, alpha = min(lam_k^t, lam_{k+1}^{t-1} - lam_k^t)
    g, lap0 = _sbm(n=300, k=3, deg=20, ratio=20, seed=8)
    k = 3
    g1 = W.edge_redraw(g, 0.02, seed=9)
    lap1 = lp.normalized_laplacian_dense(g1.n, g1.row_ptr, g1.col_idx)
    l0 = np.linalg.eigvalsh(lap0)
    l1 = np.linalg.eigvalsh(lap1)
    alpha = min(l1[k - 1], l0[k] - l1[k - 1])
    assert alpha > 0
    lhs = np.linalg.norm(sp_.ideal_projector(lap1, k) - sp_.ideal_projector(lap0, k))
    rhs = math.sqrt(2) / alpha * np.linalg.norm(lap1 - lap0)
    assert lhs <= rhs


def test_thm41_dynamic_features_reuse_error_term():
    # ||(Psi_t - Psi_{t-1}) S_dp||_F^2 <= p (1+delta) ||H_t - H_{t-1}||_F^2 (proof of Thm 4.1), delta = 1
    g, lap0 = _sbm(n=300, k=3, deg=20, ratio=20, seed=8)
    g1 = W.edge_redraw(g, 0.05, seed=10)
    lap1 = lp.normalized_laplacian_dense(g1.n, g1.row_ptr, g1.col_idx)
    k, d, p = 3, 40, 0.5
    h0, h1 = sp_.ideal_projector(lap0, k), sp_.ideal_projector(lap1, k)
    gamma2 = np.linalg.norm(h1 - h0) ** 2
    dp = int(p * d)
    fails = 0
    for s in range(50):
        r = W.gaussian_block(g.n, d, d, seed=300 + s).astype(np.float64)
        lhs = np.linalg.norm((h1 - h0) @ r[:, :dp]) ** 2
        fails += lhs > p * 2.0 * gamma2
    assert fails <= 2


def test_dynamic_p0_equals_static_each_step():
    g = W.sbm_graph(300, 3, 14, 10, seed=2)
    dyn = DynamicCSC(300, 3, 12, 0.0, 20, seed=4)
    graphs = [g, W.edge_redraw(g, 0.02, 1)]
    for t, gg in enumerate(graphs):
        idx = W.forgy_indices(300, 3, seed=t)
        dyn.step(gg.row_ptr, gg.col_idx, init_idx=idx)
        # static CSC on the same columns: fresh ids d*t .. d*t+d-1
        from oracle.philox import gaussian_columns
        r = gaussian_columns(4, 300, np.arange(12 * t, 12 * t + 12), 12)
        lt = lp.shifted_laplacian(300, gg.row_ptr, gg.col_idx)
        np.testing.assert_allclose(dyn.features(), cb.cheb_filter(lt, r, 20, dyn.lam), atol=1e-13)


def test_dynamic_zero_churn_keeps_reused_columns_bitwise():
    g = W.sbm_graph(300, 3, 14, 10, seed=2)
    dyn = DynamicCSC(300, 3, 16, 0.75, 20, seed=4)
    dyn.step(g.row_ptr, g.col_idx, init_idx=W.forgy_indices(300, 3, 0))
    before = dyn.features()
    dyn.step(g.row_ptr, g.col_idx, init_idx=W.forgy_indices(300, 3, 1))
    slots = dyn.history[-1]["slots"]
    np.testing.assert_array_equal(slots, np.arange(4))       # FIFO: oldest, lowest slot first
    kept = np.setdiff1d(np.arange(16), slots)
    np.testing.assert_array_equal(dyn.features()[:, kept], before[:, kept])
    dyn.step(g.row_ptr, g.col_idx, init_idx=W.forgy_indices(300, 3, 2))
    np.testing.assert_array_equal(dyn.history[-1]["slots"], np.arange(4, 8))
