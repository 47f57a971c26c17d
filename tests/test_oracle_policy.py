"""Pins of the edge-similarity policy of oracle/dynamic.py (Definition 4.1, Theorem 4.1 with
Corollary 4.2, Section 4.1): its special cases, the bound it guarantees, and the two facts it
rests on, checked by dense eigendecomposition."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import laplacian as lp
from oracle import similarity as sm
from oracle import spectral as sp_
from oracle.dynamic import DynamicCSC, reuse_policy


def test_special_cases():
    # no change: keep p_max, skip the check (nothing moved)
    assert reuse_policy(64, 0.75, 0.0, 0.1, 0.2, 0.0, 0.0) == (48, False, 0.0)
    # no budget: keep p_max whatever rho; rho_skip 0 -> check
    assert reuse_policy(64, 0.75, 5.0, 0.1, 0.0, 0.0, 0.0) == (48, True, 0.0)
    # a large change refreshes every column
    dp, check, acc = reuse_policy(64, 0.75, 50.0, 0.1, 0.2, 0.0, 0.0)
    assert dp == 0 and check and acc == 0.0
    # the summed rho skips the check until it exceeds rho_skip
    assert reuse_policy(10, 0.5, 0.3, 1.0, 0.0, 1.0, 0.5) == (5, False, pytest.approx(0.8))
    assert reuse_policy(10, 0.5, 0.3, 1.0, 0.0, 1.0, 0.8)[1:] == (True, 0.0)


@pytest.mark.parametrize("rho", [0.05, 0.3, 1.0, 3.0])
def test_reuse_fraction_meets_the_budget_and_is_the_largest(rho):
    """2 sqrt(2 p) gamma <= eps with gamma = sqrt(2) rho / alpha, and one more reused column would
    break it (unless p_max binds)."""
    d, p_max, alpha, eps = 128, 0.9, 0.2, 0.5
    dp, _, _ = reuse_policy(d, p_max, rho, alpha, eps, 0.0, 0.0)
    gamma = math.sqrt(2.0) * rho / alpha
    assert 2.0 * math.sqrt(2.0 * dp / d) * gamma <= eps * (1 + 1e-12)
    if dp < math.floor(p_max * d):
        assert 2.0 * math.sqrt(2.0 * (dp + 1) / d) * gamma > eps


def test_reused_columns_error_expectation():
    """The step of Theorem 4.1's proof that the policy relies on: for R with i.i.d. N(0, 1/d)
    entries and the dp reused columns, E ||(H_t - H_{t-1}) R_dp||_F^2 = (dp/d) ||H_t - H_{t-1}||_F^2
    (checked over 4000 draws on a perturbed SBM pair, dense projectors)."""
    g0 = W.sbm_graph(150, 3, 10, 10, seed=7)
    g1 = W.sbm_perturb(g0, 0.02, 0.05, seed=8)
    l0 = lp.normalized_laplacian_dense(g0.n, g0.row_ptr, g0.col_idx)
    l1 = lp.normalized_laplacian_dense(g1.n, g1.row_ptr, g1.col_idx)
    dh = sp_.ideal_projector(l1, 3) - sp_.ideal_projector(l0, 3)
    d, dp = 40, 10
    rng = np.random.default_rng(1)
    vals = np.array([np.sum((dh @ (rng.standard_normal((g0.n, dp)) / math.sqrt(d))) ** 2)
                     for _ in range(4000)])
    want = dp / d * np.sum(dh * dh)
    assert abs(vals.mean() - want) < 4.0 * vals.std() / math.sqrt(vals.size)


def test_weyl_bound_behind_the_check_skip():
    """Eigenvalues of L move by at most the summed edge distance over a perturbed sequence."""
    g = [W.sbm_graph(200, 4, 12, 10, seed=3)]
    for t in range(1, 5):
        g.append(W.sbm_perturb(g[-1], 0.01, 0.03, seed=50 + t))
    ev = [np.linalg.eigvalsh(lp.normalized_laplacian_dense(x.n, x.row_ptr, x.col_idx)) for x in g]
    rho = [sm.laplacian_distance(200, (g[t - 1].row_ptr, g[t - 1].col_idx, None),
                                 (g[t].row_ptr, g[t].col_idx, None)) for t in range(1, 5)]
    for s in range(5):
        for t in range(s + 1, 5):
            assert np.max(np.abs(ev[t] - ev[s])) <= sum(rho[s:t]) + 1e-12


def test_dynamic_oracle_under_the_policy():
    """A skipped check keeps the cutoff with no evaluation; a budget that forces dp = 0 refilters
    every column at every snapshot (the static scheme)."""
    n, k, d, m = 300, 3, 24, 20
    g = [W.sbm_graph(n, k, 12, 10, seed=4)]
    for t in range(1, 4):
        g.append(W.sbm_perturb(g[-1], 0.01, 0.03, seed=60 + t))
    rho = [0.0] + [sm.laplacian_distance(n, (g[t - 1].row_ptr, g[t - 1].col_idx, None),
                                         (g[t].row_ptr, g[t].col_idx, None)) for t in range(1, 4)]
    skip = DynamicCSC(n, k, d, 0.5, m, seed=9)
    for t in range(4):
        skip.step(g[t].row_ptr, g[t].col_idx, init_idx=W.forgy_indices(n, k, t), rho=rho[t],
                  policy=dict(alpha=0.1, budget=0.0, rho_skip=1e9))
    assert all(not h["checked"] and h["evals"] == 0 and h["lam"] == skip.history[0]["lam"]
               for h in skip.history[1:])
    assert all(h["c"] == 12 for h in skip.history[1:])
    full = DynamicCSC(n, k, d, 0.5, m, seed=9)
    static = DynamicCSC(n, k, d, 0.0, m, seed=9)
    for t in range(4):
        idx = W.forgy_indices(n, k, t)
        full.step(g[t].row_ptr, g[t].col_idx, init_idx=idx, rho=rho[t],
                  policy=dict(alpha=0.01, budget=1e-6, rho_skip=0.0))
        static.step(g[t].row_ptr, g[t].col_idx, init_idx=idx)
    for a, b in zip(full.history, static.history):
        assert a["c"] == d and a["lam"] == b["lam"] and a["evals"] == b["evals"]
    np.testing.assert_array_equal(full.features(), static.features())
