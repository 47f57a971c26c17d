"""Pins of the compressive k-means oracle (oracle/compressive.py).

Each reading is checked against something other than its own formula: the law of the draws
against the weights by a chi-square test, the sampling density against exact leverage scores
from a dense eigendecomposition, the interpolation against the ideal-projector interpolation
of a graph with a wide spectral gap, and the whole step against a planted partition.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.optimize import linear_sum_assignment

import workloads as W
from oracle import chebyshev as cb
from oracle import compressive as ck
from oracle import laplacian as lp
from oracle import philox as px


def _agreement(a, b, k):
    c = np.zeros((k, k))
    np.add.at(c, (a, b), 1)
    r, cc = linear_sum_assignment(-c)
    return c[r, cc].sum() / a.size


def test_draw_law_matches_the_weights():
    theta = np.array([[1.0, 0.0], [0.5, 0.5], [0.0, 0.0], [2.0, 1.0], [0.1, 0.2], [0.0, 3.0], [1.0, 1.0]],
                     dtype=np.float32)
    q, _ = ck.quantise(ck.row_energy(theta))
    prefix = np.cumsum(q)
    drawn = ck.draw_nodes(12345, 40000, prefix)
    assert drawn.min() >= 0 and drawn.max() < theta.shape[0]
    assert not np.any(drawn == 2), "a zero-weight node was drawn"
    counts = np.bincount(drawn, minlength=theta.shape[0])
    nz = q > 0
    expected = q[nz] / q.sum() * drawn.size
    assert stats.chisquare(counts[nz], expected).pvalue > 1e-4
    # seeded: the same seed gives the same draws, another seed other draws
    np.testing.assert_array_equal(drawn[:100], ck.draw_nodes(12345, 100, prefix))
    assert not np.array_equal(drawn[:100], ck.draw_nodes(12346, 100, prefix))


def test_draws_follow_the_inverse_distribution_by_brute_force():
    """Each drawn node is the smallest i whose prefix sum exceeds the draw position; nodes
    with zero weight (equal consecutive prefix sums) are never hit, also at the boundaries."""
    q = np.array([0, 3, 0, 0, 2, 5, 0, 1], dtype=np.int64)
    prefix = np.cumsum(q)
    total = int(prefix[-1])
    us = ck.draw_positions(77, 3000, total)
    nodes = ck.draw_nodes(77, 3000, prefix)
    assert min(us) >= 0 and max(us) < total
    for u, node in zip(us, nodes):
        brute = next(i for i in range(q.size) if prefix[i] > u)
        assert node == brute
    assert set(np.unique(nodes)) == {1, 4, 5, 7}
    # every position is reachable: position u maps to node brute(u) for all u < T
    assert sorted(set(us)) == list(range(total))


def test_uniform_energies_give_unit_weights():
    """Rows of equal energy: uniform sampling, so every weight T / (n q_i) is exactly 1."""
    theta = np.tile(np.array([[0.5, -1.0, 2.0]], dtype=np.float32), (37, 1))
    omega, q, total = ck.sample(theta, 20, 3)
    assert np.all(q == q[0]) and total == q.size * int(q[0])
    np.testing.assert_array_equal(ck.sample_weights(q, total, omega), np.ones(omega.size))


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1.0, 1e6, 1e30])
def test_quantisation_is_exact_and_fine(scale):
    rng = np.random.default_rng(4)
    s = rng.random(1000) ** 3 * scale
    s[7] = 0.0
    q, e = ck.quantise(s)
    # q_i = floor(s_i 2^E): q_i <= s_i 2^E < q_i + 1, compared exactly in integers
    for i in range(0, 1000, 37):
        num, den = float(s[i]).as_integer_ratio()
        lhs = num * 2 ** e if e >= 0 else num
        rhs_den = den if e >= 0 else den * 2 ** (-e)
        qi = int(q[i])
        assert qi * rhs_den <= lhs < (qi + 1) * rhs_den
    assert int(q.sum()) < 2 ** 62
    # resolution: the largest weight has at least 61 - ceil(log2 n) bits
    assert int(q.max()) >= 2 ** (61 - 10)
    assert q[7] == 0
    with pytest.raises(ValueError):
        ck.quantise(np.zeros(5))


def test_density_estimates_leverage_scores():
    """Under the ideal projector U_k U_k^T, E ||theta_i||^2 = ||U_k^T delta_i||^2 (the local
    cumulative coherence); with d = 4000 signals the relative spread is sqrt(2/d) ~ 2%."""
    n, k, d = 240, 4, 4000
    g = W.sbm_graph(n, W.zipf_block_sizes(n, k, 1.2), 12, 20, seed=2)
    lap = lp.normalized_laplacian_dense(n, g.row_ptr, g.col_idx)
    _, u = np.linalg.eigh(lap)
    uk = u[:, :k]
    lev = np.sum(uk * uk, axis=1)
    r = px.gaussian_columns(9, n, np.arange(d), d)
    theta = (uk @ (uk.T @ r)).astype(np.float32)
    s = ck.row_energy(theta)
    rel = np.abs(s - lev) / lev
    assert np.mean(rel) < 0.04 and np.max(rel) < 0.15
    # the density is not uniform: the smallest block is sampled more per node
    sizes = np.bincount(g.labels)
    small, large = np.argmin(sizes), np.argmax(sizes)
    assert np.mean(lev[g.labels == small]) > 1.5 * np.mean(lev[g.labels == large])


def test_interpolation_is_the_low_pass_projection():
    """With a wide spectral gap around the cutoff, h(L) z is the projection U_k U_k^T z
    up to the Jackson transition width."""
    n, k = 400, 4
    g = W.sbm_graph(n, k, 20, 80, seed=6)
    lap = lp.normalized_laplacian_dense(n, g.row_ptr, g.col_idx)
    lam, u = np.linalg.eigh(lap)
    assert lam[k] - lam[k - 1] > 0.3
    lam_c = 0.5 * (lam[k - 1] + lam[k])
    rng = np.random.default_rng(3)
    z = np.zeros((n, k))
    omega = rng.choice(n, 30, replace=False)
    z[omega, rng.integers(0, k, 30)] = rng.uniform(0.5, 2.0, 30)
    x = ck.interpolate(n, g.row_ptr, g.col_idx, None, z, 300, lam_c)
    proj = u[:, :k] @ (u[:, :k].T @ z)
    assert np.linalg.norm(x - proj) < 0.02 * np.linalg.norm(z)


def test_assignment_takes_the_lowest_maximiser():
    x = np.array([[0.0, 1.0, 1.0], [2.0, 2.0, 0.0], [0.0, 0.0, 0.0], [-1.0, -3.0, -1.0]])
    np.testing.assert_array_equal(ck.argmax_assign(x), [1, 0, 0, 0])


def test_recovers_a_planted_partition():
    n, k, d, m = 2000, 5, 40, 80
    g = W.sbm_graph(n, k, 30, 40, seed=11)
    lt = lp.shifted_laplacian(n, g.row_ptr, g.col_idx)
    lam = np.linalg.eigvalsh(lt.toarray()) + 1.0
    lam_c = 0.5 * (lam[k - 1] + lam[k])
    theta = cb.cheb_filter(lt, px.gaussian_columns(21, n, np.arange(d), d), m, lam_c).astype(np.float32)
    y = theta / np.linalg.norm(theta, axis=1, keepdims=True)
    n_draws = int(np.ceil(4 * k * np.log(k)))
    res = ck.compressive_kmeans(n, g.row_ptr, g.col_idx, None, theta, y, k, n_draws, m, lam_c, seed=8)
    om = res["omega"]
    assert np.all(np.diff(om) > 0) and om.size <= n_draws
    assert res["labels"].min() >= 0 and res["labels"].max() < k
    assert np.all(res["weights"] > 0)
    assert _agreement(res["assign"], g.labels, k) > 0.95
