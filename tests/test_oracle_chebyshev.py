"""Pins of the oracle's Chebyshev filter, moments, eigencount and dichotomy (CPU only).

Each check ties the oracle to something other than itself: closed forms,
numerical quadrature, dense eigendecomposition, algebraic identities and
hand-derived values in tests/golden/.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from conftest import graph_from_edges, read_golden
from oracle import chebyshev as cb
from oracle import laplacian as lp
from oracle import spectral as sp_


def test_scalar_recursion_is_cos_j_theta():
    # T_j(cos t) = cos(j t): the response of the unit coefficient vector e_j at lambda = 1 + cos t
    t = np.linspace(0.0, math.pi, 97)
    lam = 1.0 + np.cos(t)
    for j in range(0, 40):
        a = np.zeros(j + 1)
        a[j] = 1.0
        np.testing.assert_allclose(cb.response(a, lam), np.cos(j * t), atol=1e-12)


def test_step_coefficients_equal_projection_integral():
    # c_j = (2/pi) int_0^pi 1[cos t <= x_c] cos(j t) dt, halved for j = 0
    for lam_c in (0.13, 0.5, 1.0, 1.37, 1.9):
        x_c = lam_c - 1.0
        c = cb.step_coefficients(12, lam_c)
        for j in range(13):
            val, _ = integrate.quad(lambda t: float(np.cos(t) <= x_c) * math.cos(j * t),
                                    0.0, math.pi, points=[math.acos(x_c)], limit=200)
            ref = (2.0 / math.pi) * val * (0.5 if j == 0 else 1.0)
            assert abs(c[j] - ref) < 1e-9, (lam_c, j, c[j], ref)


def test_golden_jackson_and_step_values():
    for row in read_golden("jackson_small.txt"):
        kind, key, vals = row[0], float(row[1]), np.array([float(v) for v in row[2:]])
        if kind == "jackson":
            np.testing.assert_allclose(cb.jackson(int(key)), vals, atol=1e-15)
        else:
            np.testing.assert_allclose(cb.step_coefficients(vals.size - 1, key), vals, atol=1e-15)


@pytest.mark.parametrize("m", [1, 5, 20, 50, 100])
def test_jackson_kernel_positive(m):
    g = cb.jackson(m)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert np.all(np.diff(g) < 0) and g[-1] > 0
    theta = np.linspace(0, math.pi, 4001)
    kern = 1.0 + 2.0 * np.sum(g[1:, None] * np.cos(np.arange(1, m + 1)[:, None] * theta[None]), axis=0)
    assert kern.min() > -1e-10


@pytest.mark.parametrize("m", [10, 50, 100])
def test_damped_response_bounded_monotone(m):
    lam = np.linspace(0, 2, 2001)
    prev = None
    for lam_c in np.linspace(0.05, 1.95, 20):
        h = cb.response(cb.filter_coefficients(m, lam_c), lam)
        assert h.min() > -1e-12 and h.max() < 1 + 1e-12
        # positivity of the kernel makes h monotone in the cutoff (checked below); in lambda it
        # is monotone up to the kernel's ripple near the spectrum edges
        assert np.all(np.diff(h) < 2e-4)
        if prev is not None:
            assert np.all(h >= prev - 1e-12)       # non-decreasing in the cutoff
        prev = h
    # sharpens with m: far from the cutoff the response approaches the step
    h = cb.response(cb.filter_coefficients(m, 1.0), np.array([0.3, 1.7]))
    assert h[0] > 1 - 30.0 / m**2 and h[1] < 30.0 / m**2


def test_golden_spectra_closed_forms():
    for name, n, edges, *eig in read_golden("spectra_small.txt"):
        n = int(n)
        e = [tuple(int(x) for x in s.split("-")) for s in edges.split(",")]
        rp, ci = graph_from_edges(n, e)
        lap = lp.normalized_laplacian_dense(n, rp, ci)
        np.testing.assert_allclose(np.linalg.eigvalsh(lap), [float(x) for x in eig], atol=1e-12,
                                   err_msg=name)


def _small_graph():
    g = W.sbm_graph(300, 4, 12, 8, seed=11)
    return g, lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)


def test_filter_on_eigenvectors_returns_h_of_lambda():
    g, lt = _small_graph()
    lam, u = sp_.eig(lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx))
    m, lam_c = 40, 0.6
    a = cb.filter_coefficients(m, lam_c)
    out = cb.cheb_filter(lt, u[:, :12], m, lam_c)
    np.testing.assert_allclose(out, u[:, :12] * cb.response(a, lam[:12])[None, :], atol=1e-11)


def test_filter_equals_dense_spectral_response():
    g, lt = _small_graph()
    lap = lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(g.n, 8, 8, seed=3).astype(np.float64)
    for m, lam_c in ((7, 0.4), (50, 0.9), (100, 1.5)):
        a = cb.filter_coefficients(m, lam_c)
        ref = sp_.apply_response(lap, lambda x: cb.response(a, x), r)
        np.testing.assert_allclose(cb.cheb_filter(lt, r, m, lam_c), ref, atol=1e-11)


def test_cycle_graph_closed_form():
    # C_n: L~ = -W/2, Fourier modes cos(2 pi l v / n) with L eigenvalue 1 - cos(2 pi l / n)
    n = 64
    rp, ci = graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    lt = lp.shifted_laplacian(n, rp, ci)
    v = np.arange(n)
    m, lam_c = 30, 0.7
    a = cb.filter_coefficients(m, lam_c)
    for ell in (0, 1, 5, 16, 32):
        x = np.cos(2 * math.pi * ell * v / n)[:, None]
        lam = 1.0 - math.cos(2 * math.pi * ell / n)
        expect = cb.response(a, np.array([lam]))[0] * x
        np.testing.assert_allclose(cb.cheb_filter(lt, x, m, lam_c), expect, atol=1e-12)


def test_complete_graph_closed_form():
    # K_n: L eigenvalues 0 (vector D^1/2 1, constant here) and n/(n-1) (any vector orthogonal to it)
    n = 9
    rp, ci = graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    lt = lp.shifted_laplacian(n, rp, ci)
    m, lam_c = 25, 1.05
    a = cb.filter_coefficients(m, lam_c)
    const = np.ones((n, 1))
    orth = np.zeros((n, 1))
    orth[0], orth[1] = 1.0, -1.0
    h0, h1 = cb.response(a, np.array([0.0, n / (n - 1.0)]))
    np.testing.assert_allclose(cb.cheb_filter(lt, const, m, lam_c), h0 * const, atol=1e-12)
    np.testing.assert_allclose(cb.cheb_filter(lt, orth, m, lam_c), h1 * orth, atol=1e-12)


def test_isolated_node_row_is_zero():
    g = W.random_csr(200, 6, seed=5, isolated=7)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    iso = np.flatnonzero(np.diff(g.row_ptr) == 0)
    assert iso.size >= 7
    r = W.gaussian_block(g.n, 3, 3, seed=1).astype(np.float64)
    out = lt @ r
    assert np.all(out[iso] == 0.0)
    # T_j of an isolated node: T_0 = r, T_1 = 0, T_2 = -r, ... (eigenvalue 1 of L, x = 0)
    basis = cb.cheb_basis(lt, r, 4)
    np.testing.assert_array_equal(basis[2][iso], -r[iso])


def test_moment_identity():
    # T_i T_j = (T_{i+j} + T_{|i-j|}) / 2  =>  ||sum a_j T_j R||^2 = sum a_i a_j (mu_{i+j} + mu_{|i-j|}) / 2
    g, lt = _small_graph()
    r = W.gaussian_block(g.n, 6, 6, seed=9).astype(np.float64)
    m = 30
    mu = cb.moments(lt, r, 2 * m)
    basis = cb.cheb_basis(lt, r, m)
    for lam_c in (0.3, 0.8, 1.4):
        a = cb.filter_coefficients(m, lam_c)
        direct = float(np.sum(cb.combine(basis, a) ** 2))
        i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
        via = float(np.sum(a[i] * a[j] * (mu[i + j] + mu[np.abs(i - j)]) / 2.0))
        assert via == pytest.approx(direct, rel=1e-10)
    # the per-step quantities the GPU reduces map onto the moments
    for s in range(1, m + 1):
        e_s = float(np.sum(basis[s] * basis[s]))
        f_s = float(np.sum(basis[s] * basis[s - 1]))
        assert 2 * e_s - mu[0] == pytest.approx(mu[2 * s], rel=1e-9, abs=1e-9 * mu[0])
        assert 2 * f_s - mu[1] == pytest.approx(mu[2 * s - 1], rel=1e-9, abs=1e-9 * mu[0])


def test_eigencount_is_unbiased_for_trace_h_squared():
    g, lt = _small_graph()
    lam = np.linalg.eigvalsh(lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx))
    m, lam_c, d = 40, 0.55, 16
    a = cb.filter_coefficients(m, lam_c)
    target = float(np.sum(cb.response(a, lam) ** 2))
    counts = []
    for seed in range(60):
        r = W.gaussian_block(g.n, d, d, seed=1000 + seed).astype(np.float64)
        counts.append(cb.eigencount(cb.cheb_filter(lt, r, m, lam_c), d))
    counts = np.array(counts)
    sem = counts.std(ddof=1) / math.sqrt(counts.size)
    assert abs(counts.mean() - target) < 4 * sem + 1e-9


def test_trace_count_is_unbiased_for_trace_h():
    """The alternative (Hutchinson) estimator (d/c) tr(R^T h(L) R) has mean tr h(L)."""
    g, lt = _small_graph()
    lam = np.linalg.eigvalsh(lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx))
    m, lam_c, d = 40, 0.55, 16
    a = cb.filter_coefficients(m, lam_c)
    target = float(np.sum(cb.response(a, lam)))
    counts = []
    for seed in range(60):
        r = W.gaussian_block(g.n, d, d, seed=2000 + seed).astype(np.float64)
        counts.append(cb.trace_count(r, cb.cheb_filter(lt, r, m, lam_c), d))
    counts = np.array(counts)
    sem = counts.std(ddof=1) / math.sqrt(counts.size)
    assert abs(counts.mean() - target) < 4 * sem + 1e-9
    # the two estimators target different traces: tr h(L) > tr h(L)^2 when 0 < h < 1 somewhere
    assert target > float(np.sum(cb.response(a, lam) ** 2))


def test_count_tolerance_is_twice_the_ideal_projector_spread():
    """tau = max(0.5, 2 sqrt(2k/c)) is twice the spread of the count under the ideal low pass.
    With Psi = U_k U_k^T R (Eq. 3's projector on a graph's k lowest eigenvectors) and c signals
    of variance 1/d, (d/c) ||Psi||_F^2 is chi-square with kc degrees of freedom over c: mean k and
    standard deviation sqrt(2k/c).  Both are measured here over 3000 seeds with the oracle's
    eigencount, and the oracle's tolerance must equal max(0.5, twice the measured spread)."""
    g = W.sbm_graph(120, 4, 12, 10, seed=3)
    lap = lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx)
    hk = sp_.ideal_projector(lap, 10)
    rng = np.random.default_rng(8)
    for k, c, d in ((10, 8, 64), (4, 32, 48), (10, 128, 256)):
        proj = hk if k == 10 else sp_.ideal_projector(lap, k)
        counts = np.array([cb.eigencount(proj @ (rng.standard_normal((g.n, c)) / math.sqrt(d)), d)
                           for _ in range(3000)])
        sd = counts.std(ddof=1)
        assert abs(counts.mean() - k) < 4.0 * math.sqrt(2.0 * k / c) / math.sqrt(counts.size)
        assert abs(sd / math.sqrt(2.0 * k / c) - 1.0) < 0.06, (k, c, sd)
        tau = cb.count_tolerance(k, c)
        assert abs(tau - max(0.5, 2.0 * sd)) <= 0.06 * max(0.5, 2.0 * sd), (k, c, tau, sd)


def test_count_monotone_in_cutoff():
    g, lt = _small_graph()
    r = W.gaussian_block(g.n, 8, 8, seed=4).astype(np.float64)
    basis = cb.cheb_basis(lt, r, 50)
    cuts = np.linspace(0.0, 2.0, 41)
    cnt = [cb.eigencount(cb.combine(basis, cb.filter_coefficients(50, c)), 8) for c in cuts]
    assert np.all(np.diff(cnt) >= -1e-9)
    assert cnt[0] < 1.0 and cnt[-1] == pytest.approx(8.0 / 8.0 * np.sum(r**2) * 1.0, rel=1e-12)


def _exact_count(lam_eigs, m):
    return lambda c: float(np.sum(cb.response(cb.filter_coefficients(m, c), lam_eigs) ** 2))


def test_lambda_search_static_on_known_spectrum():
    g, _ = _small_graph()
    lam = np.linalg.eigvalsh(lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx))
    count = _exact_count(lam, 60)
    for k in (4, 10, 30):
        tau = cb.count_tolerance(k, 64)
        c, cnt, ev = cb.lambda_search(count, k, tau)
        assert abs(cnt - k) <= tau and cnt == pytest.approx(count(c))
        assert ev <= 30
        # bisection midpoints of [0, 2] are dyadic: c * 2^ev is an integer
        assert (c * 2**ev) == int(c * 2**ev)


def test_lambda_search_warm_start_paths():
    g, _ = _small_graph()
    lam = np.linalg.eigvalsh(lp.normalized_laplacian_dense(g.n, g.row_ptr, g.col_idx))
    count = _exact_count(lam, 60)
    k, tau = 10, 0.5
    c0, _, _ = cb.lambda_search(count, k, tau)
    # previous cutoff still valid: one evaluation, unchanged
    c, cnt, ev = cb.lambda_search(count, k, tau, lam_prev=c0)
    assert (c, ev) == (c0, 1)
    # previous cutoff too low / too high: bracket grows toward k, then bisects
    for start in (0.5 * c0, min(1.99, 1.6 * c0)):
        c, cnt, ev = cb.lambda_search(count, k, tau, lam_prev=start)
        assert abs(cnt - k) <= tau and ev <= 30


def test_lambda_search_step_cap():
    calls = []

    def never(c):
        calls.append(c)
        return 5.0 if c < 1.0 else 20.0     # jumps over k = 10: never accepted

    c, cnt, ev = cb.lambda_search(never, 10, 0.5, max_steps=12)
    assert ev == 12 == len(calls) and abs(c - 1.0) < 2.0**-10
