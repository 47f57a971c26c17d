"""The C-ABI library on the CPU: it builds, loads, exports every symbol of
include/csc.h, and its host-only helpers (no GPU work) agree with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import workloads as W
from conftest import ROOT
from oracle import chebyshev as cb
from oracle import laplacian as lp


@pytest.fixture(scope="module")
def lib():
    from paper_1706_03591_gb300 import build
    build.build()
    import paper_1706_03591_gb300 as csc
    return csc


def _declared():
    text = open(os.path.join(ROOT, "include", "csc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csc_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    from paper_1706_03591_gb300 import _abi
    so = ctypes.CDLL(_abi.LIB_PATH)
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # the binding declares exactly the header's entry points
    assert sorted(_abi.SIGNATURES) == names
    assert lib.csc_abi_version() == 9


def test_missing_library_fails_loudly(tmp_path):
    from paper_1706_03591_gb300 import _abi
    with pytest.raises(RuntimeError, match="not found"):
        _abi.load(str(tmp_path / "libcsc.so"))


def test_coefficients_match_oracle(lib):
    for m in (1, 2, 10, 50, 100):
        for lam in (0.0, 0.17, 0.5, 1.0, 1.33, 2.0, 2.5, -0.3):
            a = lib.csc_filter_coeffs(m, lam)
            ref = cb.filter_coefficients(m, min(2.0, max(0.0, lam)))
            np.testing.assert_allclose(a, ref, rtol=0, atol=1e-15)


def test_tolerance_matches_oracle(lib):
    for k, c in ((10, 64), (10, 32), (100, 64), (1, 1000), (64, 39)):
        assert lib.csc_count_tolerance(k, c) == cb.count_tolerance(k, c)


def _moments_case(seed=3, n=400, c=12, d=24, m=40):
    g = W.sbm_graph(n, 5, 14, 10, seed=seed)
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
    r = W.gaussian_block(n, c, d, seed=seed + 1).astype(np.float64)
    return lt, r, cb.moments(lt, r, 2 * m), cb.cheb_basis(lt, r, m), d, c, m


def test_count_from_moments_equals_direct_eigencount(lib):
    lt, r, mu, basis, d, c, m = _moments_case()
    for lam in (0.2, 0.55, 0.9, 1.5):
        direct = cb.eigencount(cb.combine(basis, cb.filter_coefficients(m, lam)), d)
        assert lib.csc_count_from_moments(m, mu, lam, d, c) == pytest.approx(direct, rel=1e-9)


def test_trace_count_from_moments_equals_direct_trace_count(lib):
    lt, r, mu, basis, d, c, m = _moments_case()
    for lam in (0.2, 0.55, 0.9, 1.5):
        direct = cb.trace_count(r, cb.combine(basis, cb.filter_coefficients(m, lam)), d)
        assert lib.csc_trace_count_from_moments(m, mu, lam, d, c) == pytest.approx(direct, rel=1e-9)


def test_lambda_search_matches_oracle_control_flow(lib):
    lt, r, mu, basis, d, c, m = _moments_case()

    def direct(lam):
        return cb.eigencount(cb.combine(basis, cb.filter_coefficients(m, lam)), d)

    for k in (3, 5, 8, 15):
        tau = cb.count_tolerance(k, c)
        for prev in (None, 0.05, 0.4, 1.2, 1.95):
            ref = cb.lambda_search(direct, k, tau, prev, 30)
            got = lib.csc_lambda_search_moments(m, mu, d, c, k, tau, -1.0 if prev is None else prev, 30)
            # same decisions -> the same cutoff bit for bit unless a count sits on a threshold
            assert got[2] == ref[2], (k, prev, got, ref)
            assert got[0] == ref[0], (k, prev, got, ref)
            assert got[1] == pytest.approx(ref[1], rel=1e-9)


def test_lambda_search_cap_and_bad_args(lib):
    m = 4
    mu = np.zeros(2 * m + 1)
    lam, cnt, ev = lib.csc_lambda_search_moments(m, mu, 8, 8, 3, 0.5, -1.0, 7)
    assert ev == 7 and cnt == 0.0 and lam == 2.0 - 2.0**-6
    with pytest.raises(lib.CscError):
        lib.csc_lambda_search_moments(m, mu, 8, 8, 0, 0.5, -1.0, 7)
    with pytest.raises(lib.CscError):
        lib.csc_filter_coeffs(-1, 0.5)


def test_binding_rejects_wrong_element_types():
    """Array arguments are passed as raw pointers, so the binding checks their element types
    before any call: a float64 feature block or an int64 assignment buffer is refused."""
    import paper_1706_03591_gb300 as csc
    with pytest.raises(TypeError, match="theta"):
        csc._arr(np.zeros((4, 3)), "theta")
    with pytest.raises(TypeError, match="assign_out"):
        csc._arr(np.zeros(4, dtype=np.int64), "assign_out")
    with pytest.raises(TypeError, match="col_idx"):
        csc._arr(np.zeros(4, dtype=np.int64), "col_idx")
    ptr, where, code, ld = csc._arr(np.zeros((4, 3), dtype=np.float32), "Y")
    assert where == csc.CSC_HOST and code == csc.CSC_F32 and ld == 3
    torch = pytest.importorskip("torch")
    _, _, code, _ = csc._arr(torch.zeros((4, 3), dtype=torch.bfloat16), "Y")
    assert code == csc.CSC_BF16
    with pytest.raises(TypeError, match="psi_out"):
        csc._arr(torch.zeros((4, 3), dtype=torch.bfloat16), "psi_out")


def test_similarity_policy_matches_oracle(lib):
    """csc_reuse_policy makes the decision of oracle.dynamic.reuse_policy, bit for bit."""
    from oracle.dynamic import reuse_policy
    rng = np.random.default_rng(3)
    for _ in range(500):
        d = int(rng.integers(1, 300))
        p_max = float(rng.uniform(0, 0.99))
        rho = float(rng.choice([0.0, rng.exponential(2.0)]))
        alpha = float(rng.uniform(0.01, 0.5))
        budget = float(rng.choice([0.0, rng.uniform(0.1, 200.0)]))
        rho_skip = float(rng.choice([0.0, rng.uniform(0, 5)]))
        since = float(rng.uniform(0, 3))
        assert lib.csc_reuse_policy(d, p_max, rho, alpha, budget, rho_skip, since) == \
            reuse_policy(d, p_max, rho, alpha, budget, rho_skip, since)
    with pytest.raises(lib.CscError):
        lib.csc_reuse_policy(10, 0.5, 1.0, 0.0, 1.0, 0.0)  # alpha must be positive with a budget


def test_tile_plan_minimises_its_cost_model():
    """The column tiles of a pass (csc_tile_plan): widths in {8, 16, 32, 64}, widest first,
    covering c, with the least sum (8 + w); against exhaustive search over tile counts."""
    import paper_1706_03591_gb300 as csc

    def best(c):
        top = c // 8 + 2
        return min(8 * (a + b + e + f) + 64 * a + 32 * b + 16 * e + 8 * f
                   for a in range(top // 8 + 2) for b in range(3) for e in range(3) for f in range(3)
                   if 64 * a + 32 * b + 16 * e + 8 * f >= c)

    for c in range(1, 260):
        plan = csc.csc_tile_plan(c)
        assert plan == sorted(plan, reverse=True)
        assert set(plan) <= {8, 16, 32, 64}
        assert sum(plan) >= c and sum(plan) - min(plan) < c  # no tile is idle
        assert sum(8 + w for w in plan) == best(c), c
    assert csc.csc_tile_plan(39) == [32, 8]
    assert csc.csc_tile_plan(64) == [64]
    assert csc.csc_tile_plan(100) == [64, 32, 8]
    assert csc.csc_tile_plan(0) == []
    assert csc.csc_tile_plan(39, 16) == [16, 16, 16]
    assert csc.csc_tile_plan(130, 128) == [128, 128]
    with pytest.raises(ValueError):
        csc.csc_tile_plan(10, 12)


def test_step_launch_bytes():
    """Algorithmic bytes of a step launch: indices (and weights), offsets and D^-1/2 once, then
    per row and column V_{j-1} (s_prev bytes), V_j, V_{j+1} and Psi read and written."""
    import paper_1706_03591_gb300 as csc
    n, nnz = 8_000_000, 198_173_034
    assert csc.csc_step_launch_bytes(n, nnz, False, 32) == 4 * nnz + 8 * (n + 1) + 4 * n + n * 32 * 20
    assert csc.csc_step_launch_bytes(n, nnz, True, 8) == 8 * nnz + 8 * (n + 1) + 4 * n + n * 8 * 20
    assert csc.csc_step_launch_bytes(1000, 0, False, 64, 2) == 8 * 1001 + 4 * 1000 + 1000 * 64 * 18
