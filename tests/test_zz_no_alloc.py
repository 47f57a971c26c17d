"""The allocation-free filter entry point (csc_cheb_filter_noalloc) against csc_cheb_filter and
the float64 oracle.

Some callers cannot call cudaMalloc while they run: a framework whose caching allocator
reserved the device memory up front, or a latency-bound service that forbids allocation after
start-up (an allocation can synchronise the whole device).  The allocation-free entry point
serves them from a fixed static device array.  Here it must give the same features and trace
moments as the context-based entry point and the oracle (Sections 2.2 and 3.3), on two calls in
a row, because the second call reuses the scratch that the first one left behind.
"""
import numpy as np
import pytest

import workloads as W
from oracle import chebyshev as cb
from oracle import laplacian as lp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cases():
    g1 = W.sbm_graph(2000, 10, 20, 10, seed=1)
    g2 = W.random_csr(3001, 9, seed=4, isolated=40)
    rng = np.random.default_rng(0)
    rows = np.repeat(np.arange(g2.n), np.diff(g2.row_ptr))
    key = np.minimum(rows, g2.col_idx) * g2.n + np.maximum(rows, g2.col_idx)
    _, inv = np.unique(key, return_inverse=True)
    vals = rng.uniform(0.1, 3.0, inv.max() + 1)[inv].astype(np.float32)
    # (graph, weights, m, cutoff, c, psi wanted)
    return [(g1, None, 50, 0.53, 13, True), (g2, vals, 40, 0.8, 24, True),
            (g2, vals, 1, 0.8, 9, True), (g1, None, 30, 0.4, 17, False)]


@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_noalloc_matches_context_entry_point_and_oracle(gpu_lib, case):
    g, vals, m, lam, c, want_psi = _cases()[case]
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    vv = None if vals is None else torch.from_numpy(vals).cuda()
    r_host = W.gaussian_block(g.n, c, 64, seed=case + 3)
    r = torch.from_numpy(r_host).cuda()
    with gpu_lib.Context() as ctx:
        ctx.set_graph(g.n, rp, ci, vv)
        ref = torch.zeros((g.n, c), device="cuda")
        mu_ref = ctx.cheb_filter(m, lam, r, ref)
    ref = ref.cpu().numpy()
    lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, vals)
    psi_oracle = cb.cheb_filter(lt, r_host.astype(np.float64), m, lam)
    mu_oracle = cb.moments(lt, r_host.astype(np.float64), 2 * m)
    for call in range(2):
        out = torch.full((g.n, c), float("nan"), device="cuda") if want_psi else None
        mu = gpu_lib.csc_cheb_filter_noalloc(g.n, rp, ci, vv, m, lam, r, out)
        assert mu.shape == (2 * m + 1,)
        assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0], f"call {call}"
        assert np.max(np.abs(mu - mu_oracle)) < FP32_TOL * mu_oracle[0], f"call {call}"
        if want_psi:
            got = out.cpu().numpy()
            assert np.isfinite(got).all(), f"call {call}"
            assert rel(got, ref) < FP32_TOL, f"call {call}"
            assert rel(got, psi_oracle) < FP32_TOL, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_limit(gpu_lib):
    rp = torch.zeros(3, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = torch.zeros((2, 2), device="cuda")
    big_n = 70_000
    with pytest.raises(gpu_lib.CscError) as err:
        gpu_lib.csc_cheb_filter_noalloc(big_n, torch.zeros(big_n + 1, dtype=torch.int64, device="cuda"),
                                        ci, None, 10, 0.5, torch.zeros((big_n, 2), device="cuda"))
    assert err.value.status == 6  # CSC_ELIMIT
    with pytest.raises(gpu_lib.CscError) as err:
        gpu_lib.csc_cheb_filter_noalloc(2, rp, ci, None, 129, 0.5, r)
    assert err.value.status == 6
    # more stored edges than the scratch's block table holds (rejected before any is read)
    many = torch.zeros((1 << 22) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.CscError) as err:
        gpu_lib.csc_cheb_filter_noalloc(2, rp, many, None, 10, 0.5, r)
    assert err.value.status == 6


def test_noalloc_rejects_bad_arrays(gpu_lib):
    n = 4
    rp = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64, device="cuda")
    ci = torch.tensor([1, 0, 3, 2], dtype=torch.int32, device="cuda")
    r = torch.zeros((n, 3), device="cuda")
    f = gpu_lib.csc_cheb_filter_noalloc
    with pytest.raises(TypeError):  # bfloat16 signals: the entry point reads float32 only
        f(n, rp, ci, None, 5, 0.5, r.to(torch.bfloat16))
    with pytest.raises(TypeError):  # host arrays
        f(n, rp.cpu(), ci, None, 5, 0.5, r)
    with pytest.raises(TypeError):
        f(n, rp, ci, None, 5, 0.5, r.cpu().numpy())
    with pytest.raises(ValueError):  # R with the wrong number of rows
        f(n, rp, ci, None, 5, 0.5, torch.zeros((n + 1, 3), device="cuda"))
    with pytest.raises(ValueError):  # output of the wrong shape
        f(n, rp, ci, None, 5, 0.5, r, torch.zeros((n, 2), device="cuda"))
    with pytest.raises(ValueError):  # row_ptr of the wrong length
        f(n, rp[:-1], ci, None, 5, 0.5, r)
    with pytest.raises(ValueError):  # one weight per stored edge
        f(n, rp, ci, torch.ones(3, device="cuda"), 5, 0.5, r)
    # the C entry point itself refuses a host pointer where device memory is required
    import ctypes
    host_r = np.zeros((n, 3), dtype=np.float32)
    mu = np.zeros(11)
    st = gpu_lib._lib().csc_cheb_filter_noalloc(
        n, 4, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()), None, 5, 0.5,
        ctypes.c_void_p(host_r.ctypes.data), 3, 3, None, 3,
        mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert st == 1  # CSC_EINVAL
