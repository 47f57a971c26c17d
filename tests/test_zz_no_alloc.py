"""The allocation-free filter entry point (csc_cheb_filter_noalloc) against csc_cheb_filter.

Some callers cannot allocate device memory while they run (inside a stream capture, under
an allocator that owns all device memory, or after a service has started).  The
allocation-free entry point serves them from a fixed static device array; here it must give
the same features and trace moments as the context-based entry point, on two calls in a row
(the second call reuses the scratch the first one left behind).
"""
import numpy as np
import pytest

import workloads as W

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
    return [(g1, None, 50, 0.53, 13), (g2, vals, 40, 0.8, 24)]


@pytest.mark.parametrize("case", [0, 1])
def test_noalloc_matches_context_entry_point(gpu_lib, case):
    g, vals, m, lam, c = _cases()[case]
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    vv = None if vals is None else torch.from_numpy(vals).cuda()
    r = torch.from_numpy(W.gaussian_block(g.n, c, 64, seed=case + 3)).cuda()
    with gpu_lib.Context() as ctx:
        ctx.set_graph(g.n, rp, ci, vv)
        ref = torch.zeros((g.n, c), device="cuda")
        mu_ref = ctx.cheb_filter(m, lam, r, ref)
    ref = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((g.n, c), float("nan"), device="cuda")
        mu = gpu_lib.csc_cheb_filter_noalloc(g.n, rp, ci, vv, m, lam, r, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), f"call {call}"
        assert rel(got, ref) < FP32_TOL, f"call {call}"
        assert np.max(np.abs(mu - mu_ref)) < FP32_TOL * mu_ref[0], f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_limit(gpu_lib):
    rp = torch.zeros(3, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = torch.zeros((4, 2), device="cuda")
    with pytest.raises(gpu_lib.CscError) as err:
        gpu_lib.csc_cheb_filter_noalloc(70_000, rp, ci, None, 10, 0.5, r)
    assert err.value.status == 6  # CSC_ELIMIT
    with pytest.raises(gpu_lib.CscError) as err:
        gpu_lib.csc_cheb_filter_noalloc(2, rp, ci, None, 129, 0.5, r)
    assert err.value.status == 6
