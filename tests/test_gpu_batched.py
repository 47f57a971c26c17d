"""Batched filtering (many graphs, one persistent launch) against per-graph filtering and the oracle."""
import numpy as np
import pytest

import workloads as W
from conftest import fp32_floor
from oracle import chebyshev as cb
from oracle import laplacian as lp
from oracle.philox import gaussian_columns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 3e-3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _batch(seed=0, count=7):
    """Uneven graphs: SBM and Chung-Lu, n from 150 to 6000, k from 5 to 20, d = 4k (ragged tiles)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(150), np.log(6000))))
        k = int(rng.integers(5, 21))
        deg = float(rng.uniform(8, 30))
        g = (W.sbm_graph(n, k, deg, 10, seed=100 + i) if i % 2 == 0 else
             W.chung_lu_graph(n, 2.5, deg, k, 0.2, seed=200 + i))
        out.append(dict(g=g, c=4 * k, d=4 * k, lam=float(rng.uniform(0.2, 1.2)), seed=1000 + i))
    return out


def _descs(batch):
    descs = []
    for b in batch:
        g = b["g"]
        descs.append(dict(n=g.n, row_ptr=torch.from_numpy(g.row_ptr).cuda(),
                          col_idx=torch.from_numpy(g.col_idx).cuda(), vals=None, c=b["c"], d=b["d"],
                          lambda_c=b["lam"], seed=b["seed"],
                          psi=torch.zeros((g.n, b["c"]), device="cuda")))
    return descs


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_matches_oracle(gpu_lib, precision):
    m = 30
    batch = _batch()
    descs = _descs(batch)
    with gpu_lib.Context({"precision": precision}) as ctx:
        mu = ctx.filter_batched(descs, m)
        st = ctx.stats()
    assert st["batched_launches"] == 1 and st["autotune_trials"] >= 1
    for b, dsc, mu_g in zip(batch, descs, mu):
        g = b["g"]
        lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx)
        r = gaussian_columns(b["seed"], g.n, np.arange(b["c"]), b["d"])
        if precision == 1:
            r_used = torch.from_numpy(r.astype(np.float32)).to(torch.bfloat16).double().numpy()
        else:
            r_used = r
        ref = cb.cheb_filter(lt, r_used, m, b["lam"])
        got = dsc["psi"].cpu().numpy()
        # float32 signals differ from the float64 draws by float32 rounding (~1e-7)
        assert rel(got, ref) < FP32_TOL, (g.n, b["c"])
        if precision == 1:
            assert rel(got, cb.cheb_filter(lt, r, m, b["lam"])) < BF16_TOL
        mu_ref = cb.moments(lt, r_used, 2 * m)
        assert np.max(np.abs(mu_g - mu_ref)) < FP32_TOL * mu_ref[0]


def test_batched_replay_and_per_graph_agreement(gpu_lib):
    m = 25
    batch = _batch(seed=3, count=5)
    descs = _descs(batch)
    with gpu_lib.Context() as ctx:
        ctx.filter_batched(descs, m)
        first = [d["psi"].clone() for d in descs]
        for d in descs:
            d["psi"].zero_()
        mu2 = ctx.filter_batched(descs, m)
        st = ctx.stats()
        assert st["batched_launches"] == 2
        for a, d in zip(first, descs):
            assert torch.equal(a, d["psi"])           # replay reproduces the first run exactly
        # per-graph path with the same counter-based signals
        for b, d, mu_g in zip(batch, descs, mu2):
            g = b["g"]
            ctx.set_graph(g.n, d["row_ptr"], d["col_idx"])
            r = torch.zeros((g.n, b["c"]), device="cuda")
            ctx.signals(b["seed"], g.n, 0, b["c"], b["d"], r)
            ref = torch.zeros_like(r)
            mu_ref = ctx.cheb_filter(m, b["lam"], r, ref)
            assert rel(d["psi"].cpu().numpy(), ref.cpu().numpy()) < FP32_TOL
            assert np.max(np.abs(mu_g - mu_ref)) < FP32_TOL * mu_ref[0]


def test_batched_weighted_edgeless_tiny_and_several_waves(gpu_lib):
    """A weighted graph, an edgeless graph, a single node, and a 3e5-node graph with 256 columns
    whose four 64-column tiles each exceed a 256 MB wave budget (so the schedule crosses waves);
    every graph against the oracle (sampled columns for the large one)."""
    m = 30
    rng = np.random.default_rng(9)
    gw = W.sbm_graph(500, 5, 12, 10, seed=41)
    rows = np.repeat(np.arange(gw.n), np.diff(gw.row_ptr))
    key = np.minimum(rows, gw.col_idx).astype(np.int64) * gw.n + np.maximum(rows, gw.col_idx)
    _, inv = np.unique(key, return_inverse=True)
    wvals = rng.uniform(0.5, 2.0, inv.max() + 1)[inv].astype(np.float32)
    class Csr:  # edgeless graphs as plain CSR
        def __init__(self, n):
            self.n, self.row_ptr, self.col_idx = n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)

    big = W.sbm_graph(300_000, 10, 10, 10, seed=42)
    cases = [(gw, wvals, 20, 0.7), (Csr(50), None, 12, 0.5), (Csr(1), None, 4, 0.9), (big, None, 256, 0.4)]
    descs = []
    for i, (g, vals, c, lam) in enumerate(cases):
        descs.append(dict(n=g.n, row_ptr=torch.from_numpy(g.row_ptr).cuda(),
                          col_idx=torch.from_numpy(g.col_idx).cuda(),
                          vals=None if vals is None else torch.from_numpy(vals).cuda(),
                          c=c, d=c, lambda_c=lam, seed=77 + i, psi=torch.zeros((g.n, c), device="cuda")))
    with gpu_lib.Context({"wave_bytes": 256 << 20}) as ctx:
        mu = ctx.filter_batched(descs, m)
        st = ctx.stats()
    assert st["batched_waves"] >= 4
    for i, ((g, vals, c, lam), dsc) in enumerate(zip(cases, descs)):
        lt = lp.shifted_laplacian(g.n, g.row_ptr, g.col_idx, vals)
        cols = np.arange(c) if g.n < 1000 else np.array([0, 70, 150, 255])
        r = gaussian_columns(77 + i, g.n, cols, c)
        ref = cb.cheb_filter(lt, r, m, lam)
        got = dsc["psi"].cpu().numpy()[:, cols]
        tol = max(FP32_TOL, 2.0 * fp32_floor(lt, r, cb.filter_coefficients(m, lam), ref))
        assert rel(got, ref) < tol, (i, rel(got, ref), tol)
        if g.n < 1000:
            mu_ref = cb.moments(lt, r, 2 * m)
            assert np.max(np.abs(mu[i] - mu_ref)) < FP32_TOL * mu_ref[0], i


def test_expired_dependency_wait_returns_etimeout(gpu_lib, monkeypatch):
    """Failure detection without a GPU fault: a host-side hook makes the first tile wait for a
    block that does not exist.  The bounded wait runs out (about a second), the call returns
    CSC_ETIMEOUT, and the same context then filters the batch correctly."""
    import time
    m = 20
    batch = _batch(seed=5, count=4)
    descs = _descs(batch)
    with gpu_lib.Context({"precision": 1}) as ref_ctx:
        mu_ref = ref_ctx.filter_batched(_descs(batch), m)
    with gpu_lib.Context({"precision": 1}) as ctx:
        monkeypatch.setenv("CSC_TEST_EXPIRE_WAIT", "1")
        t0 = time.perf_counter()
        with pytest.raises(gpu_lib.CscError) as e:
            ctx.filter_batched(descs, m)
        elapsed = time.perf_counter() - t0
        monkeypatch.delenv("CSC_TEST_EXPIRE_WAIT")
        assert e.value.status == 4 and "bounded dependency wait" in str(e.value)
        assert elapsed < 60
        mu = ctx.filter_batched(descs, m)
    np.testing.assert_array_equal(mu, mu_ref)
