"""Column-sharded Algorithm 1 (paper_1706_03591_gb300.sharded) on two gloo ranks (CPU).

Each rank filters a contiguous range of the snapshot's new global column ids; the trace moments
are all-reduced, rank 0 decides the cutoff with the library's dichotomy and broadcasts it, and the
filtered columns are all-gathered into a replicated feature ring.  The ranks' compute here is a
float64 stand-in built from the oracle (the GPU backend is the library's); the result must equal
the single-process oracle of Algorithm 1 (oracle.dynamic.DynamicCSC): the same cutoff and number
of dichotomy evaluations at every snapshot, bit for bit, the same features and the same
assignments, over a sequence perturbed by node reassignment and edge redrawing (Section 5.2).
"""
import os
import socket

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
mp = torch.multiprocessing

N, K, D, M, SEED = 600, 4, 24, 20, 31


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graphs(count=4):
    g = W.sbm_graph(N, K, 14, 10, seed=5)
    out = [g]
    for t in range(1, count):
        out.append(W.sbm_perturb(out[-1], 0.01, 0.03, seed=100 + t))
    return out


def _inits(count=4):
    return [W.forgy_indices(N, K, seed=700 + t) for t in range(count)]


class OracleColumns:
    """float64 stand-in for one rank's GPU work, built from the oracle's functions."""

    def __init__(self, n, d):
        from oracle.dynamic import oldest_slots  # noqa: F401
        self.n, self.d = n, d
        self.theta = np.zeros((n, d))
        self.stamp = np.zeros(d, dtype=np.int64)
        self.t = 0
        self.labels = None

    def set_graph(self, n, row_ptr, col_idx, vals=None):
        from oracle import laplacian as lp
        self.lt = lp.shifted_laplacian(n, row_ptr, col_idx, vals)

    def filter(self, m, lam, seed, col0, c, d, want_psi):
        from oracle import chebyshev as cb
        from oracle.philox import gaussian_columns
        r = gaussian_columns(seed, self.n, np.arange(col0, col0 + c), d)
        mu = cb.moments(self.lt, r, 2 * m)
        psi = torch.from_numpy(cb.cheb_filter(self.lt, r, m, lam)) if want_psi else None
        return psi, mu

    def splice(self, n, d, p, psi_all, lam):
        from oracle.dynamic import oldest_slots, row_normalize
        c = psi_all.shape[1]
        slots = np.arange(d) if self.t == 0 or p <= 0 else oldest_slots(self.stamp, c)
        self.t += 1
        self.theta[:, slots] = psi_all.numpy()
        self.stamp[slots] = self.t
        self.y = row_normalize(self.theta)

    def cluster(self, k, seed, init_idx, assign_out):
        from oracle import kmeans as km
        c0 = km.forgy_centroids(self.y, init_idx) if self.labels is None else \
            km.warm_centroids(self.y, self.labels, init_idx)
        labels, cents, passes, _ = km.lloyd(self.y, c0, 100)
        self.labels = labels
        assign_out[:] = labels
        return km.inertia(self.y, labels, cents), passes


def _worker(rank, world, port, p, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1706_03591_gb300.sharded import ShardedDynamicCSC
    be = OracleColumns(N, D)
    drv = ShardedDynamicCSC(be, N, K, D, p, M, SEED)
    res = []
    for g, idx in zip(_graphs(), _inits()):
        assign = np.zeros(N, dtype=np.int32)
        rec = drv.step(g.row_ptr, g.col_idx, idx, assign)
        res.append((rec["lam"], rec["evals"], rec["c"], rec["columns"], assign.copy()))
    out[rank] = (res, be.theta.copy())
    dist.destroy_process_group()


@pytest.mark.parametrize("p", [0.5, 0.75])
def test_two_rank_sharded_algorithm1_equals_single_process_oracle(p):
    from paper_1706_03591_gb300 import build
    build.build()
    from oracle.dynamic import DynamicCSC
    ref = DynamicCSC(N, K, D, p, M, SEED)
    want = []
    for g, idx in zip(_graphs(), _inits()):
        want.append(ref.step(g.row_ptr, g.col_idx, init_idx=idx))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, p, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=240)
            assert pr.exitcode == 0
        res = {r: out[r] for r in range(2)}
    for r in range(2):
        steps, theta = res[r]
        for t, (lam, evals, c, cols, assign) in enumerate(steps):
            h = ref.history[t]
            assert lam == h["lam"], (r, t, lam, h["lam"])
            assert evals == h["evals"], (r, t)
            assert c == h["c"]
            np.testing.assert_array_equal(assign, want[t])
        # the two ranks split every snapshot's columns without overlap
        for t in range(len(steps)):
            a0, b0 = res[0][0][t][3]
            a1, b1 = res[1][0][t][3]
            assert a0 == 0 and b0 == a1 and b1 == steps[t][2]
        np.testing.assert_allclose(theta, ref.features(), rtol=0, atol=1e-12)
    # the first snapshot searched the cutoff, later ones checked it first
    assert ref.history[0]["evals"] > 1


def test_column_ranges_partition():
    from paper_1706_03591_gb300.sharded import column_ranges, new_column_count
    for c in (1, 7, 39, 40, 192):
        for world in (1, 2, 3, 8):
            rr = column_ranges(c, world)
            assert rr[0][0] == 0 and rr[-1][1] == c
            assert all(rr[i][1] == rr[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rr]
            assert max(sizes) - min(sizes) <= 1
    assert new_column_count(0, 192, 0.8) == 192 and new_column_count(3, 192, 0.8) == 39
    assert new_column_count(2, 64, 0.0) == 64
