"""Edge similarity of consecutive snapshots (csc_laplacian_distance, Definition 4.1) against the
oracle's sparse difference: unweighted and weighted pairs with isolated nodes, identical graphs,
and the dynamic workload's churned snapshot pair at n = 1e6."""
import numpy as np
import pytest

import workloads as W
from oracle import similarity as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev_graph(g, vals=None):
    return (torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(),
            None if vals is None else torch.from_numpy(vals).cuda())


def with_weights(g, seed):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = np.minimum(rows, g.col_idx).astype(np.int64) * g.n + np.maximum(rows, g.col_idx)
    # weight as a hash of the undirected edge, so both snapshots agree on surviving edges
    return (1.0 + (np.sin(key.astype(np.float64) * 0.7 + seed) + 1.0)).astype(np.float32)


@pytest.mark.parametrize("weighted", [False, True])
def test_distance_matches_oracle(gpu_lib, weighted):
    g0 = W.random_csr(5000, 8, seed=3, isolated=30)
    g1 = W.edge_redraw(g0, 0.03, seed=4)
    v0 = with_weights(g0, 1) if weighted else None
    v1 = with_weights(g1, 1) if weighted else None
    with gpu_lib.Context() as ctx:
        rho = ctx.laplacian_distance(g0.n, dev_graph(g0, v0), dev_graph(g1, v1))
        same = ctx.laplacian_distance(g0.n, dev_graph(g0, v0), dev_graph(g0, v0))
    ref = sm.laplacian_distance(g0.n, (g0.row_ptr, g0.col_idx, v0), (g1.row_ptr, g1.col_idx, v1))
    assert rho == pytest.approx(ref, rel=1e-10)
    assert same == 0.0


def test_distance_of_churned_snapshots_at_scale(gpu_lib):
    sizes = W.zipf_block_sizes(1_000_000, 100, 0.8)
    g0 = W.sbm_graph(1_000_000, sizes, 30, 10, seed=2)
    g1 = W.edge_redraw(g0, 0.005, seed=3)
    with gpu_lib.Context() as ctx:
        rho = ctx.laplacian_distance(g0.n, dev_graph(g0), dev_graph(g1))
    ref = sm.laplacian_distance(g0.n, (g0.row_ptr, g0.col_idx, None), (g1.row_ptr, g1.col_idx, None))
    assert rho == pytest.approx(ref, rel=1e-10)
