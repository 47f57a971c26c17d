"""The torch graph generators draw simple symmetric graphs of the stated models (CPU, small n)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")


def _check_simple(g):
    n, k = g.n, g.keys
    assert torch.all(k[1:] > k[:-1])  # sorted, no duplicate entries
    r, c = k // n, k % n
    assert torch.all(r != c)  # no self-loops
    assert torch.equal(torch.sort(c * n + r).values, k)  # symmetric
    assert int(g.row_ptr[0]) == 0 and int(g.row_ptr[-1]) == g.nnz
    assert torch.equal(g.col_idx.long(), c)
    assert torch.equal(torch.repeat_interleave(torch.arange(n), torch.diff(g.row_ptr)), r)


def test_chung_lu_torch_model():
    n, k, deg, mix = 60000, 16, 25.0, 0.2
    g = W.chung_lu_graph_torch(n, 2.5, deg, k, mix, seed=3)
    _check_simple(g)
    # mean degree near the target (duplicates and self-loops are dropped)
    assert 0.85 * deg < g.nnz / n <= deg
    r, c = g.keys // n, g.keys % n
    lab = g.labels.long()
    intra = float((lab[r] == lab[c]).double().mean())
    # intra-community share: 1 - mixing, plus the mixed draws that land in u's community
    assert abs(intra - (1 - mix + mix / k)) < 0.02
    # power-law tail: the degree of the heaviest nodes far above the mean
    assert int(torch.diff(g.row_ptr).max()) > 20 * deg
    again = W.chung_lu_graph_torch(n, 2.5, deg, k, mix, seed=3)
    assert torch.equal(again.keys, g.keys)


def test_edge_redraw_torch_changes_exactly_the_fraction():
    g = W.chung_lu_graph_torch(20000, 2.5, 20.0, 8, 0.2, seed=1)
    frac = 0.01
    h = W.edge_redraw_torch(g, frac, seed=2)
    _check_simple(h)
    n = g.n
    up = lambda x: set(x.keys[(x.keys // n) < (x.keys % n)].tolist())
    a, b = up(g), up(h)
    want = round(frac * len(a))
    assert len(a - b) == want and len(b - a) == want


def test_sbm_torch_model():
    n, k, deg, ratio = 40000, 10, 20.0, 10.0
    g = W.sbm_graph_torch(n, k, deg, ratio, seed=5)
    _check_simple(g)
    assert abs(g.nnz / n - deg) < 0.05 * deg
    r, c = g.keys // n, g.keys % n
    lab = g.labels.long()
    intra = float((lab[r] == lab[c]).double().mean())
    s = n / k
    want = ratio * (s - 1) / (ratio * (s - 1) + (n - s))
    assert abs(intra - want) < 0.02
    assert np.array_equal(np.bincount(g.labels.numpy(), minlength=k), np.full(k, n // k))


def test_edge_redraw_torch_sbm_keeps_the_block_structure():
    n, k, ratio = 30000, 6, 10.0
    g = W.sbm_graph_torch(n, W.zipf_block_sizes(n, k, 0.8), 20.0, ratio, seed=4)
    h = W.edge_redraw_torch(g, 0.05, seed=5)
    _check_simple(h)
    up = lambda x: x.keys[(x.keys // n) < (x.keys % n)]
    a, b = up(g), up(h)
    new = b[~torch.isin(b, a)]
    old = a[~torch.isin(a, b)]
    assert new.numel() == old.numel() == round(0.05 * a.numel())
    lab = g.labels.long()
    frac = lambda e: float((lab[e // n] == lab[e % n]).double().mean())
    # redrawn edges follow the model: the same intra-block share as the original edges
    assert abs(frac(new) - frac(a)) < 0.03
