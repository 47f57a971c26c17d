"""Pins of the similarity oracle (oracle/similarity.py, Definition 4.1 and Corollary 4.2)."""
import numpy as np
import pytest

import workloads as W
from oracle import laplacian as lp
from oracle import similarity as sm


def _cycle(n, chord=None):
    edges = [(i, (i + 1) % n) for i in range(n)]
    if chord is not None:
        edges.append(chord)
    rows = [u for u, v in edges] + [v for u, v in edges]
    cols = [v for u, v in edges] + [u for u, v in edges]
    order = np.lexsort((cols, rows))
    rows, cols = np.asarray(rows)[order], np.asarray(cols)[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int64)


def test_distance_matches_dense_definition():
    g0 = W.sbm_graph(300, 3, 8, 10, seed=1)
    g1 = W.edge_redraw(g0, 0.05, seed=2)
    d = sm.laplacian_distance(g0.n, (g0.row_ptr, g0.col_idx, None), (g1.row_ptr, g1.col_idx, None))
    dense = np.linalg.norm(lp.normalized_laplacian_dense(g1.n, g1.row_ptr, g1.col_idx) -
                           lp.normalized_laplacian_dense(g0.n, g0.row_ptr, g0.col_idx))
    assert d == pytest.approx(dense, rel=1e-12)
    assert sm.laplacian_distance(g0.n, (g0.row_ptr, g0.col_idx, None), (g0.row_ptr, g0.col_idx, None)) == 0.0


def test_single_chord_on_a_cycle_by_hand():
    """C_n has every off-diagonal entry -1/2.  A chord (0, m) makes nodes 0 and m degree 3:
    their two cycle edges each become -1/sqrt(6) (4 edges, 8 entries) and the chord adds
    -1/3 twice; every other entry is unchanged."""
    n, m = 12, 6
    rp0, c0 = _cycle(n)
    rp1, c1 = _cycle(n, (0, m))
    d = sm.laplacian_distance(n, (rp0, c0, None), (rp1, c1, None))
    expect = np.sqrt(8 * (0.5 - 1 / np.sqrt(6)) ** 2 + 2 * (1 / 3) ** 2)
    assert d == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_corollary_4_2_inequality(seed):
    g0 = W.sbm_graph(200, 4, 12, 20, seed=seed)
    g1 = W.edge_redraw(g0, 0.02, seed=seed + 10)
    l0 = lp.normalized_laplacian_dense(g0.n, g0.row_ptr, g0.col_idx)
    l1 = lp.normalized_laplacian_dense(g1.n, g1.row_ptr, g1.col_idx)
    k = 4
    alpha = sm.cor42_alpha(l0, l1, k)
    assert alpha > 0
    lhs = sm.spectral_distance(l0, l1, k)
    rhs = np.sqrt(2) / alpha * np.linalg.norm(l1 - l0)
    assert lhs <= rhs
