"""The numpy graph generators: node reassignment churn of Section 5.1 (CPU)."""
import numpy as np

import workloads as W


def _upper(g):
    return set(g.upper_keys().tolist())


def test_node_reassign_moves_and_rewires_only_the_picked_nodes():
    n, k = 4000, 8
    g = W.sbm_graph(n, k, 20, 10, seed=2)
    h = W.node_reassign(g, 0.01, seed=3)
    picked = h.model["reassigned"]
    assert picked.size == 40 and np.unique(picked).size == 40
    # every picked node changed block, no other node did
    assert np.all(h.labels[picked] != g.labels[picked])
    other = np.setdiff1d(np.arange(n), picked)
    assert np.array_equal(h.labels[other], g.labels[other])
    # simple symmetric graph
    rows = h.keys // n
    cols = h.keys % n
    assert np.all(rows != cols) and np.all(np.diff(h.keys) > 0)
    assert np.array_equal(np.sort(cols * n + rows), h.keys)
    # edges away from the picked nodes are untouched
    is_p = np.zeros(n, dtype=bool)
    is_p[picked] = True
    touch = lambda keys: is_p[np.array(sorted(keys)) // n] | is_p[np.array(sorted(keys)) % n]
    a, b = _upper(g), _upper(h)
    gone, new = a - b, b - a
    assert touch(gone).all() and touch(new).all()
    # the rewired nodes follow the model: degree near the average and the intra share of
    # their new blocks near the model's value
    deg = np.diff(h.row_ptr)[picked]
    assert abs(deg.mean() - 20) < 4
    nk = np.array(sorted(new))
    intra = np.mean(h.labels[nk // n] == h.labels[nk % n])
    s = n / k
    want = 10 * (s - 1) / (10 * (s - 1) + (n - s))
    assert abs(intra - want) < 0.12


def test_sbm_perturb_combines_both_models():
    g = W.sbm_graph(3000, 6, 20, 10, seed=4)
    h = W.sbm_perturb(g, 0.01, 0.03, seed=9)
    assert np.sum(h.labels != g.labels) == 30
    # a later redraw samples from the model of the new block sizes
    assert np.array_equal(h.model["sizes"], np.bincount(h.labels, minlength=6))
    h2 = W.edge_redraw(h, 0.03, seed=11)
    assert h2.nnz > 0
