"""Pins of the oracle's k-means (Section 2.1, Eq. 1-2) on the CPU."""
import numpy as np
import pytest

import workloads as W
from conftest import read_golden
from oracle import kmeans as km


def test_golden_line6_brute_force_and_cost():
    rows = {r[0]: r[1:] for r in read_golden("kmeans_line6.txt")}
    pts = np.array([float(x) for x in rows["points"]])[:, None]
    lab_ref = np.array([int(x) for x in rows["labels"]])
    cost_ref = float(rows["cost"][0])
    lab, val = km.brute_force(pts, 2)
    np.testing.assert_array_equal(lab, lab_ref)
    assert val == pytest.approx(cost_ref, abs=1e-14)
    assert km.cost(pts, lab_ref, 2) == pytest.approx(cost_ref, abs=1e-14)
    # Lloyd from a reasonable start reaches the same optimum
    lab2, c, it, conv = km.lloyd(pts, km.forgy_centroids(pts, [0, 5]))
    assert conv and np.array_equal(lab2, lab_ref)


def test_cost_is_root_within_cluster_sum_of_squares():
    y, _ = W.clustered_points(200, 5, 4, seed=2, normalize=False)
    lab = np.random.default_rng(0).integers(0, 4, 200)
    c = km.update(y, lab, np.zeros((4, 5)))
    assert km.cost(y, lab, 4) == pytest.approx(np.sqrt(km.inertia(y, lab, c)), rel=1e-12)


def test_lloyd_matches_brute_force_on_tiny_sets():
    rng = np.random.default_rng(7)
    for trial in range(6):
        y = np.concatenate([rng.normal(0, 0.2, (3, 2)), rng.normal(3, 0.2, (3, 2)),
                            rng.normal([0, 4], 0.2, (3, 2))])
        lab_bf, val = km.brute_force(y, 3)
        best = np.inf
        for start in ([0, 3, 6], [1, 4, 7], [2, 5, 8]):
            lab, c, it, conv = km.lloyd(y, km.forgy_centroids(y, start))
            best = min(best, km.cost(y, lab, 3))
        assert best == pytest.approx(val, rel=1e-12)


def test_lloyd_fixed_point_invariants():
    y, _ = W.clustered_points(3000, 16, 8, seed=3)
    idx = W.forgy_indices(3000, 8, seed=4)
    lab, c, it, conv = km.lloyd(y, km.forgy_centroids(y, idx), max_iter=200)
    assert conv
    # converged: labels are the argmin for c, and c are the means of labels
    lab2, margin = km.assign(y, c)
    np.testing.assert_array_equal(lab, lab2)
    np.testing.assert_allclose(km.update(y, lab, c), c, atol=1e-15)
    assert np.all(margin >= 0)


def test_assign_ties_go_to_lowest_index():
    y = np.array([[0.0, 0.0], [1.0, 0.0]])
    c = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0]])  # row 0 equidistant to all three
    lab, margin = km.assign(y, c)
    assert lab[0] == 0 and margin[0] == 0.0


def test_empty_cluster_keeps_centroid():
    y = np.array([[0.0], [0.1], [5.0]])
    c_old = np.array([[0.0], [100.0], [5.0]])
    lab, _ = km.assign(y, c_old)
    c = km.update(y, lab, c_old)
    assert c[1, 0] == 100.0


def test_warm_start_uses_previous_labels():
    y, lab_true = W.clustered_points(500, 6, 5, seed=8)
    idx = W.forgy_indices(500, 5, seed=1)
    c = km.warm_centroids(y, lab_true, idx)
    np.testing.assert_allclose(c, km.update(y, lab_true, np.zeros((5, 6))), atol=1e-15)
