"""k-means on the feature rows (Section 2.1, Eq. 1 and Eq. 2).  Test infrastructure only.

The paper clusters the feature rows with k-means and measures the result with
C_X = ||Phi - X X^T Phi||_F, X the n x k indicator with X_ij = 1/sqrt(s_j) (Eq. 1-2);
C_X^2 is the usual within-cluster sum of squares.  It does not fix the algorithm; the
readings taken here are Lloyd's iteration with

* initial centroids given by the caller: Forgy (k row indices) or a warm start
  (means of the previous snapshot's assignment on the new features, an empty
  cluster taking the Forgy row of the same index);
* assignment by float64 squared Euclidean distance, ties to the lowest index;
* update by float64 means, an empty cluster keeping its previous centroid;
* stop when an assignment equals the previous one, or after max_iter
  assignment passes.

Pins (tests/test_oracle_kmeans.py): brute-force optimum on tiny sets (n <= 10),
C_X equals the within-cluster root sum of squares, fixed-point invariants,
hand-checked tiny example in tests/golden/.
"""
from __future__ import annotations

import itertools

import numpy as np


def sq_distances(y: np.ndarray, c: np.ndarray) -> np.ndarray:
    """n x k matrix of sum_l (y_il - c_jl)^2 in float64."""
    y = np.asarray(y, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    out = np.empty((y.shape[0], c.shape[0]))
    for j in range(c.shape[0]):
        diff = y - c[j][None, :]
        out[:, j] = np.sum(diff * diff, axis=1)
    return out


def assign(y: np.ndarray, c: np.ndarray, chunk: int = 65536):
    """(labels, margin): argmin over centroids (lowest index on ties) and the top-2 gap."""
    n = y.shape[0]
    labels = np.empty(n, dtype=np.int32)
    margin = np.empty(n)
    for s in range(0, n, chunk):
        dist = sq_distances(y[s:s + chunk], c)
        lab = np.argmin(dist, axis=1)
        labels[s:s + chunk] = lab
        if c.shape[0] > 1:
            part = np.partition(dist, 1, axis=1)
            margin[s:s + chunk] = part[:, 1] - part[:, 0]
        else:
            margin[s:s + chunk] = np.inf
    return labels, margin


def update(y: np.ndarray, labels: np.ndarray, c_old: np.ndarray) -> np.ndarray:
    """Cluster means in float64; an empty cluster keeps its previous centroid."""
    y = np.asarray(y, dtype=np.float64)
    k = c_old.shape[0]
    c = np.array(c_old, dtype=np.float64, copy=True)
    for j in range(k):
        members = labels == j
        cnt = int(np.count_nonzero(members))
        if cnt > 0:
            c[j] = y[members].sum(axis=0) / cnt
    return c


def forgy_centroids(y: np.ndarray, idx) -> np.ndarray:
    return np.asarray(y, dtype=np.float64)[np.asarray(idx, dtype=np.int64)].copy()


def warm_centroids(y: np.ndarray, prev_labels: np.ndarray, idx) -> np.ndarray:
    """Means of the previous assignment on the current features; empty -> Forgy row."""
    return update(y, prev_labels, forgy_centroids(y, idx))


def lloyd(y: np.ndarray, c0: np.ndarray, max_iter: int = 100):
    """Lloyd's iteration.  Returns (labels, centroids, passes, converged).

    ``centroids`` are the ones the returned labels were assigned against; at
    convergence they are the means of those labels.
    """
    c = np.array(c0, dtype=np.float64, copy=True)
    prev = None
    labels = None
    for it in range(1, max_iter + 1):
        labels, _ = assign(y, c)
        converged = prev is not None and np.array_equal(labels, prev)
        if converged or it == max_iter:
            return labels, c, it, converged
        c = update(y, labels, c)
        prev = labels
    return labels, c, max_iter, False


def inertia(y: np.ndarray, labels: np.ndarray, c: np.ndarray) -> float:
    """sum_i ||y_i - c_{labels_i}||^2 in float64."""
    y = np.asarray(y, dtype=np.float64)
    diff = y - np.asarray(c, dtype=np.float64)[labels]
    return float(np.sum(diff * diff))


def indicator(labels: np.ndarray, k: int) -> np.ndarray:
    """X with X_ij = 1/sqrt(s_j) if i is in cluster j (Eq. 2), dense n x k."""
    n = labels.size
    x = np.zeros((n, k))
    for j in range(k):
        members = labels == j
        s = int(np.count_nonzero(members))
        if s:
            x[members, j] = 1.0 / np.sqrt(s)
    return x


def cost(phi: np.ndarray, labels: np.ndarray, k: int) -> float:
    """C_X = ||Phi - X X^T Phi||_F (Eq. 1) for the assignment ``labels``."""
    x = indicator(labels, k)
    phi = np.asarray(phi, dtype=np.float64)
    return float(np.linalg.norm(phi - x @ (x.T @ phi)))


def brute_force(y: np.ndarray, k: int):
    """Optimal k-means partition by enumeration (n <= 10).  Returns (labels, C_X)."""
    n = y.shape[0]
    best = (None, np.inf)
    for lab in itertools.product(range(k), repeat=n):
        lab = np.array(lab)
        if lab[0] != 0:
            continue  # label symmetry
        if np.unique(lab).size != k:
            continue
        val = cost(y, lab, k)
        if val < best[1] - 1e-15:
            best = (lab.astype(np.int32), val)
    return best
