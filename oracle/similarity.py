"""Graph similarity metrics of a dynamic sequence (Definition 4.1, Corollary 4.2).  Test
infrastructure only.

* rho-edge similarity: ||L_t - L_{t-1}||_F with L = I - D^{-1/2} W D^{-1/2} (Section 2.1) on
  a common node set; the identity cancels (an isolated node has L_ii = 1 in both), so this is
  the Frobenius norm of the difference of the off-diagonal parts, over the union of the two
  edge sets (an edge absent from one graph contributes its full entry).
* (rho, k)-spectral similarity: ||H_k^t - H_k^{t-1}||_F with H_k the projector on the first k
  eigenvectors (Eq. 3), by dense eigendecomposition (small graphs).
* Corollary 4.2: if alpha > 0, alpha <= lambda_{k+1}^{(t-1)} - lambda_k^{(t)} and
  alpha <= lambda_k^{(t)}, then ||H_k^t - H_k^{t-1}||_F <= sqrt(2)/alpha ||L_t - L_{t-1}||_F.

Pins (tests/test_oracle_similarity.py): the sparse difference against the dense matrices of
oracle.laplacian, zero for identical graphs, a hand-computed single-edge toggle on a cycle,
and Corollary 4.2's inequality on random pairs.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg  # noqa: F401  (sparse norm)

from . import laplacian as lp


def laplacian_distance(n: int, g_prev, g_cur) -> float:
    """||L_cur - L_prev||_F; each graph is (row_ptr, col_idx, vals or None)."""
    a = lp.shifted_laplacian(n, *g_prev)
    b = lp.shifted_laplacian(n, *g_cur)
    return float(scipy.sparse.linalg.norm(b - a, "fro"))


def spectral_distance(lap_prev: np.ndarray, lap_cur: np.ndarray, k: int) -> float:
    """||H_k^cur - H_k^prev||_F from dense Laplacians."""
    _, u0 = np.linalg.eigh(lap_prev)
    _, u1 = np.linalg.eigh(lap_cur)
    h0 = u0[:, :k] @ u0[:, :k].T
    h1 = u1[:, :k] @ u1[:, :k].T
    return float(np.linalg.norm(h1 - h0))


def cor42_alpha(lap_prev: np.ndarray, lap_cur: np.ndarray, k: int) -> float:
    """Largest alpha allowed by Corollary 4.2 (<= 0 when the corollary does not apply)."""
    ev0 = np.linalg.eigvalsh(lap_prev)
    ev1 = np.linalg.eigvalsh(lap_cur)
    return float(min(ev0[k] - ev1[k - 1], ev1[k - 1]))
