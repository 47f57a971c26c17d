"""Exact spectral clustering quantities by dense eigendecomposition (Sections 2.1, 3 and 4).

Test infrastructure only, for small graphs (n of a few thousand at most).

* Phi = U_k, the eigenvectors of the k smallest eigenvalues of L (Section 2.1).
* H_k = U diag(I_k, 0) U^T, the ideal low-pass (Eq. 3).
* h(L) R = U h(Lambda) U^T R for any polynomial response h (Section 3.3).
* Thm 3.3: min over unitary Q of ||H_k R - Phi I_{k x d} Q||_F equals
  ||Sigma - I_{k x d}||_F with Sigma the singular values of U_k^T R; the
  minimiser is built from the SVD of U_k^T R.
* Definition 4.1 similarity metrics ||H_k^t - H_k^{t-1}||_F and
  ||L_t - L_{t-1}||_F.

These are exact definitions written out with LAPACK (numpy.linalg.eigh/svd).
"""
from __future__ import annotations

import numpy as np


def eig(lap_dense: np.ndarray):
    """Eigenvalues (ascending) and orthonormal eigenvectors of a symmetric matrix."""
    return np.linalg.eigh(lap_dense)


def features(lap_dense: np.ndarray, k: int) -> np.ndarray:
    """Phi = U_k (n x k)."""
    _, u = eig(lap_dense)
    return u[:, :k]


def ideal_projector(lap_dense: np.ndarray, k: int) -> np.ndarray:
    """H_k = U_k U_k^T (Eq. 3)."""
    uk = features(lap_dense, k)
    return uk @ uk.T


def apply_response(lap_dense: np.ndarray, h, r: np.ndarray) -> np.ndarray:
    """U h(Lambda) U^T R for a vectorised scalar response h."""
    lam, u = eig(lap_dense)
    return u @ (h(lam)[:, None] * (u.T @ r))


def thm33_gap(phi: np.ndarray, psi: np.ndarray, r: np.ndarray):
    """Both sides of the Thm 3.3 equality for Psi = H_k R.

    Returns (||Psi - Phi I_{k x d} Q||_F with the constructed Q,
             ||Sigma - I_{k x d}||_F).
    """
    k = phi.shape[1]
    d = r.shape[1]
    rp = phi.T @ r                                  # R' = I_{k x n} U^T R  (k x d)
    ql, sig, qrt = np.linalg.svd(rp, full_matrices=True)  # R' = Q_L Sigma Q_R^T
    block = np.eye(d)
    block[:k, :k] = ql
    q = block @ qrt                                 # Q = diag(Q_L, I) Q_R^T
    lhs = np.linalg.norm(psi - phi @ np.eye(k, d) @ q)
    rhs = np.linalg.norm(np.diag(sig) - np.eye(k, k)) if d >= k else np.nan
    return float(lhs), float(rhs)


def sc_assignment_cost(phi: np.ndarray, labels: np.ndarray, k: int) -> float:
    """C_X with the SC features Phi (Eq. 1, Eq. 4/5)."""
    from .kmeans import cost
    return cost(phi, labels, k)
