"""Graph Laplacians (Section 2.1).  Test infrastructure only.

The paper lets spectral clustering use either the combinatorial or the
normalized Laplacian; this oracle follows the normalized one,
L = I - D^{-1/2} W D^{-1/2}, whose spectrum lies in [0, 2].  The Chebyshev
recursion runs on the shifted operator L~ = L - I = -D^{-1/2} W D^{-1/2},
whose spectrum lies in [-1, 1] (lambda_max fixed at 2, not estimated).

An isolated node (degree 0) has no defined D^{-1/2}; its row and column of
D^{-1/2} W D^{-1/2} are empty, so its L~ row is zero and its L eigenvalue is 1.

Pins: dense spectra of the cycle C_n and complete graph K_n (closed forms),
symmetry, zero row sums of L D^{1/2} 1 (L annihilates D^{1/2} 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def degrees(n: int, row_ptr: np.ndarray, col_idx: np.ndarray, vals=None) -> np.ndarray:
    """deg_i = sum_j W_ij (Section 2.1), float64."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    if vals is None:
        return np.diff(row_ptr).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return np.bincount(rows, weights=np.asarray(vals, dtype=np.float64), minlength=n)


def inv_sqrt_degree(deg: np.ndarray) -> np.ndarray:
    """D^{-1/2} with 0 for isolated nodes."""
    out = np.zeros_like(deg, dtype=np.float64)
    nz = deg > 0
    out[nz] = 1.0 / np.sqrt(deg[nz])
    return out


def adjacency(n: int, row_ptr, col_idx, vals=None) -> sp.csr_matrix:
    """W as a scipy CSR matrix (float64)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    data = np.ones(col_idx.size) if vals is None else np.asarray(vals, dtype=np.float64)
    return sp.csr_matrix((data, col_idx, row_ptr), shape=(n, n))


def shifted_laplacian(n: int, row_ptr, col_idx, vals=None) -> sp.csr_matrix:
    """L~ = L - I = -D^{-1/2} W D^{-1/2} as a float64 CSR matrix."""
    w = adjacency(n, row_ptr, col_idx, vals)
    s = inv_sqrt_degree(degrees(n, row_ptr, col_idx, vals))
    dmat = sp.diags(s)
    return (-(dmat @ w @ dmat)).tocsr()


def normalized_laplacian_dense(n: int, row_ptr, col_idx, vals=None) -> np.ndarray:
    """L = I - D^{-1/2} W D^{-1/2} as a dense float64 matrix (small n only)."""
    return np.eye(n) + shifted_laplacian(n, row_ptr, col_idx, vals).toarray()
