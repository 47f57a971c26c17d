"""Gradients of a feature-space loss through the Chebyshev filter.  Test infrastructure only.

The paper has no derivative; this is the differentiation pattern grown from its filter
(Section 2.2 features Psi = sum_j a_j T_j(L~) R, Section 3.3 coefficients, Section 2.1
normalized Laplacian L~ = -D^{-1/2} W D^{-1/2}).  Everything here is float64 and plain:
every T_j R is kept, no checkpointing, no fusion.

* Loss: the k-means cost of the row-normalised features against fixed centroids mu and a
  fixed assignment a(i) (Eq. 1 with X fixed): loss = sum_i ||y_i - mu_a(i)||^2,
  y_i = psi_i / ||psi_i|| (a zero row stays zero and passes no gradient).
* dloss/dpsi_i = (g_i - y_i <y_i, g_i>) / ||psi_i|| with g_i = 2 (y_i - mu_a(i)).
* dloss/da_j = <G, T_j R> (Frobenius), G = dloss/dPsi.
* Adjoint of the recursion (L~ symmetric): Lambda_m = a_m G, Lambda_{m-1} = a_{m-1} G +
  2 L~ Lambda_m, Lambda_j = a_j G + 2 L~ Lambda_{j+1} - Lambda_{j+2}; the gradient with
  respect to the stored entries of L~ is dL~_uv = <Lambda_1[u], T_0 R[v]> +
  2 sum_{j=1}^{m-1} <Lambda_{j+1}[u], T_j R[v]> (T_1 = L~ T_0 carries factor 1, every later
  step factor 2).
* Edge weights: l~_uv = -w_uv / sqrt(d_u d_v), d_u = sum_v w_uv.  For a symmetric weight
  w_e, e = {u, v}, stored at (u, v) and (v, u):
  dloss/dw_e = -(dL~_uv + dL~_vu) / sqrt(d_u d_v) - s_u / (2 d_u) - s_v / (2 d_v),
  s_u = sum over the stored entries of row u and of column u of dL~ * l~.

Pins (tests/test_oracle_grad.py): central finite differences of the loss evaluated by the
plain forward recursion (no adjoint code) for the coefficients and the edge weights,
Euler's relation sum_e w_e dloss/dw_e = 0 (L~ does not change when every weight is scaled),
and the coefficient gradient of a one-step filter against its closed form.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as cb
from . import laplacian as lp


def filter_psi(lt, r: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Psi = sum_j a_j T_j(L~) R for an arbitrary coefficient vector a (float64)."""
    return cb.combine(cb.cheb_basis(lt, r, a.size - 1), np.asarray(a, dtype=np.float64))


def kmeans_loss(psi: np.ndarray, mu: np.ndarray, assign: np.ndarray) -> float:
    """sum_i ||psi_i / ||psi_i|| - mu_a(i)||^2, a zero row contributing ||mu_a(i)||^2."""
    psi = np.asarray(psi, dtype=np.float64)
    nrm = np.linalg.norm(psi, axis=1)
    y = np.zeros_like(psi)
    nz = nrm > 0
    y[nz] = psi[nz] / nrm[nz, None]
    diff = y - np.asarray(mu, dtype=np.float64)[np.asarray(assign)]
    return float(np.sum(diff * diff))


def kmeans_loss_grad(psi: np.ndarray, mu: np.ndarray, assign: np.ndarray):
    """(loss, dloss/dPsi)."""
    psi = np.asarray(psi, dtype=np.float64)
    nrm = np.linalg.norm(psi, axis=1)
    y = np.zeros_like(psi)
    nz = nrm > 0
    y[nz] = psi[nz] / nrm[nz, None]
    diff = y - np.asarray(mu, dtype=np.float64)[np.asarray(assign)]
    g = 2.0 * diff
    grad = np.zeros_like(psi)
    proj = np.sum(y * g, axis=1)
    grad[nz] = (g[nz] - y[nz] * proj[nz, None]) / nrm[nz, None]
    return float(np.sum(diff * diff)), grad


def filter_vjp(lt, r: np.ndarray, a: np.ndarray, gbar: np.ndarray):
    """(dloss/da, dloss/dL~ at the stored entries of lt in CSR order) for Psi = p(L~) R."""
    a = np.asarray(a, dtype=np.float64)
    m = a.size - 1
    basis = cb.cheb_basis(lt, r, m)
    gbar = np.asarray(gbar, dtype=np.float64)
    grad_a = np.array([float(np.sum(gbar * tj)) for tj in basis])
    lt = lt.tocsr()
    rows = np.repeat(np.arange(lt.shape[0]), np.diff(lt.indptr))
    cols = lt.indices
    grad_l = np.zeros(cols.size)
    if m == 0:
        return grad_a, grad_l
    lam = [None] * (m + 2)
    lam[m + 1] = np.zeros_like(gbar)
    lam[m] = a[m] * gbar
    for j in range(m - 1, 0, -1):
        lam[j] = a[j] * gbar + 2.0 * (lt @ lam[j + 1]) - lam[j + 2]
    # dL~_uv = <Lambda_1[u], T_0[v]> + 2 sum_{j>=1} <Lambda_{j+1}[u], T_j[v]>
    grad_l += np.sum(lam[1][rows] * basis[0][cols], axis=1)
    for j in range(1, m):
        grad_l += 2.0 * np.sum(lam[j + 1][rows] * basis[j][cols], axis=1)
    return grad_a, grad_l


def edge_weight_grad(n: int, row_ptr, col_idx, vals, grad_l: np.ndarray) -> np.ndarray:
    """dloss/dw_e per stored entry (both stored copies of an edge get the same value)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    w = np.ones(col_idx.size) if vals is None else np.asarray(vals, dtype=np.float64)
    deg = lp.degrees(n, row_ptr, col_idx, w)
    s_inv = lp.inv_sqrt_degree(deg)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    ltv = -w * s_inv[rows] * s_inv[col_idx]
    prod = np.asarray(grad_l, dtype=np.float64) * ltv
    s = np.bincount(rows, weights=prod, minlength=n) + np.bincount(col_idx, weights=prod, minlength=n)
    # position of the transposed entry (v, u) of every stored (u, v)
    key = rows * n + col_idx
    tkey = col_idx * n + rows
    order = np.argsort(key)
    pos = order[np.searchsorted(key[order], tkey)]
    gsym = np.asarray(grad_l, dtype=np.float64) + np.asarray(grad_l, dtype=np.float64)[pos]
    with np.errstate(divide="ignore", invalid="ignore"):
        half_u = np.where(deg[rows] > 0, s[rows] / (2.0 * deg[rows]), 0.0)
        half_v = np.where(deg[col_idx] > 0, s[col_idx] / (2.0 * deg[col_idx]), 0.0)
    return -gsym * s_inv[rows] * s_inv[col_idx] - half_u - half_v


def loss_and_grads(n: int, row_ptr, col_idx, vals, r: np.ndarray, a: np.ndarray, mu: np.ndarray,
                   assign: np.ndarray):
    """(loss, dloss/da, dloss/dw per stored entry) of the k-means loss of the filtered features."""
    lt = lp.shifted_laplacian(n, row_ptr, col_idx, vals)
    psi = filter_psi(lt, r, a)
    loss, gbar = kmeans_loss_grad(psi, mu, assign)
    grad_a, grad_l = filter_vjp(lt, r, a, gbar)
    return loss, grad_a, edge_weight_grad(n, row_ptr, col_idx, vals, grad_l)
