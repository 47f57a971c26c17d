"""Dynamic compressive spectral clustering, Algorithm 1 (Section 4.1).  Test infrastructure only.

Per snapshot G_t (fixed vertex set):

1. t = 1 (the static start of Algorithm 1): draw d signals, find the cutoff by the
   dichotomy on [0, 2] using the eigencount of the filtered block, filter,
   cluster.
2. t >= 2 (the loop of Algorithm 1): keep dp = floor(p d) previously filtered columns, draw
   dq = d - dp new signals, filter them with the previous cutoff, compute the
   eigencount on them, keep the cutoff if the count is within tau of k, else
   refine it by the dichotomy (starting from the previous cutoff); the block
   filtered with the final cutoff is Psi_t's new part.  Combine (Eq. 6), row
   normalise, cluster.

Readings beyond the paper's text:

* Which dp columns are kept: the paper draws them at random and assumes
  p <= 0.5 so that they always come from G_{t-1}.  The feature matrix is kept
  as a ring of d slots stamped with the snapshot that filtered them; the dq
  slots with the oldest stamp (lowest slot index on ties) are overwritten,
  new column v going to the v-th of those slots in ascending order.  For
  p <= 0.5 this keeps only G_{t-1} columns (i.i.d., so equivalent to a random
  pick); for p > 0.5 staleness is bounded by ceil(d/dq) snapshots.
* Row normalisation y_i = theta_i / ||theta_i|| over all d columns (a zero
  row stays zero) before k-means.
* k-means: Forgy at t = 1; for t >= 2 a warm start from the previous
  assignment (Lloyd, see oracle.kmeans).
* Column g of the signal block is the Philox stream of global column id g;
  ids are handed out in order (0..d-1 at t = 1, then dq per snapshot).

Edge-similarity policy (optional; Section 4, Definition 4.1, Theorem 4.1, Corollary 4.2), with
rho_t = ||L_t - L_{t-1}||_F given per snapshot:

* Reuse fraction.  The proof of Theorem 4.1 bounds the error of the reused columns by
  ||(Psi_t - Psi_{t-1}) S||_F <= sqrt(p (1 + delta)) ||H_t - H_{t-1}||_F, and the k-means cost
  by twice that; Corollary 4.2 bounds ||H_t - H_{t-1}||_F by gamma = sqrt(2) rho_t / alpha for
  an eigengap alpha.  (The theorem's statement writes the term as (1 + delta) p gamma; the
  reading follows the proof.)  With delta = 1 and a budget eps on the added cost,
  2 sqrt(2 p) gamma <= eps gives p_t = min(p_max, eps^2 / (8 gamma^2)); dp_t = floor(p_t d), and
  dp_t = 0 refilters all d columns.  eps <= 0 or rho_t = 0 keeps p_max.
* Eigencount check.  Weyl's inequality gives |lambda_i(L_t) - lambda_i(L_s)| <= ||L_t - L_s||_2
  <= sum of rho since snapshot s, so while the sum of rho since the last check stays <= rho_skip
  the previous cutoff is kept without the check (Section 4.1: recompute lambda_k from time to
  time only); otherwise the check (and refinement) of Algorithm 1 runs and the sum restarts.
  rho_skip = 0 keeps Algorithm 1's check at every snapshot with rho_t > 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import chebyshev as cb
from . import kmeans as km
from . import laplacian as lp
from .philox import forgy_draw, gaussian_columns


def row_normalize(theta: np.ndarray) -> np.ndarray:
    """y_i = theta_i / ||theta_i||_2; a zero row stays zero."""
    theta = np.asarray(theta, dtype=np.float64)
    nrm = np.sqrt(np.sum(theta * theta, axis=1))
    out = np.zeros_like(theta)
    nz = nrm > 0
    out[nz] = theta[nz] / nrm[nz, None]
    return out


def reuse_policy(d: int, p_max: float, rho: float, alpha: float, budget: float, rho_skip: float,
                 rho_since: float) -> tuple[int, bool, float]:
    """(dp, run the eigencount check, rho summed since the last check) for one snapshot under the
    edge-similarity policy of the module header."""
    acc = rho_since + rho
    p = p_max
    if budget > 0.0 and rho > 0.0:
        gamma = math.sqrt(2.0) * rho / alpha
        p = min(p_max, budget * budget / (8.0 * gamma * gamma))
    dp = int(math.floor(p * d))
    check = not (acc <= rho_skip)
    return dp, check, (0.0 if check else acc)


def oldest_slots(stamp: np.ndarray, count: int) -> np.ndarray:
    """The `count` slots with the smallest stamp, ties to the lowest slot, ascending slot order."""
    order = np.lexsort((np.arange(stamp.size), stamp))
    return np.sort(order[:count])


class DynamicCSC:
    """Algorithm 1 in float64.  ``step`` consumes one snapshot and returns its assignment."""

    def __init__(self, n: int, k: int, d: int, p: float, m: int, seed: int,
                 max_iter: int = 100, max_bisect: int = 30, tau: float | None = None):
        self.n, self.k, self.d, self.p, self.m, self.seed = n, k, d, p, m, seed
        self.max_iter, self.max_bisect, self.tau_fixed = max_iter, max_bisect, tau
        self.theta = np.zeros((n, d))
        self.stamp = np.zeros(d, dtype=np.int64)
        self.t = 0
        self.next_id = 0
        self.lam = None
        self.labels = None
        self.rho_since = 0.0
        self.history: list[dict] = []

    def step(self, row_ptr, col_idx, vals=None, init_idx=None, rho=None, policy=None) -> np.ndarray:
        """One snapshot.  With ``policy`` = dict(alpha, budget, rho_skip) and ``rho`` =
        ||L_t - L_{t-1}||_F the edge-similarity policy of the module header sets dp and whether
        the eigencount check runs (from the second snapshot on)."""
        self.t += 1
        n, d, k, m = self.n, self.d, self.k, self.m
        lt = lp.shifted_laplacian(n, row_ptr, col_idx, vals)
        check = True
        dp = int(math.floor(self.p * d)) if self.p > 0.0 else 0
        if policy is not None and self.t > 1:
            dp, check, self.rho_since = reuse_policy(d, self.p, rho, policy["alpha"], policy["budget"],
                                                     policy["rho_skip"], self.rho_since)
        if self.t == 1 or dp == 0:
            slots = np.arange(d)
        else:
            slots = oldest_slots(self.stamp, d - dp)
        c = slots.size
        ids = np.arange(self.next_id, self.next_id + c)
        r = gaussian_columns(self.seed, n, ids, d)
        basis = cb.cheb_basis(lt, r, m)

        def count_fn(lam):
            return cb.eigencount(cb.combine(basis, cb.filter_coefficients(m, lam)), d)

        tau = self.tau_fixed if self.tau_fixed is not None else cb.count_tolerance(k, c)
        if check or self.lam is None:
            lam, cnt, evals = cb.lambda_search(count_fn, k, tau, self.lam, self.max_bisect)
        else:
            lam, cnt, evals = self.lam, count_fn(self.lam), 0
        psi = cb.combine(basis, cb.filter_coefficients(m, lam))
        self.theta[:, slots] = psi
        self.stamp[slots] = self.t
        self.next_id += c
        self.lam = lam
        y = row_normalize(self.theta)
        if init_idx is None:
            init_idx = forgy_draw(self.seed ^ (self.t * 0x9E3779B97F4A7C15 & (2**64 - 1)), n, k)
        if self.labels is None:
            c0 = km.forgy_centroids(y, init_idx)
        else:
            c0 = km.warm_centroids(y, self.labels, init_idx)
        labels, cents, passes, conv = km.lloyd(y, c0, self.max_iter)
        self.labels = labels
        self.history.append(dict(t=self.t, lam=lam, count=cnt, evals=evals, c=c, slots=slots, checked=check,
                                 passes=passes, converged=conv,
                                 inertia=km.inertia(y, labels, cents)))
        return labels

    def features(self) -> np.ndarray:
        return self.theta.copy()
