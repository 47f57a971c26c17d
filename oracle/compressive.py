"""Compressive k-means (Section 2.2, step 2; Section 4.2 complexity).  Test infrastructure only.

The paper clusters only a sampled subset of the nodes and infers the remaining assignments
from a Tikhonov-regularised problem solved with k graph filterings, one per cluster, each of
cost linear in m|E|.  It names the ingredients (variable density sampling of O(k log k)
nodes, k-means on the sample, Tikhonov interpolation) and leaves their definitions to the
cited work.  The readings taken here, all float64 and plain:

* Sampling density.  p_i is proportional to s_i = ||theta_i||^2, the energy of node i's row of
  the unnormalised filtered signals Theta.  With R Gaussian of variance 1/d,
  E ||theta_i||^2 = ||h(L) delta_i||^2, which for the ideal low pass is the local cumulative
  coherence ||U_k^T delta_i||^2: the variable density under which O(k log k) samples
  suffice.
  - s_i is the float64 sum over l = 0, 1, ..., d-1, in that order, of theta_il^2 (each square
    of a float32 value is exact in float64).
  - Quantised to integers so that every prefix sum is exact: q_i = floor(s_i 2^E) with
    E = 62 - ceil(log2 n) - e and 2^(e-1) <= max_i s_i < 2^e; then every prefix sum
    P_i = q_0 + ... + q_i, and the total T = P_(n-1), is below 2^62.
* Draws.  n_draws independent draws with replacement.  Draw t uses Philox-4x32-10 with
  counter (t, 0, 0, 2) and the seed as key (the generator of oracle/philox.py);
  U = x0 2^32 + x1, u = floor(U T / 2^64), and the drawn node is the smallest i with P_i > u
  (a node with q_i = 0 is never drawn).  The sample Omega is the set of distinct drawn
  nodes in increasing order.
* Reduced k-means.  Lloyd's iteration of oracle/kmeans.py on the normalised rows y_i,
  i in Omega (in that order), restarted n_init times: restart r starts from the Forgy rows
  forgy_draw(seed_r, |Omega|, k) of the reduced set, seed_r = seed + r * 0x9E3779B97F4A7C15
  mod 2^64.  The restart with the lowest inertia (sum of squared distances to the centroids
  of its last assignment) is kept; inertias within a relative 1e-6 of the lowest count as
  equal and the lowest restart index wins among them.  A few hundred rows are cheap to
  cluster, and a single Forgy start on so few rows often merges two clusters.
* Interpolation (Tikhonov, one graph filtering per cluster).  For cluster j,
      x_j = argmin_x ||x - z_j||^2 + x^T G x,   z_ij = w_i [i in Omega and a_i = j],
  with the high-pass regulariser G = h(L)^{-1} - I built from the features' own low pass h
  (the order-m Jackson-damped step of cutoff lambda_c, Section 3.3): G vanishes on the pass
  band and grows without bound in the stop band.  The minimiser solves (I + G) x = z, that
  is x_j = h(L) z_j: one filtering of the weighted indicator per cluster with the recursion
  and coefficients of the features, the k filterings of cost O(m|E|) the paper counts.
  - w_i = 1 / (n p_i) = T / (n q_i) reweights by the inverse sampling density (weight 1
    under uniform sampling); evaluated as float(T) / (float(n) * float(q_i)) in float64.
  - Weaker regularisers were tried on a 4000-node, 8-block Zipf stochastic block model with
    the same sample and reduced labels (one Forgy start): G = gamma L (label propagation),
    in this denoising form or fitted on Omega only, put 45-70% of the nodes where full
    k-means puts them, against 84-93% for this one (98-99% with the restarts below).
* Assignment.  Node i goes to the lowest j maximising x_j(i).

Pins (tests/test_oracle_compressive.py): the empirical law of the draws against q / T
(chi-square); the density against the exact leverage scores ||U_k^T delta_i||^2 of a small
graph under the ideal projector; the quantisation bounds; the interpolation against the
ideal-projector interpolation U_k U_k^T z of a graph with a spectral gap (dense
eigendecomposition); the tie rule of the assignment; and the recovery of a planted partition.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as cb
from . import kmeans as km
from . import laplacian as lp
from . import philox as px


def row_energy(theta: np.ndarray) -> np.ndarray:
    """s_i = sum_l theta_il^2 accumulated in float64 over l = 0..d-1 in order."""
    theta = np.asarray(theta)
    s = np.zeros(theta.shape[0], dtype=np.float64)
    for l in range(theta.shape[1]):
        v = theta[:, l].astype(np.float64)
        s = s + v * v
    return s


def quantise(s: np.ndarray):
    """(q int64[n], E): q_i = floor(s_i 2^E), every prefix sum of q below 2^62."""
    s = np.asarray(s, dtype=np.float64)
    n = s.size
    smax = float(np.max(s)) if n else 0.0
    if not smax > 0.0:
        raise ValueError("all sampling weights are zero")
    _, e = np.frexp(smax)                      # smax = f 2^e, 0.5 <= f < 1
    lg_n = int(np.ceil(np.log2(max(n, 2))))
    big_e = 62 - lg_n - int(e)
    q = np.floor(np.ldexp(s, big_e)).astype(np.int64)
    return q, big_e


def draw_positions(seed: int, n_draws: int, total: int) -> list[int]:
    """u_t = floor(U_t T / 2^64) in [0, T) for t < n_draws, U_t = x0 2^32 + x1 of Philox
    counter (t, 0, 0, 2) under the seed."""
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    t = np.arange(n_draws, dtype=np.uint64)
    x0, x1, _, _ = px.philox4x32_10(t, 0, 0, 2, k0, k1)
    return [(((int(x0[i]) << 32) | int(x1[i])) * total) >> 64 for i in range(n_draws)]


def draw_nodes(seed: int, n_draws: int, prefix: np.ndarray) -> np.ndarray:
    """The n_draws drawn node indices (with repetitions), in draw order: for each u_t the
    smallest i with P_i > u_t."""
    prefix = np.asarray(prefix, dtype=np.int64)
    us = draw_positions(seed, n_draws, int(prefix[-1]))
    return np.array([int(np.searchsorted(prefix, u, side="right")) for u in us], dtype=np.int64)


def sample(theta: np.ndarray, n_draws: int, seed: int):
    """(Omega, q, T): distinct drawn nodes in increasing order, the weights, their total."""
    q, _ = quantise(row_energy(theta))
    prefix = np.cumsum(q)
    drawn = draw_nodes(seed, n_draws, prefix)
    return np.unique(drawn), q, int(prefix[-1])


def sample_weights(q: np.ndarray, total: int, omega: np.ndarray) -> np.ndarray:
    """w_i = T / (n q_i) for i in Omega, float64."""
    n = q.size
    return float(total) / (float(n) * q[omega].astype(np.float64))


def restart_seed(seed: int, r: int) -> int:
    """Key of the Forgy draw of restart r."""
    return (seed + r * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


def reduced_kmeans(y: np.ndarray, omega: np.ndarray, k: int, seed: int, max_iter: int, n_init: int):
    """Lloyd on the rows y[Omega], best of n_init Forgy restarts: (labels, passes, restart)."""
    yo = np.asarray(y, dtype=np.float64)[omega]
    runs = []
    for r in range(n_init):
        idx = px.forgy_draw(restart_seed(seed, r), omega.size, k)
        labels, c, passes, _ = km.lloyd(yo, km.forgy_centroids(yo, idx), max_iter)
        runs.append((km.inertia(yo, labels, c), labels, passes))
    best = min(v[0] for v in runs)
    for r, (val, labels, passes) in enumerate(runs):
        if val <= best * (1.0 + 1e-6):
            return labels, passes, r
    raise AssertionError("unreachable")


def tikhonov_rhs(n: int, k: int, omega: np.ndarray, labels: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Z (n x k): z_ij = w_i for i in Omega with label j, zero elsewhere."""
    z = np.zeros((n, k))
    z[omega, labels] = w
    return z


def interpolate(n: int, row_ptr, col_idx, vals, z: np.ndarray, m: int, lam_c: float) -> np.ndarray:
    """X = h(L) Z, h the order-m Jackson-damped low pass of cutoff lam_c (the Tikhonov minimiser)."""
    lt = lp.shifted_laplacian(n, row_ptr, col_idx, vals)
    return cb.cheb_filter(lt, np.asarray(z, dtype=np.float64), m, lam_c)


def argmax_assign(x: np.ndarray) -> np.ndarray:
    """Lowest index of the row maximum (np.argmax returns the first maximiser)."""
    return np.argmax(x, axis=1).astype(np.int32)


def compressive_kmeans(n: int, row_ptr, col_idx, vals, theta: np.ndarray, y: np.ndarray, k: int,
                       n_draws: int, m: int, lam_c: float, seed: int, max_iter: int = 100,
                       n_init: int = 10):
    """The whole step: dict with omega, labels (reduced), x (interpolated), assign."""
    omega, q, total = sample(theta, n_draws, seed)
    if omega.size < k:
        raise ValueError("fewer distinct sampled nodes than clusters")
    labels, passes, restart = reduced_kmeans(y, omega, k, seed, max_iter, n_init)
    w = sample_weights(q, total, omega)
    z = tikhonov_rhs(n, k, omega, labels, w)
    x = interpolate(n, row_ptr, col_idx, vals, z, m, lam_c)
    return {"omega": omega, "labels": labels, "passes": passes, "restart": restart, "weights": w, "z": z, "x": x,
            "assign": argmax_assign(x), "q": q, "total": total}
