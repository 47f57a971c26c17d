"""Jackson-damped Chebyshev low-pass filtering (Sections 2.2 and 3.3).  Test infrastructure only.

The paper replaces the ideal low-pass H_k = U diag(I_k, 0) U^T (Eq. 3) by a
polynomial filter h(L) = U h(Lambda) U^T evaluated with Chebyshev polynomials
in O(|E| d m) operations (Section 2.2, approximate features; Section 3.3).  It does not print
the coefficients; the readings taken here are:

* h approximates the step 1[lambda <= lambda_c] on [0, 2].  With x = lambda - 1
  and theta_c = arccos(lambda_c - 1), the Chebyshev projection of 1[x <= x_c]
  is c_0 = (pi - theta_c)/pi and c_j = -2 sin(j theta_c)/(j pi), j >= 1, with
  the series written h = sum_{j=0}^m a_j T_j(x) (c_0 not halved).
* The series is damped with Jackson coefficients g_j (kernel polynomial
  method), alpha = pi/(m+2):
  g_j = [(m+2-j) sin(alpha) cos(j alpha) + cos(alpha) sin(j alpha)] / ((m+2) sin(alpha)),
  and a_j = g_j c_j.  The Jackson kernel is positive, so h stays in [0, 1] and
  is monotone in the cutoff (in lambda up to the kernel's small edge ripple).
* T_j(L~) R comes from the three-term recursion T_0 R = R, T_1 R = L~ R,
  T_{j+1} R = 2 L~ T_j R - T_{j-1} R.
* Eigencount (the paper's Section 3.3 cites eigencount techniques without
  stating the estimator): count(lambda_c) = (d/c) ||h(L) R_c||_F^2 for a block
  of c signals of variance 1/d, an unbiased estimate of tr(h(L)^2).
* Dichotomy (Algorithm 1 and Section 4.1): accept a cutoff when
  |count - k| <= tau with tau = max(0.5, 2 sqrt(2k/c)); with no previous cutoff
  bisect [0, 2]; with a previous cutoff test it first, then grow a bracket
  geometrically (0.01 * 2^i) in the direction of k until the count crosses k,
  then bisect; at most 30 evaluations.

Pins (tests/test_oracle_chebyshev.py): T_j(cos t) = cos(j t); c_j equal to the
numerical projection integral; Jackson g_0 = 1 and a positive kernel; the
filter applied to an eigenvector u_i returns h(lambda_i) u_i; dense
U h(Lambda) U^T R equality; cycle-graph closed form; moment identity;
E[count] = tr(h(L)^2) over seeds; monotone count; dichotomy on a known spectrum.
"""
from __future__ import annotations

import math

import numpy as np


def step_coefficients(m: int, lam_c: float) -> np.ndarray:
    """Chebyshev coefficients c_0..c_m of 1[lambda <= lam_c] on [0, 2] (x = lambda - 1)."""
    x_c = min(1.0, max(-1.0, lam_c - 1.0))
    theta = math.acos(x_c)
    c = np.empty(m + 1)
    c[0] = (math.pi - theta) / math.pi
    for j in range(1, m + 1):
        c[j] = -2.0 * math.sin(j * theta) / (j * math.pi)
    return c


def jackson(m: int) -> np.ndarray:
    """Jackson damping factors g_0..g_m for an order-m series."""
    mp2 = m + 2.0
    alpha = math.pi / mp2
    g = np.empty(m + 1)
    for j in range(m + 1):
        g[j] = ((mp2 - j) * math.sin(alpha) * math.cos(j * alpha)
                + math.cos(alpha) * math.sin(j * alpha)) / (mp2 * math.sin(alpha))
    return g


def filter_coefficients(m: int, lam_c: float) -> np.ndarray:
    """a_j = g_j c_j: the damped low-pass h(lambda) = sum_j a_j T_j(lambda - 1)."""
    return jackson(m) * step_coefficients(m, lam_c)


def response(a: np.ndarray, lam) -> np.ndarray:
    """h(lambda) = sum_j a_j T_j(lambda - 1), scalar three-term recursion."""
    x = np.asarray(lam, dtype=np.float64) - 1.0
    t_prev = np.ones_like(x)
    out = a[0] * t_prev
    if a.size == 1:
        return out
    t_cur = x.copy()
    out = out + a[1] * t_cur
    for j in range(2, a.size):
        t_next = 2.0 * x * t_cur - t_prev
        out = out + a[j] * t_next
        t_prev, t_cur = t_cur, t_next
    return out


def cheb_basis(lt, r: np.ndarray, order: int) -> list[np.ndarray]:
    """[T_0(L~) R, ..., T_order(L~) R] by the three-term recursion (float64)."""
    r = np.asarray(r, dtype=np.float64)
    basis = [r]
    if order >= 1:
        basis.append(lt @ r)
    for _ in range(2, order + 1):
        basis.append(2.0 * (lt @ basis[-1]) - basis[-2])
    return basis


def combine(basis: list[np.ndarray], a: np.ndarray) -> np.ndarray:
    """Psi~ = sum_j a_j T_j(L~) R."""
    out = np.zeros_like(basis[0])
    for j, tj in enumerate(basis[: a.size]):
        out += a[j] * tj
    return out


def cheb_filter(lt, r: np.ndarray, m: int, lam_c: float) -> np.ndarray:
    """Psi~ = h(L) R with the order-m Jackson-damped low-pass of cutoff lam_c."""
    return combine(cheb_basis(lt, r, m), filter_coefficients(m, lam_c))


def moments(lt, r: np.ndarray, top: int) -> np.ndarray:
    """mu_l = tr(R^T T_l(L~) R) for l = 0..top, by definition (float64)."""
    basis = cheb_basis(lt, r, top)
    r64 = np.asarray(r, dtype=np.float64)
    return np.array([float(np.sum(r64 * b)) for b in basis])


def eigencount(psi: np.ndarray, d: int) -> float:
    """count = (d/c) ||Psi~||_F^2 for a block of c signals of variance 1/d."""
    c = psi.shape[1]
    return float(d) / float(c) * float(np.sum(np.asarray(psi, dtype=np.float64) ** 2))


def trace_count(r: np.ndarray, psi: np.ndarray, d: int) -> float:
    """Hutchinson-type count (d/c) tr(R^T Psi~) = (d/c) tr(R^T h(L) R), an unbiased estimate
    of tr h(L) for a block of c signals of variance 1/d (the alternative estimator)."""
    c = psi.shape[1]
    return float(d) / float(c) * float(np.sum(np.asarray(r, dtype=np.float64) * np.asarray(psi, dtype=np.float64)))


def count_tolerance(k: int, c: int) -> float:
    """Acceptance half-width tau = max(0.5, 2 sqrt(2k/c))."""
    return max(0.5, 2.0 * math.sqrt(2.0 * k / c))


def lambda_search(count_fn, k: int, tau: float, lam_prev=None, max_steps: int = 30):
    """Dichotomy for the cutoff whose eigencount is within tau of k.

    Returns (lambda_c, count, evaluations).  See the module header for the rule.
    """
    evals = 0
    lam = cnt = None

    def ev(x):
        nonlocal evals
        evals += 1
        return count_fn(x)

    if lam_prev is None:
        lo, hi = 0.0, 2.0
    else:
        lam, cnt = lam_prev, ev(lam_prev)
        if abs(cnt - k) <= tau:
            return lam, cnt, evals
        direction = 1.0 if cnt < k else -1.0
        step = 0.01
        prev = lam_prev
        lo = hi = None
        while evals < max_steps:
            probe = min(2.0, max(0.0, lam_prev + direction * step))
            lam, cnt = probe, ev(probe)
            if abs(cnt - k) <= tau:
                return lam, cnt, evals
            crossed = (cnt > k) if direction > 0 else (cnt < k)
            if crossed or probe == 0.0 or probe == 2.0:
                lo, hi = min(prev, probe), max(prev, probe)
                break
            prev = probe
            step *= 2.0
        if lo is None:
            return lam, cnt, evals
    while evals < max_steps:
        mid = 0.5 * (lo + hi)
        lam, cnt = mid, ev(mid)
        if abs(cnt - k) <= tau:
            return lam, cnt, evals
        if cnt < k:
            lo = mid
        else:
            hi = mid
    return lam, cnt, evals
