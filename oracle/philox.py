"""Counter-based random signals (Section 2.2, approximate features).  Test infrastructure only.

The paper draws R in R^{n x d} with centred i.i.d. Gaussian entries of
variance 1/d.  The method's draws must be reproducible per column so that a
reused column (Eq. 6) is never regenerated and a refiltered column sees the
same signal; both the oracle and the CUDA path therefore implement one
counter-based generator from its published definition:

* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC 2011): multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key
  increments 0x9E3779B9 and 0xBB67AE85, ten rounds.
* Element (row i, global column g) uses counter (i mod 2^32, i div 2^32, g, 0)
  and key (seed mod 2^32, seed div 2^32).  Outputs x0, x1 give
  u1 = (floor(x0 / 2^8) + 1) 2^-24 in (0, 1] and u2 = floor(x1 / 2^8) 2^-24,
  both exact in float32; Box-Muller (1958) gives z = sqrt(-2 ln u1) cos(2 pi u2);
  R_ig = z / sqrt(d).
* Forgy indices: draw j uses counter (j, attempt, 0, 1); idx = floor(U n / 2^64)
  with U = x0 * 2^32 + x1; a repeated index is redrawn with attempt + 1.

Pins (tests/test_oracle_philox.py): the published known-answer vectors of
Philox-4x32-10 (tests/golden/philox4x32_10_kat.txt); the statistics of the
signals (mean, variance 1/d, normality, column independence); the index map
on the published output words, evaluated by hand (tests/golden/forgy_index_map.txt);
chi-square uniformity of single Forgy draws over many seeds and of ordered
distinct pairs (the redraw of a repeated index).
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on uint32 counters (carried in uint64 arrays)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def gaussian_columns(seed: int, n: int, col_ids, d: int) -> np.ndarray:
    """n x len(col_ids) float64 block, entry (i, v) = N(0, 1/d) draw for (row i, column col_ids[v])."""
    col_ids = np.asarray(col_ids, dtype=np.uint64)
    rows = np.arange(n, dtype=np.uint64)[:, None]
    g = col_ids[None, :]
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    x0, x1, _, _ = philox4x32_10(rows & _MASK, rows >> np.uint64(32), g, np.uint64(0), k0, k1)
    u1 = ((x0 >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (x1 >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z / np.sqrt(float(d))


def index_from_words(x0: int, x1: int, n: int) -> int:
    """Index in [0, n) of one draw: floor(U n / 2^64) with the 64-bit word U = x0 2^32 + x1
    (exact integer arithmetic, so every index has probability within 2^-64 n of 1/n)."""
    u = (int(x0) << 32) | int(x1)
    return (u * int(n)) >> 64


def forgy_draw(seed: int, n: int, k: int) -> np.ndarray:
    """k distinct row indices in [0, n) from the counter-based stream 1."""
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    chosen: list[int] = []
    seen = set()
    for j in range(k):
        attempt = 0
        while True:
            x0, x1, _, _ = philox4x32_10(j, attempt, 0, 1, k0, k1)
            idx = index_from_words(x0, x1, n)
            if idx not in seen:
                break
            attempt += 1
        seen.add(idx)
        chosen.append(idx)
    return np.array(chosen, dtype=np.int64)
