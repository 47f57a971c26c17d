"""Pins of the feature ring of Algorithm 1 (Eq. 6) in oracle/dynamic.py.

The reading keeps the dp most recently filtered columns (FIFO) and replaces the dq = d - dp
oldest, ties to the lowest slot.  The pins: a brute-force choice over all slot subsets, the
staleness bound of the ring (no column older than ceil(d / dq) snapshots), the exact column
bookkeeping of a sequence, and the row normalisation's invariants.
"""
import itertools
import math

import numpy as np
import pytest

from oracle.dynamic import oldest_slots, row_normalize


def _brute_oldest(stamp, count):
    """The subset of `count` slots whose (stamp, slot) pairs are the smallest, by enumeration."""
    best = None
    for sub in itertools.combinations(range(stamp.size), count):
        key = sorted((int(stamp[i]), i) for i in sub)
        if best is None or key < best[0]:
            best = (key, sub)
    return np.array(sorted(best[1]))


@pytest.mark.parametrize("seed", range(6))
def test_oldest_slots_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    stamp = rng.integers(0, 4, 8)          # many ties
    for count in range(0, 9):
        np.testing.assert_array_equal(oldest_slots(stamp, count), _brute_oldest(stamp, count))


@pytest.mark.parametrize("d,p", [(8, 0.75), (10, 0.5), (12, 0.8), (7, 0.3)])
def test_ring_staleness_and_column_bookkeeping(d, p):
    """Simulates the ring's stamps over many snapshots: each snapshot replaces exactly the dq
    oldest slots with the next dq column ids, and no slot is older than ceil(d / dq)."""
    dp = int(math.floor(p * d))
    dq = d - dp
    stamp = np.zeros(d, dtype=np.int64)
    col = -np.ones(d, dtype=np.int64)
    next_id = 0
    for t in range(1, 40):
        slots = np.arange(d) if t == 1 else oldest_slots(stamp, dq)
        assert slots.size == (d if t == 1 else dq)
        col[slots] = np.arange(next_id, next_id + slots.size)
        next_id += slots.size
        stamp[slots] = t
        assert t - stamp.min() < math.ceil(d / dq)
        # the ring holds the d most recent column ids of the columns it kept, none twice
        assert np.unique(col).size == d and col.max() == next_id - 1


def test_row_normalisation_invariants():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal((50, 7))
    theta[3] = 0.0
    y = row_normalize(theta)
    norms = np.linalg.norm(y, axis=1)
    np.testing.assert_allclose(np.delete(norms, 3), 1.0, rtol=1e-15)
    assert np.all(y[3] == 0.0)
    # direction preserved and scale invariant per row
    np.testing.assert_allclose(row_normalize(theta * rng.uniform(0.1, 10.0, (50, 1))), y, rtol=1e-13, atol=1e-15)
    assert np.all(np.sign(y[theta != 0]) == np.sign(theta[theta != 0]))
