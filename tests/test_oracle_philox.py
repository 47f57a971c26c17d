"""Pins of the oracle's counter-based generator and Gaussian signals (Section 2.2, approximate features)."""
import numpy as np
import pytest
from scipy import stats

from oracle.philox import forgy_draw, gaussian_columns, index_from_words, philox4x32_10


def test_gaussian_moments_and_normality():
    d = 64
    r = gaussian_columns(12345, 20000, np.arange(8), d)
    z = (r * np.sqrt(d)).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    corr = np.corrcoef(r.T)
    off = corr[~np.eye(8, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(20000)


def test_columns_are_keyed_independently():
    full = gaussian_columns(7, 500, np.arange(10), 10)
    part = gaussian_columns(7, 500, np.array([3, 9]), 10)
    np.testing.assert_array_equal(part, full[:, [3, 9]])
    other_seed = gaussian_columns(8, 500, np.array([3]), 10)
    assert not np.allclose(other_seed[:, 0], full[:, 3])


def test_uniform_bits_are_uniform():
    x0, x1, x2, x3 = philox4x32_10(np.arange(100000), 0, 5, 0, 1, 2)
    for x in (x0, x1, x2, x3):
        u = x.astype(np.float64) / 2.0**32
        assert stats.kstest(u, "uniform").pvalue > 1e-3
    # the round function mixes all inputs: changing one counter word changes every output word
    y = philox4x32_10(np.arange(1000), 0, 6, 0, 1, 2)
    for a, b in zip((x0[:1000], x1[:1000], x2[:1000], x3[:1000]), y):
        assert np.mean(a == b) < 0.01


def test_forgy_draw_distinct_in_range():
    idx = forgy_draw(99, 50, 50)
    assert sorted(idx.tolist()) == list(range(50))
    idx = forgy_draw(99, 10**6, 100)
    assert idx.min() >= 0 and idx.max() < 10**6 and np.unique(idx).size == 100


def test_forgy_index_map_on_published_words():
    """floor(U n / 2^64) on the published output words, worked out by hand
    (tests/golden/forgy_index_map.txt): power-of-two n reads off the top bits of x0, and at
    n = 2^31 - 2 the low word x1 decides the result, so a map that drops x1, reduces U mod n or
    uses one word only fails."""
    from conftest import read_golden
    rows = read_golden("forgy_index_map.txt")
    assert len(rows) == 12
    for x0, x1, n, want in rows:
        assert index_from_words(int(x0, 16), int(x1, 16), int(n)) == int(want)
    # the words come from the known-answer outputs of the generator itself
    kat = read_golden("philox4x32_10_kat.txt")
    words = {(int(r[6], 16), int(r[7], 16)) for r in kat}
    assert {(int(x0, 16), int(x1, 16)) for x0, x1, _, _ in rows} == words


def test_forgy_single_draw_uniform_over_seeds():
    """The first Forgy index is uniform on [0, n): chi-square over 7000 seeds (n = 7)."""
    n, seeds = 7, 7000
    counts = np.bincount([int(forgy_draw(s, n, 1)[0]) for s in range(seeds)], minlength=n)
    assert counts.size == n
    assert stats.chisquare(counts).pvalue > 1e-3


def test_forgy_ordered_pairs_uniform_over_seeds():
    """With the redraw of a repeated index, (first, second) is uniform over the n (n - 1)
    ordered distinct pairs: chi-square over 6000 seeds (n = 4, 12 pairs)."""
    n, seeds = 4, 6000
    counts = np.zeros((n, n), dtype=np.int64)
    for s in range(seeds):
        a, b = forgy_draw(1000 + s, n, 2)
        counts[a, b] += 1
    assert np.all(np.diag(counts) == 0)
    off = counts[~np.eye(n, dtype=bool)]
    assert stats.chisquare(off).pvalue > 1e-3


def test_published_known_answer_vectors():
    """The generator is Philox-4x32-10 as published: the known-answer vectors of its authors'
    Random123 distribution (tests/golden/philox4x32_10_kat.txt)."""
    from conftest import read_golden
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        words = [int(x, 16) for x in row]
        ctr, key, want = words[:4], words[4:6], words[6:10]
        got = philox4x32_10(*ctr, *key)
        assert [int(v) for v in got] == want
