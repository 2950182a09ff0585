"""Pins of the oracle's 16 tuner features (oracle/features.py) against values the mathematics fixes.

Each matrix below is built so that its features have closed forms, and each closed form is chosen so a
plausible misreading fails: population vs sample standard deviation, floor vs round vs ceil vs
interpolated percentiles, ranks counted from 0 vs 1 in the Gini sum, "longer than 32" vs "at least 32",
strict vs non-strict diagonal dominance, a band of ceil(n/P) vs floor(n/P), blocks vs bands.  The
library's features are compared with this oracle in test_tuner_host.py.
"""
import math

import numpy as np
import pytest

import gen
from oracle import features as of


def _csr(n, rows):
    """CSR from a list of (columns, values) per row."""
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(c) for c, _ in rows])
    col = np.concatenate([np.asarray(c, np.int32) for c, _ in rows]) if n else np.zeros(0, np.int32)
    val = np.concatenate([np.asarray(v, np.float64) for _, v in rows]) if n else np.zeros(0)
    return gen.CSR(n, rp, col, val)


def _lower_triangle(n):
    """Row i holds columns 0..i, every value 1: row lengths 1, 2, ..., n."""
    return _csr(n, [(np.arange(i + 1), np.ones(i + 1)) for i in range(n)])


def test_row_length_statistics_of_lengths_one_to_n():
    n = 50
    f = of.features(_lower_triangle(n), P=10)
    nnz = n * (n + 1) // 2
    assert f[0] == pytest.approx(math.log2(n + 1))
    assert f[1] == pytest.approx(math.log2(nnz + 1))
    assert f[2] == pytest.approx((n + 1) / 2)
    assert f[3] == pytest.approx(math.sqrt((n * n - 1) / 12))             # population, not sample, std
    assert f[3] != pytest.approx(math.sqrt(n * (n + 1) / 12))
    assert f[4] == pytest.approx(math.log2(n + 1))                         # log2(max + 1), max = n
    assert f[5] == 1
    # percentile q = the floor(q (n - 1))-th (from 0) ascending length = floor(q (n - 1)) + 1 here:
    # p50 -> 25 (ceil 26), p90 -> 45 (ceil or interpolation 46 / 45.1), p99 -> 49 (round or ceil 50)
    assert (f[6], f[7], f[8]) == (25, 45, 49)
    assert f[9] == pytest.approx(18 / n)                                   # rows 33..50 are longer than 32
    assert f[10] == pytest.approx((n - 1) / (3 * n))                       # Gini of 1..n, ranks from 1


def test_gini_of_equal_lengths_is_zero_and_of_one_nonempty_row_is_maximal():
    n = 40
    eq = _csr(n, [([i, (i + 1) % n], [1.0, 1.0]) for i in range(n)])
    assert of.features(eq)[10] == pytest.approx(0.0, abs=1e-15)
    one = _csr(n, [(list(range(n)), np.ones(n)) if i == n - 1 else ([], []) for i in range(n)])
    assert of.features(one)[10] == pytest.approx((n - 1) / n)              # all mass on the last rank


def test_locality_dominance_symmetry_and_blocks_of_the_lower_triangle():
    n, P = 50, 10
    f = of.features(_lower_triangle(n), P=P)
    nnz = n * (n + 1) // 2
    # mean |i - j| over entries: sum_i i (i + 1) / 2 = (n - 1) n (n + 1) / 6 over nnz, then / n
    assert f[11] == pytest.approx((n - 1) / (3 * n))
    band = math.ceil(n / P)                                                # 5
    within = sum(min(i, band) + 1 for i in range(n))                       # entries with i - j <= band
    assert within == 6 * (n - 5) + 15
    assert f[12] == pytest.approx(within / nnz)
    # |a_ii| = 1 against an off-diagonal sum of i: rows 0 and 1 dominate (row 1 only with >=)
    assert f[13] == pytest.approx(2 / n)
    # only diagonal entries have a mirror; every row is sampled (n < 2000)
    assert f[14] == pytest.approx(n / nnz)
    # same block of 5 consecutive rows: row i keeps (i mod 5) + 1 of its entries
    assert f[15] == pytest.approx((n // band) * 15 / nnz)


@pytest.mark.parametrize("n,b", [(60, 0), (60, 3), (97, 5)])
def test_band_matrix(n, b):
    rows = [(list(range(max(0, i - b), min(n, i + b + 1))), None) for i in range(n)]
    rows = [(c, np.full(len(c), -1.0)) for c, _ in rows]
    for i, (c, v) in enumerate(rows):
        v[c.index(i)] = 2.0 * b + 0.5
    A = _csr(n, rows)
    f = of.features(A, P=152)
    nnz = sum(len(c) for c, _ in rows)
    total = sum(abs(i - j) for i, (c, _) in enumerate(rows) for j in c)
    # closed form of the total distance: interior rows give b (b + 1); the 2 x b edge rows lose the
    # distances of their cut-off neighbours
    closed = n * b * (b + 1) - 2 * sum(sum(range(k + 1, b + 1)) for k in range(b))
    assert total == closed
    assert f[11] == pytest.approx(closed / nnz / n)
    assert f[14] == 1.0                                                    # a band is structurally symmetric
    t = math.ceil(n / 152)                                                 # 1: entries with |i - j| <= 1
    within = n * (2 * min(t, b) + 1) - min(t, b) * (min(t, b) + 1)        # diagonals 0, +-1, ... +-min(t, b)
    assert f[12] == pytest.approx(within / nnz)
    # diagonal 2b + 0.5 against at most 2b off-diagonal ones: every row dominates
    assert f[13] == 1.0
    if b == 0:
        assert f[15] == 1.0 and f[11] == 0.0 and f[3] == 0.0 and f[10] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("n", [40, 41])
def test_anti_diagonal(n):
    A = _csr(n, [([n - 1 - i], [1.0]) for i in range(n)])
    f = of.features(A, P=8)
    expect = 0.5 if n % 2 == 0 else (n * n - 1) / (2 * n * n)              # mean |2i - n + 1| / n
    assert f[11] == pytest.approx(expect)
    assert f[14] == 1.0                                                    # (i, n-1-i) mirrors (n-1-i, i)
    # only the middle row of an odd n has its entry on the diagonal (dominant: 1 >= 0)
    assert f[13] == pytest.approx((n % 2) / n)
    band = math.ceil(n / 8)
    assert f[15] == pytest.approx(sum(i // band == (n - 1 - i) // band for i in range(n)) / n)
    assert f[15] < 0.5


def test_one_long_row_sets_log_max_and_the_tail_shares():
    n, L = 300, 250
    rows = [([i], [1.0]) for i in range(n)]
    rows[7] = (sorted(set(range(L)) | {7}), np.ones(len(set(range(L)) | {7})))
    A = _csr(n, rows)
    f = of.features(A)
    assert f[4] == pytest.approx(math.log2(L + 1))
    assert f[9] == pytest.approx(1 / n)                                    # one row longer than 32
    assert (f[5], f[6], f[7], f[8]) == (1, 1, 1, 1)                        # floor(0.99 x 299) = 296 < 299
    mean = (n - 1 + L) / n
    assert f[2] == pytest.approx(mean)
    assert f[3] == pytest.approx(math.sqrt(((n - 1) * (1 - mean) ** 2 + (L - mean) ** 2) / n))


def test_threshold_32_is_strict():
    n = 64
    rows = [(list(range(32)) if i < 10 else [i], None) for i in range(n)]
    rows = [(c, np.ones(len(c))) for c, _ in rows]
    assert of.features(_csr(n, rows))[9] == 0.0                            # length 32 is not longer than 32


def test_empty_matrix_and_matrix_without_entries():
    f = of.features(_csr(0, []))
    assert f[0] == 0.0 and np.all(f == 0.0)
    g = of.features(_csr(5, [([], [])] * 5))
    assert g[0] == pytest.approx(math.log2(6)) and g[1] == 0.0
    assert g[11] == g[12] == g[13] == g[15] == 0.0 and g[14] == 1.0       # nothing to mirror counts as symmetric
