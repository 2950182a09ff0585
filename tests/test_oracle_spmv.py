"""Pins of the oracle SpMV/SpMM to values fixed by mathematics, not by the oracle itself."""
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle


def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col[k]] += A.val[k]
    return D


@pytest.mark.parametrize("seed", range(6))
def test_spmv_vs_dense_brute_force(seed):
    # non-symmetric, duplicates, empty rows: a transposed operand or a dropped duplicate fails here
    A = gen.random_csr(48 + seed, seed, mean_row=5, duplicates=True, empty_frac=0.15)
    x = np.random.default_rng(100 + seed).uniform(-1, 1, A.n)
    y = oracle.spmv(A, x)
    D = _dense(A)
    assert not np.allclose(D, D.T)
    yd = D @ x
    assert np.allclose(y, yd, rtol=0, atol=1e-14 * (abs(D) @ abs(x)).max())
    assert np.all(y[np.diff(A.row_ptr) == 0] == 0.0)


def test_spmv_unit_vectors_give_columns():
    A = gen.random_csr(40, 11, mean_row=6)
    D = _dense(A)
    for j in range(A.n):
        e = np.zeros(A.n); e[j] = 1.0
        assert np.array_equal(oracle.spmv(A, e), D[:, j])  # exact: each product is val*1, one term per entry


@pytest.mark.parametrize("seed", range(3))
def test_spmv_integer_exact(seed):
    # small integers: every partial sum is an integer below 2^53, so FP64 is exact
    A = gen.random_csr(500, seed, mean_row=20, int_values=True, duplicates=True, long_rows=4, long_len=3000)
    x = gen.int_vector(A.n, seed + 7)
    y = oracle.spmv(A, x)
    exact = np.zeros(A.n, dtype=object)
    for i in range(A.n):
        exact[i] = sum(int(A.val[k]) * int(x[A.col[k]]) for k in range(A.row_ptr[i], A.row_ptr[i + 1]))
    assert np.array_equal(y, exact.astype(np.float64))


def test_spmv_fractions_exact_row():
    # one row summed in exact rational arithmetic: the oracle is within the recursive-summation bound
    rng = np.random.default_rng(5)
    n = 300
    A = gen.CSR(n, np.r_[0, np.full(n, n)].astype(np.int64), np.arange(n, dtype=np.int32), rng.uniform(-1, 1, n))
    x = rng.uniform(-1, 1, n)
    y = oracle.spmv(A, x)[0]
    exact = sum(Fraction(float(v)) * Fraction(float(xx)) for v, xx in zip(A.val, x))
    err = abs(Fraction(y) - exact)
    bound = oracle.gamma(n) * float(np.sum(np.abs(A.val * x)))
    assert float(err) <= bound


def test_spmv_scipy_cross_check():
    A = gen.fem2d_p1(N=40)
    x = gen.uniform(A.n, 3)
    y = oracle.spmv(A, x)
    ys = A.to_scipy() @ x
    assert np.abs(y - ys).max() <= 4 * oracle.gamma(7) * oracle.abs_spmv(A, x).max()


def test_spmv_empty_matrix():
    A = gen.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.spmv(A, np.zeros(0)).size == 0


def test_spmm_is_columnwise_dense_product():
    A = gen.random_csr(60, 3, mean_row=7, duplicates=True)
    X = np.random.default_rng(4).uniform(-1, 1, (A.n, 8))
    Y = oracle.spmm(A, X)
    D = _dense(A)
    assert np.allclose(Y, D @ X, rtol=0, atol=1e-14 * (abs(D) @ abs(X)).max())
    for j in range(8):
        assert np.array_equal(Y[:, j], oracle.spmv(A, X[:, j].copy()))


def test_spmv_low_precision_rounding():
    # integer data is exact in FP32/BF16 (|v| <= 8, |x| <= 8, row sums < 2^24)
    A = gen.random_csr(300, 9, mean_row=12, int_values=True)
    x = gen.int_vector(A.n, 10)
    for bf in (False, True):
        assert np.array_equal(oracle.spmv_low(A, x, bf), oracle.spmv(A, x))
    # BF16 keeps 8 significant bits: 1 + 2^-8 rounds to 1 (ties to even), 1 + 3*2^-8 rounds up to 1 + 2^-6
    B = gen.CSR(2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32), np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8]))
    y = oracle.spmv_low(B, np.ones(2), True)
    assert y[0] == 1.0 and y[1] == 1.0 + 2 ** -6
    yf = oracle.spmv_low(B, np.ones(2), False)
    assert yf[0] == 1 + 2 ** -8
