"""Pins of the oracle CG and mixed-precision refinement (LAPACK solves, closed-form spectra, exact residuals)."""
import numpy as np
import pytest

import gen
import oracle


def _csr_from_dense(D):
    n = D.shape[0]
    rows, cols = np.nonzero(D)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return gen.CSR(n, np.cumsum(rp), cols.astype(np.int32), D[rows, cols].astype(np.float64))


def _laplace1d(n):
    D = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return _csr_from_dense(D), D


@pytest.mark.parametrize("seed", range(4))
def test_cg_matches_lapack_on_small_spd(seed):
    rng = np.random.default_rng(seed)
    n = 30
    M = rng.standard_normal((n, n))
    D = M @ M.T + n * np.eye(n)
    D[np.abs(D) < 0.5] = 0.0  # sparsify, keeping strict diagonal dominance -> SPD
    D = (D + D.T) / 2
    D += np.diag(np.abs(D).sum(1))
    A = _csr_from_dense(D)
    b = rng.uniform(-1, 1, n)
    x, ok, it, rel = oracle.cg(A, b, rtol=1e-14, max_iter=500)
    assert ok
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_cg_1d_laplacian_spectrum_and_iteration_count():
    n = 64
    A, D = _laplace1d(n)
    # closed-form eigenvalues 2 - 2 cos(j pi / (n+1)): the operator really is the 1D Laplacian
    lam = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    assert np.allclose(np.linalg.eigvalsh(D), lam, rtol=0, atol=1e-12)
    xstar = np.sin(np.arange(1, n + 1) * 3 * np.pi / (n + 1)) + np.linspace(0, 1, n)
    b = oracle.spmv(A, xstar)
    x, ok, it, rel, hist = oracle.cg(A, b, rtol=1e-12, max_iter=10 * n, history=True)
    assert ok and it <= n + 2          # at most n steps in exact arithmetic (a few extra for rounding)
    assert np.linalg.norm(x - xstar) <= 1e-9 * np.linalg.norm(xstar)
    assert rel <= 1e-11
    # an eigenvector right-hand side converges in one step
    v = np.sin(np.arange(1, n + 1) * 5 * np.pi / (n + 1))
    x1, ok1, it1, _ = oracle.cg(A, v, rtol=1e-12, max_iter=10)
    assert ok1 and it1 == 1
    assert np.allclose(x1, v / (2 - 2 * np.cos(5 * np.pi / (n + 1))), rtol=1e-12, atol=0)


def test_cg_known_solution_fem():
    A = gen.tet_lap3d(N=12, dirichlet=True)
    xstar = gen.uniform(A.n, 23)
    b = oracle.spmv(A, xstar)
    x, ok, it, rel = oracle.cg(A, b, rtol=1e-10, max_iter=5000)
    assert ok
    r = b - oracle.spmv(A, x)                     # true residual recomputed independently
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b) + 1e-15
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-15
    assert np.linalg.norm(x - xstar) <= 1e-6 * np.linalg.norm(xstar)


def test_cg_reports_nonconvergence():
    A, _ = _laplace1d(200)
    b = np.ones(200)
    x, ok, it, rel = oracle.cg(A, b, rtol=1e-12, max_iter=5)
    assert not ok and it == 5 and rel > 1e-3


def test_cg_zero_rhs_is_immediate():
    A, _ = _laplace1d(10)
    x, ok, it, rel = oracle.cg(A, np.zeros(10), rtol=1e-10)
    assert ok and it == 0 and np.all(x == 0)


@pytest.mark.parametrize("bf16,inner", [(False, 1e-4), (True, 1e-2)])
def test_refined_cg_reaches_fp64_accuracy(bf16, inner):
    A = gen.tet_lap3d(N=10, dirichlet=True)
    xstar = gen.uniform(A.n, 23)
    b = oracle.spmv(A, xstar)
    x, ok, outer, inner_total, rel = oracle.cg_refined(A, b, bf16=bf16, rtol=1e-10, inner_rtol=inner)
    assert ok and outer >= 2   # the low-precision inner solve alone cannot reach 1e-10
    r = b - oracle.spmv(A, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-15


def test_refined_cg_on_clamped_elasticity():
    A = gen.hex_elast3d(N=5, clamp_minz=True)
    xstar = gen.uniform(A.n, 24)
    b = oracle.spmv(A, xstar)
    x, ok, outer, inner_total, rel = oracle.cg_refined(A, b, bf16=False, rtol=1e-10, inner_rtol=1e-4)
    assert ok
    assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= 1e-10
