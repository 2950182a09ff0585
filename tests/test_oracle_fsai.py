"""Pins of the FSAI / preconditioned-CG oracle against what the mathematics fixes: the full pattern gives the
inverse Cholesky factor, the diagonal pattern gives Jacobi scaling, every FSAI row satisfies its defining
equations, PCG solves against LAPACK, and PCG with the identity preconditioner is CG."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle
from oracle import fsai as of


def _dense_spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    S = sp.csr_matrix(A)
    return gen.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.copy()), A


def test_full_pattern_is_the_inverse_cholesky_factor():
    A, D = _dense_spd(12, 1)
    G = of.fsai(A, pattern="full").toarray()
    Linv = np.linalg.inv(np.linalg.cholesky(D))
    assert np.allclose(G, Linv, rtol=1e-11, atol=1e-13)
    assert np.allclose(G @ D @ G.T, np.eye(12), atol=1e-11)


def test_diagonal_pattern_is_jacobi_scaling():
    A = gen.tet_lap3d(N=5)
    G = of.fsai(A, pattern="diag").toarray()
    d = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).diagonal()
    assert np.allclose(G, np.diag(1.0 / np.sqrt(d)), rtol=1e-14)


@pytest.mark.parametrize("which", ["tet", "hex"])
def test_lower_pattern_rows_satisfy_their_defining_equations(which):
    A = gen.tet_lap3d(N=6) if which == "tet" else gen.hex_elast3d(N=4, clamp_minz=True)
    perm = np.random.default_rng(5).permutation(A.n)
    G = of.fsai(A, perm)
    B = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))[perm][:, perm].toarray()
    Gd = G.toarray()
    # pattern: lower triangle of B's pattern plus the diagonal
    want = np.tril(B != 0) | np.eye(A.n, dtype=bool)
    assert np.array_equal(Gd != 0, want)
    GB = Gd @ B
    assert np.allclose(np.diag(Gd @ B @ Gd.T), 1.0, rtol=1e-12)          # unit diagonal of G B G^T
    scale = np.abs(GB).max()
    for i in range(A.n):                                                # (G B)[i, j] = 0 for j in J_i, j != i
        J = np.nonzero(want[i])[0]
        J = J[J != i]
        assert np.all(np.abs(GB[i, J]) <= 1e-12 * scale), i


def test_pcg_solves_against_lapack():
    A = gen.tet_lap3d(N=8)
    D = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    xs = np.random.default_rng(2).uniform(-1, 1, A.n)
    b = D @ xs
    G = of.fsai(A)
    x, k, rr, rz = of.pcg(A, G, b, rtol=1e-12)
    ref = np.linalg.solve(D, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(b - D @ x) <= 1e-12 * np.linalg.norm(b)
    assert k < A.n


def test_pcg_with_the_identity_is_cg():
    A = gen.tet_lap3d(N=7)
    b = oracle.spmv(A, np.random.default_rng(3).uniform(-1, 1, A.n))
    _, _, k, _, hist = oracle.cg(A, b, rtol=1e-10, history=True)
    _, kp, rr, _ = of.pcg(A, sp.identity(A.n, format="csr"), b, rtol=1e-10)
    assert kp == k
    assert np.allclose(np.sqrt(rr / rr[0]), hist, rtol=1e-9, atol=0)   # the CG oracle records ||r_k|| / ||b||


def test_fsai_cuts_iterations_on_fem_matrices():
    for A in (gen.tet_lap3d(N=12), gen.hex_elast3d(N=6, clamp_minz=True)):
        b = oracle.spmv(A, np.random.default_rng(4).uniform(-1, 1, A.n))
        _, _, k_cg, _ = oracle.cg(A, b, rtol=1e-10)
        _, k_pcg, _, _ = of.pcg(A, of.fsai(A), b, rtol=1e-10)
        assert k_pcg < 0.75 * k_cg, (A.name, k_pcg, k_cg)
