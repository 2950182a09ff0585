"""Pins for the seeded FEM generators (closed forms and invariants of the assembled operators)."""
import numpy as np
import pytest

import gen


def _sym_err(A):
    S = A.to_scipy()
    return abs(S - S.T).max()


@pytest.mark.parametrize("N", [2, 3, 7, 30])
def test_fem2d_closed_form_nnz_and_laplacian_invariants(N):
    A = gen.fem2d_p1(N=N)
    assert A.n == N * N
    assert A.nnz == N * N + 2 * (2 * N * (N - 1) + (N - 1) ** 2)
    assert _sym_err(A) == 0.0
    S = A.to_scipy()
    scale = abs(S).sum(1).max()
    # P1 Laplacian (pure Neumann): constants are in the null space ...
    assert abs(S @ np.ones(A.n)).max() <= 1e-13 * scale
    # ... and linear functions are reproduced exactly at interior nodes
    xyz = gen.coords("tri", N, 0.3, 1, 2)
    lin = S @ (2.0 * xyz[:, 0] - 3.0 * xyz[:, 1])
    # an interior node is one whose 6 neighbours exist: row length 7
    interior = np.diff(A.row_ptr) == 7
    if interior.any():
        assert abs(lin[interior]).max() <= 1e-12 * scale


def test_fem2d_full_config_size():
    A = gen.fem2d_p1()
    assert (A.n, A.nnz) == (40000, 278402)
    assert np.all(np.diff(A.row_ptr) <= 7) and np.isfinite(A.val).all()


def test_fem2d_psd_small():
    S = gen.fem2d_p1(N=9).to_scipy().toarray()
    w = np.linalg.eigvalsh(S)
    assert w.min() >= -1e-12 * w.max()
    assert abs(w.min()) <= 1e-12 * w.max()  # exactly one zero mode (constants)
    assert w[1] > 1e-6 * w.max()


@pytest.mark.parametrize("N", [2, 4, 9])
def test_hex_elasticity_closed_form_and_rigid_modes(N):
    A = gen.hex_elast3d(N=N)
    assert A.n == 3 * N ** 3 and A.nnz == 9 * (3 * N - 2) ** 3
    assert _sym_err(A) == 0.0
    S = A.to_scipy()
    scale = abs(S).sum(1).max()
    xyz = gen.coords("hex", N, 0.2, 11, 12)
    nn = N ** 3
    modes = []
    for d in range(3):
        u = np.zeros((nn, 3)); u[:, d] = 1.0; modes.append(u.ravel())
    for a, b in [(0, 1), (1, 2), (0, 2)]:
        u = np.zeros((nn, 3)); u[:, a] = -xyz[:, b]; u[:, b] = xyz[:, a]; modes.append(u.ravel())
    for m in modes:  # the six rigid-body modes are in the null space of the Neumann operator
        assert abs(S @ m).max() <= 1e-13 * scale * max(1.0, abs(m).max())


def test_hex_elasticity_psd_rank():
    S = gen.hex_elast3d(N=3).to_scipy().toarray()
    w = np.linalg.eigvalsh(S)
    assert w.min() >= -1e-12 * w.max()
    assert np.sum(np.abs(w) <= 1e-10 * w.max()) == 6  # exactly the rigid-body modes
    # clamping the min-z face removes them
    Sc = gen.hex_elast3d(N=3, clamp_minz=True).to_scipy().toarray()
    assert np.linalg.eigvalsh(Sc).min() > 1e-8


def test_hex_scalar_laplacian():
    N = 5
    A = gen.hex_lap3d(N)
    assert A.n == N ** 3 and A.nnz == (3 * N - 2) ** 3
    S = A.to_scipy()
    assert _sym_err(A) == 0.0
    assert abs(S @ np.ones(A.n)).max() <= 1e-13 * abs(S).sum(1).max()


@pytest.mark.parametrize("N", [2, 3, 6])
def test_tet_closed_form_and_invariants(N):
    A = gen.tet_lap3d(N=N, dirichlet=False)
    m = N - 1
    assert A.n == N ** 3
    assert A.nnz == N ** 3 + 2 * (3 * N * N * m + 3 * N * m * m + m ** 3)
    assert _sym_err(A) == 0.0
    S = A.to_scipy()
    scale = abs(S).sum(1).max()
    assert abs(S @ np.ones(A.n)).max() <= 1e-13 * scale
    xyz = gen.coords("tet", N, 0.2, 21, 22)
    interior = np.diff(A.row_ptr) == 15
    if interior.any():
        lin = S @ (xyz[:, 0] + 2 * xyz[:, 1] - xyz[:, 2])
        assert abs(lin[interior]).max() <= 1e-12 * scale


def test_tet_dirichlet_spd_and_nnz_kept():
    N = 5
    A = gen.tet_lap3d(N=N, dirichlet=True)
    B = gen.tet_lap3d(N=N, dirichlet=False)
    assert A.nnz == B.nnz and np.array_equal(A.col, B.col)
    S = A.to_scipy().toarray()
    assert np.allclose(S, S.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(S).min() > 0


def test_generators_deterministic_and_seeded():
    a, b = gen.hex_elast3d(N=5), gen.hex_elast3d(N=5)
    assert np.array_equal(a.val.view(np.int64), b.val.view(np.int64)) and np.array_equal(a.col, b.col)
    c = gen.hex_elast3d(N=5, seed_perm=99)
    assert not np.array_equal(a.col, c.col)
    x1, x2 = gen.uniform(1000, 3), gen.uniform(1000, 3)
    assert np.array_equal(x1, x2) and x1.min() >= -1 and x1.max() < 1
    assert abs(x1.mean()) < 0.1
    p = gen.permutation(1000, 7)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_random_csr_shapes():
    A = gen.random_csr(300, 5, mean_row=6, int_values=True, empty_frac=0.1, long_rows=3, long_len=200,
                       duplicates=True)
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.col.size == A.val.size
    assert (np.diff(A.row_ptr) == 0).any() and np.diff(A.row_ptr).max() >= 150
    assert A.col.min() >= 0 and A.col.max() < A.n
    assert np.all(A.val == np.round(A.val))
