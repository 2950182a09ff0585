"""Pins of the oracle's flexible CG (oracle/fcg.py) against cases the mathematics fixes: the identity
preconditioner gives CG's residuals, a fixed SPD preconditioner gives preconditioned CG's iterates, the
exact inverse solves in one step, and a preconditioner that changes every step (an inexact inner solve on
perturbed values) still reaches 1e-10."""
import numpy as np
import pytest

import gen
import oracle
from oracle import fcg as of


def _spd():
    return gen.tet_lap3d(N=9)      # Dirichlet P1 Laplacian on a jittered tet mesh: SPD, n = 729


def _dense(A):
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    np.add.at(D, (rows, A.col), A.val)
    return D


def test_identity_preconditioner_gives_cg():
    A = _spd()
    b = gen.uniform(A.n, 5)
    _, ok, steps, rel, hist = of.fcg(A, b, lambda r, k: r, rtol=1e-10, max_steps=400, history=True)
    _, ok_cg, it_cg, rel_cg, hist_cg = oracle.cg(A, b, rtol=1e-10, max_iter=400, history=True)
    assert ok and ok_cg and abs(steps - it_cg) <= 1
    m = min(25, steps, it_cg)
    # CG's history holds ||r_k|| / ||b|| (= ||r_0|| from x_0 = 0); the first tens of norms agree to rounding
    assert np.allclose(np.asarray(hist[:m]) / hist[0], hist_cg[:m], rtol=1e-8)


def test_fixed_spd_preconditioner_gives_pcg_iterates():
    A = _spd()
    b = gen.uniform(A.n, 6)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    diag = np.zeros(A.n)
    np.add.at(diag, rows[A.col == rows], A.val[A.col == rows])
    jac = lambda r: r / diag                                               # Jacobi: fixed and SPD
    xs = of.pcg(A, b, jac, rtol=0.0, max_steps=12)
    for k in (1, 2, 5, 12):
        x, *_ = of.fcg(A, b, lambda r, j: jac(r), rtol=0.0, max_steps=k)
        assert np.linalg.norm(x - xs[k]) <= 1e-10 * np.linalg.norm(xs[k]), k


def test_exact_inverse_solves_in_one_step():
    A = _spd()
    b = gen.uniform(A.n, 7)
    D = _dense(A)
    x, ok, steps, rel = of.fcg(A, b, lambda r, k: np.linalg.solve(D, r), rtol=1e-12, max_steps=5)
    assert ok and steps == 1 and rel <= 1e-12


def test_variable_inexact_preconditioner_converges():
    # B_k: a few CG steps (3 + k mod 4 of them) on the values cut to BF16 precision (8 significant bits) -- a
    # different operator every step
    A = _spd()
    b = gen.uniform(A.n, 8)
    cut = (A.val.astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    low = gen.CSR(A.n, A.row_ptr, A.col, cut)

    def inner(r, k):
        x, *_ = oracle.cg(low, r, rtol=0.0, max_iter=3 + k % 4)
        return x
    x, ok, steps, rel = of.fcg(A, b, inner, rtol=1e-10, max_steps=500)
    assert ok and rel <= 1e-10
    # and it needs fewer outer steps than plain CG needs iterations
    _, _, it_cg, _ = oracle.cg(A, b, rtol=1e-10, max_iter=2000)
    assert steps < it_cg
