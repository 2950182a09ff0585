"""Flexible conjugate gradients -- TEST INFRASTRUCTURE ONLY.

Notay's flexible CG ("Flexible conjugate gradients", SIAM J. Sci. Comput. 22 (2000) 1444-1460) with one
kept direction: a CG whose preconditioner may change from step to step (here: an inner iterative solve in
lower precision, the mixed-precision use of the SpMV that Sec. 6 of the EHYB paper motivates).  Step k:

    z_k = B_k(r_k)
    p_k = z_k - (z_k . A p_{k-1}) / (p_{k-1} . A p_{k-1}) p_{k-1}     (p_0 = z_0)
    alpha_k = (p_k . r_k) / (p_k . A p_k)
    x_{k+1} = x_k + alpha_k p_k,   r_{k+1} = r_k - alpha_k A p_k

With a fixed SPD B the iterates are those of preconditioned CG; with B = I those of CG; with B = A^-1 the
first step solves the system.  These three cases are the pins (tests/test_oracle_fcg.py).  Plain numpy in
FP64; the products A p use the oracle's C SpMV.
"""
from __future__ import annotations

import numpy as np


def fcg(A, b, apply_b, x0=None, rtol: float = 1e-10, max_steps: int = 1000, history: bool = False):
    """Solve A x = b.  apply_b(r, k) returns z_k.  Stops when ||r_k|| <= rtol ||b||.

    Returns (x, converged, steps, true_relres[, list of ||r_k||])."""
    from oracle import spmv
    b = np.asarray(b, np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, np.float64, copy=True)
    r = b - spmv(A, x)
    bnorm = np.linalg.norm(b) or 1.0
    p = q = None
    hist = [float(np.linalg.norm(r))]
    k = 0
    while hist[-1] > rtol * bnorm and k < max_steps:
        z = np.asarray(apply_b(r.copy(), k), np.float64)
        if p is None:
            p = z
        else:
            p = z - (z @ q) / (p @ q) * p
        q = spmv(A, p)
        alpha = (p @ r) / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        hist.append(float(np.linalg.norm(r)))
    rel = float(np.linalg.norm(b - spmv(A, x)) / bnorm)
    out = (x, hist[-1] <= rtol * bnorm, k, rel)
    return out + (hist,) if history else out


def pcg(A, b, apply_minv, x0=None, rtol: float = 1e-10, max_steps: int = 1000):
    """Textbook preconditioned CG (Hestenes-Stiefel with z = M^-1 r, beta = (r.z)_new / (r.z)_old): the
    reference the fixed-preconditioner pin compares flexible CG with.  Returns the list of iterates."""
    from oracle import spmv
    b = np.asarray(b, np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, np.float64, copy=True)
    r = b - spmv(A, x)
    z = apply_minv(r)
    p = z.copy()
    rz = r @ z
    xs = [x.copy()]
    for _ in range(max_steps):
        if np.linalg.norm(r) <= rtol * np.linalg.norm(b):
            break
        q = spmv(A, p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        xs.append(x.copy())
        z = apply_minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return xs
