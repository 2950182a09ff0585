"""FSAI preconditioner and preconditioned CG -- oracle, TEST INFRASTRUCTURE ONLY.

The paper motivates EHYB with iterative solvers whose preconditioner is applied as a further sparse
product (Sec. 6: approximate-inverse preconditioners).  The preconditioner here is the factorized sparse
approximate inverse (FSAI) of an SPD matrix A (Kolotilina and Yeremin): a lower-triangular G with a
prescribed pattern, row i restricted to the column set J_i (all j <= i of the pattern, i itself included),

    g_i = A[J_i, J_i]^{-1} e_i / sqrt((A[J_i, J_i]^{-1})_{ii}),

so that (G A G^T)_{ii} = 1 and row i of G A vanishes on J_i \\ {i}.  The preconditioner is M^{-1} = G^T G.

``fsai(A, new_to_old, pattern)`` builds G for B = P A P^T (B[r, s] = A[new_to_old[r], new_to_old[s]]);
pattern "lower" (the lower triangle of B's pattern, the default), "diag" (only the diagonal: Jacobi
scaling) or "full" (every j <= i: the inverse Cholesky factor).  Dense blocks come from scipy.sparse
slicing, solves from numpy.linalg.solve.

``pcg(A, G, b, ...)`` is textbook preconditioned CG (Saad, Alg. 9.1) with M^{-1} r = G^T (G r), stopping on
||r_k|| <= rtol ||b||.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _scipy(A):
    return sp.csr_matrix((np.asarray(A.val, float), np.asarray(A.col, np.int64), np.asarray(A.row_ptr, np.int64)),
                         shape=(A.n, A.n))


def fsai(A, new_to_old=None, pattern: str = "lower") -> sp.csr_matrix:
    n = A.n
    perm = np.arange(n) if new_to_old is None else np.asarray(new_to_old, np.int64)
    B = _scipy(A)[perm][:, perm].tocsr()
    B.sum_duplicates()
    B.sort_indices()
    rows, cols, vals = [], [], []
    for i in range(n):
        if pattern == "diag":
            J = np.array([i])
        elif pattern == "full":
            J = np.arange(i + 1)
        else:
            row = B.indices[B.indptr[i]:B.indptr[i + 1]]
            J = np.union1d(row[row <= i], [i])
        Bj = B[J][:, J].toarray()
        e = np.zeros(len(J))
        e[-1] = 1.0                      # i is the largest index of J_i
        g = np.linalg.solve(Bj, e)
        g = g / np.sqrt(g[-1])
        rows.append(np.full(len(J), i))
        cols.append(J)
        vals.append(g)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def pcg(A, G, b, x0=None, rtol: float = 1e-10, max_iter: int = 10000):
    """Returns (x, iterations, rr_history, rz_history): r.r and r.z of iterations 0..k."""
    M = _scipy(A)
    G = sp.csr_matrix(G)
    GT = G.T.tocsr()
    x = np.zeros(A.n) if x0 is None else np.array(x0, float)
    r = b - M @ x
    z = GT @ (G @ r)
    p = z.copy()
    rz = float(r @ z)
    rr_hist, rz_hist = [float(r @ r)], [rz]
    tol2 = (rtol * np.linalg.norm(b)) ** 2
    k = 0
    while k < max_iter and rr_hist[-1] > tol2:
        q = M @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        rr_hist.append(float(r @ r))
        if rr_hist[-1] <= tol2:
            break
        z = GT @ (G @ r)
        rz_new = float(r @ z)
        rz_hist.append(rz_new)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, k, np.array(rr_hist), np.array(rz_hist)
