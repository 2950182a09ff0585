"""CPU oracle for the EHYB SpMV library -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2204_06666_gb300``): it is a plain, slow, FP64 statement of what the
path computes, checked in ``tests/test_oracle_*.py`` against values fixed by
mathematics (dense brute force, closed forms, exact integer arithmetic,
LAPACK, finite differences), never against the CUDA path.

Contents
  * ``spmv``, ``spmm``, ``cg``, ``cg_refined``, ``spmv_low`` -- ctypes wrappers of
    ``oracle.c`` (plain FP64 C, no FMA contraction).
  * ``mlp``     -- FP64 forward/backward/Adam of the tuner's 16-64-64-4 MLP.
  * ``fsai``    -- the FSAI preconditioner (per-row dense solves) and textbook preconditioned CG.
  * ``ehyb_format`` -- an independent decoder of the EHYB plan arrays back to
    (row, col, val) triplets, the Eq. 1 / Eq. 2 cache-size rule, the Sec. 3.4
    footprint byte model and the per-row rounding-error bound used by parity tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2 -ffp-contract=off) into liboracle.so."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, dbl, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        lib.oracle_spmv_csr.argtypes = [i64, p, p, p, p, p]
        lib.oracle_spmv_csr_rows.argtypes = [i64, i64, p, p, p, p, p]
        lib.oracle_spmm_csr.argtypes = [i64, i32, p, p, p, p, p]
        lib.oracle_cg.argtypes = [i64, p, p, p, p, p, dbl, i32, p, p, p]
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_spmv_low.argtypes = [i64, p, p, p, i32, p, p]
        lib.oracle_cg_refined.argtypes = [i64, p, p, p, i32, p, p, dbl, dbl, i32, i32, p, p, p]
        lib.oracle_cg_refined.restype = ctypes.c_int
        _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def spmv(A, x) -> np.ndarray:
    """y = A x, y_i = sum_k val_k x[col_k] over row i in storage order (FP64)."""
    rp, prp = _c(A.row_ptr, np.int64)
    c, pc = _c(A.col, np.int32)
    v, pv = _c(A.val, np.float64)
    xx, px = _c(x, np.float64)
    y = np.zeros(A.n, np.float64)
    _load().oracle_spmv_csr(A.n, prp, pc, pv, px, y.ctypes.data)
    return y


def spmv_rows(A, x, r0: int, r1: int, y: np.ndarray) -> None:
    """Rows [r0, r1) of y = A x into y (the CPU-baseline sample)."""
    _load().oracle_spmv_csr_rows(r0, r1, A.row_ptr.ctypes.data, A.col.ctypes.data, A.val.ctypes.data,
                                 x.ctypes.data, y.ctypes.data)


def spmm(A, X) -> np.ndarray:
    """Y = A X, X row-major (n x k)."""
    X, pX = _c(X, np.float64)
    k = X.shape[1]
    Y = np.zeros((A.n, k), np.float64)
    _load().oracle_spmm_csr(A.n, k, A.row_ptr.ctypes.data, A.col.ctypes.data, A.val.ctypes.data, pX, Y.ctypes.data)
    return Y


def spmv_low(A, x, bf16: bool) -> np.ndarray:
    """y = A_low x_f32 in float arithmetic, values rounded to FP32 (or BF16 when bf16)."""
    xx, px = _c(x, np.float64)
    y = np.zeros(A.n, np.float64)
    _load().oracle_spmv_low(A.n, A.row_ptr.ctypes.data, A.col.ctypes.data, A.val.ctypes.data, int(bf16), px,
                            y.ctypes.data)
    return y


def cg(A, b, x0=None, rtol: float = 1e-10, max_iter: int = 10000, history: bool = False):
    """Textbook CG.  Returns (x, converged, iters, true_relres[, hist])."""
    b, pb = _c(b, np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, np.float64, copy=True)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    hist = np.zeros(max_iter + 1) if history else None
    st = _load().oracle_cg(A.n, A.row_ptr.ctypes.data, A.col.ctypes.data, A.val.ctypes.data, pb, x.ctypes.data,
                           rtol, max_iter, ctypes.byref(it), ctypes.byref(rel),
                           hist.ctypes.data if history else None)
    out = (x, st == 0, it.value, rel.value)
    if history:
        out = out + (hist[: it.value + 1],)
    return out


def cg_refined(A, b, bf16: bool, rtol: float = 1e-10, inner_rtol: float = 1e-4, inner_max: int = 5000,
               outer_max: int = 50):
    """Mixed-precision iterative refinement.  Returns (x, converged, outer, inner_total, relres)."""
    b, pb = _c(b, np.float64)
    x = np.zeros(A.n)
    o, it, rel = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    st = _load().oracle_cg_refined(A.n, A.row_ptr.ctypes.data, A.col.ctypes.data, A.val.ctypes.data, int(bf16), pb,
                                   x.ctypes.data, rtol, inner_rtol, inner_max, outer_max, ctypes.byref(o),
                                   ctypes.byref(it), ctypes.byref(rel))
    return x, st == 0, o.value, it.value, rel.value


def abs_spmv(A, x) -> np.ndarray:
    """(|A| |x|)_i, the scale of the rounding-error bound."""
    return spmv(type(A)(A.n, A.row_ptr, A.col, np.abs(A.val)), np.abs(x))


def gamma(k, u: float = 2.0 ** -53):
    """gamma_k = k u / (1 - k u): the classical bound on recursive-summation error (Higham, Thm 3.1)."""
    k = np.asarray(k, np.float64)
    return k * u / (1.0 - k * u)
