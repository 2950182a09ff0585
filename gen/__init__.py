"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no EHYB arithmetic: it only builds matrices A (CSR) and
vectors x with the shapes of the paper's workloads (Sec. 5: unstructured-mesh
FEM matrices from structural, CFD and electromagnetic problems), plus small
random CSR matrices for edge cases.  The FEM families are assembled by
``gen.c`` (compiled to ``libgen.so`` on first use or by ``__graft_entry__.build``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgen.so")
_SRC = os.path.join(_HERE, "gen.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so (plain C, no FMA contraction: identical bits on x86-64 and aarch64)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, u64, dbl, p = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.gen_uniform.argtypes = [i64, u64, dbl, dbl, p]
        lib.gen_permutation.argtypes = [i64, u64, p]
        lib.gen_fem2d_p1_nnz.argtypes = [i32]
        lib.gen_fem2d_p1_nnz.restype = i64
        lib.gen_hex_nnz.argtypes = [i32, i32]
        lib.gen_hex_nnz.restype = i64
        lib.gen_tet_lap3d_nnz.argtypes = [i32]
        lib.gen_tet_lap3d_nnz.restype = i64
        lib.gen_fem2d_p1.argtypes = [i32, dbl, u64, u64, p, p, p]
        lib.gen_hex3d.argtypes = [i32, i32, dbl, dbl, dbl, u64, u64, i32, p, p, p]
        lib.gen_tet_lap3d.argtypes = [i32, dbl, u64, u64, i32, p, p, p]
        lib.gen_coords.argtypes = [i32, i32, dbl, u64, u64, i32, p]
        _lib = lib
    return _lib


@dataclass
class CSR:
    """Square sparse matrix in CSR: row_ptr int64[n+1], col int32[nnz], val float64[nnz]."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def _alloc(n: int, nnz: int):
    return (np.zeros(n + 1, np.int64), np.zeros(nnz, np.int32), np.zeros(nnz, np.float64))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform vector in [lo, hi) (counter-based splitmix64 stream)."""
    out = np.empty(n, np.float64)
    _load().gen_uniform(n, seed, lo, hi, _ptr(out))
    return out


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded Fisher-Yates permutation: perm[old] = new."""
    out = np.empty(n, np.int32)
    _load().gen_permutation(n, seed, _ptr(out))
    return out


def fem2d_p1(N: int = 200, jitter: float = 0.3, seed_mesh: int = 1, seed_perm: int = 2) -> CSR:
    """2D P1 Laplacian on an N x N jittered node grid, diagonal split, random node relabelling."""
    lib = _load()
    n, nnz = N * N, lib.gen_fem2d_p1_nnz(N)
    rp, c, v = _alloc(n, nnz)
    if lib.gen_fem2d_p1(N, jitter, seed_mesh, seed_perm, _ptr(rp), _ptr(c), _ptr(v)) != 0:
        raise RuntimeError("gen_fem2d_p1 failed")
    return CSR(n, rp, c, v, f"fem2d_p1_N{N}")


def hex_elast3d(N: int = 70, jitter: float = 0.2, seed_mesh: int = 11, seed_perm: int = 12,
                clamp_minz: bool = False, E: float = 1.0, nu: float = 0.3) -> CSR:
    """3D Q1 hexahedral isotropic elasticity (3 dof/node) on an N^3 jittered grid, node relabelling."""
    lib = _load()
    n, nnz = 3 * N ** 3, lib.gen_hex_nnz(N, 3)
    rp, c, v = _alloc(n, nnz)
    if lib.gen_hex3d(N, 3, jitter, E, nu, seed_mesh, seed_perm, int(clamp_minz), _ptr(rp), _ptr(c), _ptr(v)) != 0:
        raise RuntimeError("gen_hex3d failed")
    return CSR(n, rp, c, v, f"hex_elast3d_N{N}" + ("_clamped" if clamp_minz else ""))


def hex_lap3d(N: int, jitter: float = 0.2, seed_mesh: int = 41, seed_perm: int = 42) -> CSR:
    """3D Q1 hexahedral scalar Laplacian (27-point pattern) on an N^3 jittered grid."""
    lib = _load()
    n, nnz = N ** 3, lib.gen_hex_nnz(N, 1)
    rp, c, v = _alloc(n, nnz)
    if lib.gen_hex3d(N, 1, jitter, 1.0, 0.0, seed_mesh, seed_perm, 0, _ptr(rp), _ptr(c), _ptr(v)) != 0:
        raise RuntimeError("gen_hex3d failed")
    return CSR(n, rp, c, v, f"hex_lap3d_N{N}")


def tet_lap3d(N: int = 126, jitter: float = 0.2, seed_mesh: int = 21, seed_perm: int = 22,
              dirichlet: bool = True) -> CSR:
    """3D P1 Laplacian on the Freudenthal 6-tet split of an N^3 jittered grid."""
    lib = _load()
    n, nnz = N ** 3, lib.gen_tet_lap3d_nnz(N)
    rp, c, v = _alloc(n, nnz)
    if lib.gen_tet_lap3d(N, jitter, seed_mesh, seed_perm, int(dirichlet), _ptr(rp), _ptr(c), _ptr(v)) != 0:
        raise RuntimeError("gen_tet_lap3d failed")
    return CSR(n, rp, c, v, f"tet_lap3d_N{N}" + ("_dirichlet" if dirichlet else ""))


def shifted(A: CSR, c: float) -> CSR:
    """A + c I for a matrix whose every row stores its diagonal entry (the implicit-Euler operator
    M/dt + K with a lumped mass M = (c dt) I); the pattern is unchanged."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.row_ptr))
    diag = A.col.astype(np.int64) == rows
    if np.count_nonzero(diag) != A.n or np.any(np.bincount(rows[diag], minlength=A.n) != 1):
        raise ValueError("every row needs exactly one stored diagonal entry")
    val = A.val.copy()
    val[diag] += c
    return CSR(A.n, A.row_ptr.copy(), A.col.copy(), val, A.name + f"_shift{c:g}")


def scaled_identity(n: int, c: float) -> CSR:
    """c I as a CSR matrix (one entry per row)."""
    return CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.full(n, float(c)), f"I_{c:g}")


def coords(kind: str, N: int, jitter: float, seed_mesh: int, seed_perm: int) -> np.ndarray:
    """Jittered node coordinates (nodes x 3) indexed by the relabelled node number."""
    dim, k = {"tri": (2, 0), "tet": (3, 1), "hex": (3, 2)}[kind]
    nn = N ** dim
    out = np.zeros((nn, 3), np.float64)
    if _load().gen_coords(dim, N, jitter, seed_mesh, seed_perm, k, _ptr(out)) != 0:
        raise RuntimeError("gen_coords failed")
    return out


def random_csr(n: int, seed: int, mean_row: float = 8.0, int_values: bool = False, empty_frac: float = 0.0,
               long_rows: int = 0, long_len: int = 0, local_frac: float = 0.7, window: int = 64,
               duplicates: bool = False, symmetric: bool = False) -> CSR:
    """Small random square CSR for edge cases: ragged rows, empty rows, a few very long
    rows, mostly-local columns in a hidden order, optional duplicate entries, and either
    small integer values in [-8, 8] or uniform values in [-1, 1)."""
    rng = np.random.default_rng(seed)
    hidden = rng.permutation(n)
    pos = np.empty(n, np.int64)
    pos[hidden] = np.arange(n)
    lens = rng.poisson(mean_row, n).astype(np.int64)
    if empty_frac > 0:
        lens[rng.random(n) < empty_frac] = 0
    if long_rows > 0 and n > 0:
        lens[rng.choice(n, size=min(long_rows, n), replace=False)] = long_len
    rows, cols = [], []
    for i in range(n):
        k = int(lens[i])
        if k == 0:
            continue
        loc = rng.random(k) < local_frac
        c = np.where(loc, hidden[np.clip(pos[i] + rng.integers(-window, window + 1, k), 0, n - 1)],
                     rng.integers(0, n, k))
        if not duplicates:
            c = np.unique(c)
        rows.append(np.full(c.size, i, np.int64))
        cols.append(c.astype(np.int64))
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    if symmetric:
        r, c = np.concatenate([r, c]), np.concatenate([c, r])
        key = np.unique(r * n + c)
        r, c = key // n, key % n
    if int_values:
        v = rng.integers(-8, 9, r.size).astype(np.float64)
    else:
        v = rng.uniform(-1.0, 1.0, r.size)
    if symmetric:
        lo = np.minimum(r, c) * n + np.maximum(r, c)
        _, inv = np.unique(lo, return_inverse=True)
        base = rng.integers(-8, 9, inv.max() + 1).astype(np.float64) if int_values else rng.uniform(-1, 1, inv.max() + 1)
        v = base[inv] if r.size else v
    order = np.lexsort((rng.random(r.size), r))  # row-major; columns unsorted within a row
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr, c.astype(np.int32), v.astype(np.float64), f"random_n{n}_s{seed}")


def int_vector(n: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Small-integer vector (exact in every precision the path uses)."""
    return np.random.default_rng(seed).integers(lo, hi + 1, n).astype(np.float64)


BATCH_KINDS = ("fem2d_p1", "tet_lap3d", "hex_lap3d", "hex_elast3d")


def fem_batch(count: int = 64, seed: int = 31, n_min: int = 5000, n_max: int = 300000):
    """`count` FEM matrices with row counts log-uniform in [n_min, n_max] and a kind drawn uniformly among
    2D P1 (7/row), 3D P1 tet (15/row), 3D Q1 scalar hex (27/row) and 3D Q1 hex elasticity (81/row);
    each jittered and relabelled with its own seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        kind = BATCH_KINDS[int(rng.integers(0, 4))]
        s_mesh, s_perm = 1000 + 2 * i + 10000 * seed, 1001 + 2 * i + 10000 * seed
        if kind == "fem2d_p1":
            A = fem2d_p1(N=max(2, int(round(n ** 0.5))), seed_mesh=s_mesh, seed_perm=s_perm)
        elif kind == "tet_lap3d":
            A = tet_lap3d(N=max(2, int(round(n ** (1 / 3)))), seed_mesh=s_mesh, seed_perm=s_perm, dirichlet=False)
        elif kind == "hex_lap3d":
            A = hex_lap3d(N=max(2, int(round(n ** (1 / 3)))), seed_mesh=s_mesh, seed_perm=s_perm)
        else:
            A = hex_elast3d(N=max(2, int(round((n / 3) ** (1 / 3)))), seed_mesh=s_mesh, seed_perm=s_perm)
        out.append(A)
    return out


def powerlaw_csr(n: int, seed: int, alpha: float, min_len: int = 2, max_len: int = 5000, local_frac: float = 0.7,
                 symmetric: bool = True) -> CSR:
    """Random sparse matrix with power-law row lengths, to stress the extra-row tail.

    Row lengths follow P(k) ~ k^-alpha on [min_len, max_len]; 70 % of each row's columns fall in a window of
    +-max(32, k) around the row in a hidden order (locality a partitioner can find), 30 % are uniform.  The
    pattern is symmetrised and given a diagonal; values are symmetric U[-1, 1) off the diagonal and the
    diagonal is 1 + the row's absolute off-diagonal sum (so the matrix is SPD).  The row order is random.
    """
    rng = np.random.default_rng(seed)
    ks = np.arange(min_len, max_len + 1, dtype=np.float64)
    pk = ks ** (-alpha)
    lens = rng.choice(np.arange(min_len, max_len + 1), size=n, p=pk / pk.sum())
    hidden = rng.permutation(n)            # hidden[pos] = row at that position
    pos = np.empty(n, np.int64)
    pos[hidden] = np.arange(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    total = rows.size
    win = np.maximum(32, lens)[rows]
    off = np.floor((rng.random(total) * 2.0 - 1.0) * (win + 1)).astype(np.int64)
    loc_cols = hidden[np.clip(pos[rows] + off, 0, n - 1)]
    cols = np.where(rng.random(total) < local_frac, loc_cols, rng.integers(0, n, total))
    if symmetric:
        rows, cols = np.concatenate([rows, cols]), np.concatenate([cols, rows])
    key = np.unique(rows * n + cols)
    r, c = key // n, key % n
    off_mask = r != c
    r, c = r[off_mask], c[off_mask]
    lo, hi = np.minimum(r, c), np.maximum(r, c)
    with np.errstate(over="ignore"):
        h = (lo.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15) + hi.astype(np.uint64) * np.uint64(0xBF58476D1CE4E5B9)
             + np.uint64(seed)) >> np.uint64(11)
    v = (h.astype(np.float64) / float(1 << 53)) * 2.0 - 1.0   # symmetric value per unordered pair
    diag = np.bincount(r, weights=np.abs(v), minlength=n) + 1.0
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, diag])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return CSR(n, np.cumsum(rp), c.astype(np.int32), v, f"powerlaw_n{n}_a{alpha:.2f}")


def tuner_matrix(index: int, base_seed: int = 1000, n_min: int = 5000, n_max: int = 300000) -> CSR:
    """Matrix number `index` of the tuner's data set: even indices are FEM-like (the four element kinds of
    fem_batch), odd ones power-law (alpha ~ U[2, 3]); rows log-uniform in [n_min, n_max]; seed base + index."""
    seed = base_seed + index
    rng = np.random.default_rng(seed)
    n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
    if index % 2 == 1:
        return powerlaw_csr(int(n), seed, float(rng.uniform(2.0, 3.0)))
    kind = BATCH_KINDS[int(rng.integers(0, 4))]
    sm, sp = 2 * seed + 1, 2 * seed + 2
    if kind == "fem2d_p1":
        return fem2d_p1(N=max(2, int(round(n ** 0.5))), seed_mesh=sm, seed_perm=sp)
    if kind == "tet_lap3d":
        return tet_lap3d(N=max(2, int(round(n ** (1 / 3)))), seed_mesh=sm, seed_perm=sp, dirichlet=False)
    if kind == "hex_lap3d":
        return hex_lap3d(N=max(2, int(round(n ** (1 / 3)))), seed_mesh=sm, seed_perm=sp)
    return hex_elast3d(N=max(2, int(round((n / 3) ** (1 / 3)))), seed_mesh=sm, seed_perm=sp)
