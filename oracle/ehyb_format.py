"""Independent checks of the EHYB format -- TEST INFRASTRUCTURE ONLY.

Nothing here builds a plan.  It reads the arrays a plan exports and states, from
the paper's definitions, what they must mean:

* ``decode`` rebuilds the (row, col, val) triplets of A in the ORIGINAL index
  space from the sliced-ELL part (Sec. 3.2, Alg. 2: entries whose row and column
  lie in the same partition, 32-lane slices, 16-bit column offsets into the
  partition's cached slice of x, Sec. 3.4) and from the extra-rows (ER) part
  (entries outside the partition, each ER line mapped back to its row by yIdxER,
  Sec. 3.2).  Every stored entry must come back exactly once.
* ``slot_index`` states where slot k of a lane sits in a slice (the library's slot
  layout, see below).
* ``eq1`` is the cache-size rule of Eq. 1 and Eq. 2 (Sec. 3.3).
* ``ell_bytes_per_entry`` is the Sec. 3.4 footprint model (value + column index).

Plan-array names follow the paper: partBoundary -> ``part_ptr``, PositionELL ->
``slice_pos``, ColELL -> ``ell_col``, ValELL -> ``ell_val``, yIdxER -> ``er_row``,
ReorderTable (old -> new) is the inverse of ``new_to_old``.
"""
from __future__ import annotations

import math

import numpy as np


def eq1(n: int, tau: int, P: int, shm_max: int, max_local: int = 1 << 16):
    """Eq. 1: the smallest integer K >= 1 with n*tau/(K*P) < SHM_max; Eq. 2: VecSize = n/(K*P),
    rounded up to whole rows.  The 16-bit column offset additionally needs VecSize <= 2^16.
    Returns (K, VecSize)."""
    if n <= 0:
        return 1, 0
    K = 1
    while not (n * tau / (K * P) < shm_max and math.ceil(n / (K * P)) <= max_local):
        K += 1
    return K, math.ceil(n / (K * P))


def ell_bytes_per_entry(tau: int, index_bytes: int) -> int:
    """Bytes one ELL entry occupies: a value of tau bytes plus a column index."""
    return tau + index_bytes


GROUP = 4   # slots of one lane kept together in the runs layout of the low-precision copies


def slot_index(base: int, width: int, k: int, lane: int, group: int = 1) -> int:
    """Storage index of slot k (0 <= k < width) of lane `lane` in a 32-lane slice of `width` slots per lane that
    starts at `base`.  Alg. 2 stores slot k of every lane side by side (column-major: base + 32 k + lane); that
    is group 1, the layout of the FP64 arrays.  In group 4 (the library's FP32 / BF16 copies in runs of four)
    only the last width mod 4 slots keep that order; before them, each lane's slots come in runs of 4
    consecutive slots (one vector load), the 32 lanes' runs for slots 4q..4q+3 side by side:
    base + 128 q + 4 lane + (k - 4 q).  Either way [base, base + 32 width) is filled exactly once."""
    grouped = width - width % GROUP if group == GROUP else 0
    if k < grouped:
        q, r = divmod(k, GROUP)
        return base + 32 * GROUP * q + GROUP * lane + r
    return base + 32 * k + lane


def low_values(ex: dict) -> dict:
    """The exported plan with its low-precision copy in place of the FP64 arrays (values widened to FP64,
    BF16 bits as the FP32 value with those upper 16 bits), for decode(..., group=ex["lowp_group"])."""
    q = dict(ex)

    def wide(v):
        v = np.asarray(v)
        if v.dtype == np.uint16:
            v = (v.astype(np.uint32) << 16).view(np.float32)
        return v.astype(np.float64)
    q["ell_val"], q["ell_col"] = wide(ex["ell_val_low"]), np.asarray(ex["ell_col_low"], np.uint16)
    q["er_sval"], q["er_scol"] = wide(ex["er_sval_low"]), np.asarray(ex["er_scol_low"])
    return q


def decode(ex: dict, group: int = 1):
    """Triplets (rows, cols, vals) in the original numbering, ELL entries first then ER; `group` is the slot
    layout of the arrays (slot_index).

    ``ex`` holds the exported plan arrays: n, tpr (lanes per row in a slice), new_to_old,
    part_ptr, slice_ptr, slice_pos, ell_col (uint16), ell_val, row_ell_count (per new row), and the
    extra rows either as CSR lines (er_layout 1: er_row, er_ptr, er_col, er_val), sliced like the
    slab (er_layout 0: er_slice_pos, er_scol, er_sval, row_er_count), or in the slab slices right after
    each row's own entries (er_layout 2: row_er_count, halo_ptr, halo_new), where a 16-bit column past
    the partition's rows names entry (column - rows) of the partition's halo list.
    """
    n = int(ex["n"])
    tpr = int(ex["tpr"])
    rps = 32 // tpr                       # rows per 32-lane slice
    n2o = np.asarray(ex["new_to_old"], np.int64)
    part_ptr = np.asarray(ex["part_ptr"], np.int64)
    slice_ptr = np.asarray(ex["slice_ptr"], np.int64)
    slice_pos = np.asarray(ex["slice_pos"], np.int64)
    ell_col = np.asarray(ex["ell_col"])
    ell_val = np.asarray(ex["ell_val"])
    cnt = np.asarray(ex["row_ell_count"], np.int64)
    assert ell_col.dtype == np.uint16
    layout = int(ex.get("er_layout", 1))
    if layout == 2:                       # the extra entries follow each row's own in the slab slots
        extra = np.asarray(ex["row_er_count"], np.int64)
        halo_ptr = np.asarray(ex["halo_ptr"], np.int64)
        halo_new = np.asarray(ex["halo_new"], np.int64)
    else:
        extra = np.zeros(n, np.int64)
    rows, cols, vals = [], [], []
    for p in range(len(part_ptr) - 1):
        pb, pe = part_ptr[p], part_ptr[p + 1]
        for s in range(slice_ptr[p], slice_ptr[p + 1]):
            pos = slice_pos[s]
            width = (slice_pos[s + 1] - pos) // 32
            assert (slice_pos[s + 1] - pos) % 32 == 0
            for lane in range(32):
                row = pb + (s - slice_ptr[p]) * rps + lane // tpr
                if row >= pe:
                    continue
                sub = lane % tpr
                for k in range(width):
                    j = k * tpr + sub          # entry j of this row's slots (its ELL entries, then any extra)
                    if j >= cnt[row] + extra[row]:
                        continue
                    e = slot_index(pos, width, k, lane, group)
                    local = int(ell_col[e])
                    if pb + local < pe:
                        col = pb + local
                    else:
                        assert j >= cnt[row], "ELL column outside its partition"
                        h = local - (pe - pb)
                        assert halo_ptr[p] + h < halo_ptr[p + 1], "halo column past the partition's halo"
                        col = halo_new[halo_ptr[p] + h]
                        assert not (pb <= col < pe), "halo entry inside its own partition"
                    rows.append(n2o[row])
                    cols.append(n2o[col])
                    vals.append(ell_val[e])
    if layout == 2:
        pass
    elif layout == 0:
        # extra entries stored in the slab's own slices: same lane -> row map, 32-bit new columns
        er_pos = np.asarray(ex["er_slice_pos"], np.int64)
        er_col = np.asarray(ex["er_scol"], np.int64)
        er_val = np.asarray(ex["er_sval"])
        ecnt = np.asarray(ex["row_er_count"], np.int64)
        for p in range(len(part_ptr) - 1):
            pb, pe = part_ptr[p], part_ptr[p + 1]
            for s in range(slice_ptr[p], slice_ptr[p + 1]):
                width = (er_pos[s + 1] - er_pos[s]) // 32
                for lane in range(32):
                    row = pb + (s - slice_ptr[p]) * rps + lane // tpr
                    if row >= pe:
                        continue
                    for k in range(width):
                        j = k * tpr + lane % tpr
                        if j >= ecnt[row]:
                            continue
                        e = slot_index(er_pos[s], width, k, lane, group)
                        rows.append(n2o[row])
                        cols.append(n2o[er_col[e]])
                        vals.append(er_val[e])
    else:
        er_row = np.asarray(ex["er_row"], np.int64)
        er_ptr = np.asarray(ex["er_ptr"], np.int64)
        er_col = np.asarray(ex["er_col"], np.int64)
        er_val = np.asarray(ex["er_val"])
        for i in range(len(er_row)):
            for k in range(er_ptr[i], er_ptr[i + 1]):
                rows.append(n2o[er_row[i]])
                cols.append(n2o[er_col[k]])
                vals.append(er_val[k])
    return (np.asarray(rows, np.int64), np.asarray(cols, np.int64), np.asarray(vals, np.float64))


def triplets(A):
    """(rows, cols, vals) of a CSR matrix in storage order."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.row_ptr))
    return rows, A.col.astype(np.int64), A.val.astype(np.float64)


def same_multiset(a, b) -> bool:
    """True when two triplet lists hold the same multiset of (row, col, value-bits)."""
    def key(t):
        r, c, v = t
        bits = np.asarray(v, np.float64).view(np.int64)
        return np.lexsort((bits, c, r)), (r, c, bits)
    (ia, (ra, ca, va)), (ib, (rb, cb, vb)) = key(a), key(b)
    if ra.size != rb.size:
        return False
    return bool(np.array_equal(ra[ia], rb[ib]) and np.array_equal(ca[ia], cb[ib]) and np.array_equal(va[ia], vb[ib]))
