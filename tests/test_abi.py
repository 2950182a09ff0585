"""The C ABI library loads, exports every declared symbol, and rejects bad input (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ehyb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ehyb_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2204_06666_gb300 as eh
    lib = ctypes.CDLL(eh.lib_path())
    names = _declared()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    import paper_2204_06666_gb300 as eh
    for code in range(11):
        assert eh._lib.ehyb_status_string(code).decode()


def _create(n, nc, rp, col, val, **opt):
    import paper_2204_06666_gb300 as eh
    h = ctypes.c_void_p()
    o = eh.make_options(**opt)
    rp = np.ascontiguousarray(rp, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    nnz = int(col.size)
    st = eh.ehyb_plan_create_csr(n, nc, nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data, o, None, h)
    if st == 0:
        eh.ehyb_destroy(h)
    return st


def test_invalid_inputs_return_codes():
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([0, 1], np.int32)
    val = np.ones(2)
    assert _create(2, 3, rp, col, val, host_only=1) == 2                       # not square
    assert _create(2, 2, np.array([0, 2, 1]), col, val, host_only=1) == 3      # row_ptr decreasing / inconsistent
    assert _create(2, 2, np.array([1, 1, 2]), col, val, host_only=1) == 3      # row_ptr[0] != 0
    assert _create(2, 2, rp, np.array([0, 2], np.int32), val, host_only=1) == 3   # column out of range
    assert _create(2, 2, rp, np.array([0, -1], np.int32), val, host_only=1) == 3  # negative column
    assert _create(-1, -1, rp, col, val, host_only=1) == 1
    assert _create(2 ** 31, 2 ** 31, rp, col, val, host_only=1) == 4         # n too large for the 32-bit numbering
    assert _create(2, 2, rp, col, val, host_only=1, ell_tpr=3) == 1            # not a power of two
    assert _create(2, 2, rp, col, val, host_only=1, block_threads=100) == 1
    assert _create(2, 2, rp, col, val, host_only=1, slice_rows=70000) == 4     # beyond the 16-bit offset
    assert _create(2, 2, rp, col, val, host_only=1) == 0


def test_invalid_inputs_found_anywhere_in_large_arrays():
    # the row-pointer and column scans run in parallel pieces: a single violation at the start, in the
    # middle or at the end of arrays spanning many pieces is still reported
    n = 1 << 20
    rp = np.arange(n + 1, dtype=np.int64) * 2
    col = np.repeat(np.arange(n, dtype=np.int32), 2)
    val = np.ones(2 * n)
    assert _create(n, n, rp, col, val, host_only=1, num_sms=8) == 0
    for at in (0, n, 2 * n - 1):
        for bad in (n, -1, 2 ** 31 - 1):
            c = col.copy()
            c[at] = bad
            assert _create(n, n, rp, c, val, host_only=1, num_sms=8) == 3, (at, bad)
    for at in (1, n // 2, n - 1):
        r = rp.copy()
        r[at] = r[at + 1] + 1  # one decrease
        assert _create(n, n, r, col, val, host_only=1, num_sms=8) == 3, at


def test_partition_too_large_for_shared_memory():
    import paper_2204_06666_gb300 as eh
    A = gen.random_csr(40000, 1, mean_row=3)
    with pytest.raises(eh.EhybError) as e:
        eh.Plan(A, host_only=1, part_vec=np.zeros(A.n, np.int32))   # one 40000-row partition: 320 KB of x
    assert e.value.status == 4


def test_host_only_plan_refuses_device_calls():
    import paper_2204_06666_gb300 as eh
    A = gen.random_csr(100, 2)
    P = eh.Plan(A, host_only=1)
    assert eh._lib.ehyb_spmv(P.handle, None, None, None) == 7
    assert eh._lib.ehyb_plan_check(P.handle) == 7
    assert eh._lib.ehyb_spmv_host(P.handle, None, None, None) == 7
    assert eh._lib.ehyb_spmv_host_many(P.handle, 1, None, None, None) == 7
    assert eh._lib.ehyb_spmv_host_many(None, 0, None, None, None) == 1      # no plan


def test_no_device_is_reported_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2204_06666_gb300 as eh
    A = gen.random_csr(100, 2)
    with pytest.raises(eh.EhybError) as e:
        eh.Plan(A, stream=0)
    assert e.value.status == 10
