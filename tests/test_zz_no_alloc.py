"""ehyb_spmv_noalloc: the SpMV for callers that cannot allocate device memory when they call.

Such a caller (a plug-in inside a framework that owns all device memory, a latency-critical loop)
gets the same product as ehyb_spmv while the gathered copy of x lives in a fixed array compiled
into the library instead of plan workspace.  These tests call it through the C ABI and compare it
with ehyb_spmv, twice in a row (the second call must not be affected by what the first one left in
the shared array), and check that matrices above its 2^20-row limit are refused.
"""
import ctypes

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu

MAX_ROWS = 1 << 20


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    torch.cuda.set_device(0)
    return m


def _both(eh, P, x):
    """(y from ehyb_spmv, y from ehyb_spmv_noalloc), both through the C ABI."""
    s = torch.cuda.current_stream().cuda_stream
    xd = torch.from_numpy(x).cuda()
    y_ref = torch.full_like(xd, np.nan)
    y_new = torch.full_like(xd, np.nan)
    assert eh.ehyb_spmv(P.handle, xd.data_ptr(), y_ref.data_ptr(), s) == 0
    assert eh.ehyb_spmv_noalloc(P.handle, xd.data_ptr(), y_new.data_ptr(), s) == 0
    torch.cuda.synchronize()
    assert P.check() == 0
    return y_ref.cpu().numpy(), y_new.cpu().numpy()


def _close(a, b):
    # both entry points sum every row in the same order (slab slots, then the row's extra entries), so
    # the results agree bit for bit; a lost or doubled extra-row term would show even when small in norm
    return np.array_equal(a, b)


def test_noalloc_matches_spmv_on_two_calls_in_a_row(eh):
    A = gen.fem2d_p1(N=200)                      # 40,000 rows
    B = gen.hex_elast3d(N=16)                    # 12,288 rows: a smaller second call over stale scratch
    PA, PB = eh.Plan(A), eh.Plan(B, slice_rows=500)
    ref1, new1 = _both(eh, PA, gen.uniform(A.n, 31))
    assert _close(ref1, new1)
    ref2, new2 = _both(eh, PB, gen.uniform(B.n, 32))
    assert _close(ref2, new2)
    ref3, new3 = _both(eh, PA, gen.uniform(A.n, 33))   # and back to the larger plan
    assert _close(ref3, new3)


def test_noalloc_integer_inputs_exact(eh):
    A = gen.random_csr(5000, 3, mean_row=12, int_values=True, empty_frac=0.05, long_rows=2, long_len=800)
    P = eh.Plan(A, slice_rows=333)
    for seed in (1, 2):
        ref, new = _both(eh, P, gen.int_vector(A.n, seed))
        assert np.array_equal(ref, new)


def test_noalloc_refuses_more_rows_than_its_array(eh):
    n = MAX_ROWS + 1
    A = gen.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    P = eh.Plan(A)
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st = eh.ehyb_spmv_noalloc(P.handle, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 4  # EHYB_ERR_TOO_LARGE
    assert eh.ehyb_spmv_noalloc(None, x.data_ptr(), y.data_ptr(), None) == 1
    # a plan exactly at the limit is accepted
    m = MAX_ROWS
    C = gen.CSR(m, np.arange(m + 1, dtype=np.int64), np.arange(m, dtype=np.int32), np.full(m, 2.0))
    Q = eh.Plan(C)
    xm = torch.arange(m, dtype=torch.float64, device="cuda")
    ym = torch.empty_like(xm)
    assert eh.ehyb_spmv_noalloc(Q.handle, xm.data_ptr(), ym.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(ym, 2.0 * xm)
