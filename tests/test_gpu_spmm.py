"""EHYB SpMM (k right-hand sides) against the oracle and against ehyb_spmv column by column."""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.mark.parametrize("k", [1, 2, 3, 8, 12, 32])
def test_spmm_integer_exact(eh, k):
    A = gen.random_csr(3000, k, mean_row=10, int_values=True, empty_frac=0.05, long_rows=2, long_len=900,
                       duplicates=True)
    X = np.random.default_rng(k).integers(-8, 9, (A.n, k)).astype(np.float64)
    P = eh.Plan(A, slice_rows=400)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full_like(Xd, np.nan)
    P.spmm(Xd, Yd)
    torch.cuda.synchronize()
    assert np.array_equal(Yd.cpu().numpy(), oracle.spmm(A, X))


@pytest.mark.parametrize("N,k,rhs", [(16, 8, 0), (12, 32, 0), (16, 8, 8), (12, 32, 32)])
def test_spmm_columns_equal_spmv(eh, N, k, rhs):
    # rhs: a plan built for k right-hand sides (smaller partitions, whole 8-column chunks)
    A = gen.hex_elast3d(N=N)
    X = np.stack([gen.uniform(A.n, 50 + j) for j in range(k)], axis=1)
    P = eh.Plan(A, spmm_rhs=rhs)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.empty_like(Xd)
    P.spmm(Xd, Yd)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    for j in range(k):
        P.spmv(Xd[:, j].contiguous(), y)
        assert torch.equal(Yd[:, j], y), j
    ref = oracle.spmm(A, X)
    Y = Yd.cpu().numpy()
    assert np.linalg.norm(Y - ref) <= 1e-13 * np.linalg.norm(ref)
    kk = np.diff(A.row_ptr).astype(np.float64)
    absA = gen.CSR(A.n, A.row_ptr, A.col, np.abs(A.val))
    bound = 2 * oracle.gamma(kk + 6)[:, None] * oracle.spmm(absA, np.abs(X))
    assert np.all(np.abs(Y - ref) <= bound)


def test_spmm_hex70_k8_as_benchmarked(eh):
    A = gen.hex_elast3d()
    k = 8
    X = np.stack([gen.uniform(A.n, 32 + j) for j in range(k)], axis=1)
    P = eh.Plan(A, spmm_rhs=k)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.empty_like(Xd)
    P.spmm(Xd, Yd)
    torch.cuda.synchronize()
    ref = oracle.spmm(A, X)
    Y = Yd.cpu().numpy()
    assert np.linalg.norm(Y - ref) <= 1e-13 * np.linalg.norm(ref)
    assert P.check() == 0


def test_spmm_errors(eh):
    A = gen.fem2d_p1(N=20)
    P = eh.Plan(A, er_layout=1)
    X = torch.zeros((A.n, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(eh.EhybError) as e:
        P.spmm(X, torch.empty_like(X))
    assert e.value.status == 7
