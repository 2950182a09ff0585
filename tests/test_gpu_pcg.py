"""FSAI preconditioner and preconditioned CG through the C ABI against the oracle: G entry by entry, the
PCG residual history, convergence to 1e-10 with the true residual recomputed by the oracle, and the
error statuses."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import gen
import oracle
from oracle import fsai as of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    torch.cuda.set_device(0)
    return m


def _permuted(A, n2o):
    B = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))[n2o][:, n2o].tocsr()
    B.sort_indices()
    return gen.CSR(A.n, B.indptr.astype(np.int64), B.indices.astype(np.int32), B.data.copy())


@pytest.mark.parametrize("which", ["tet", "hex"])
def test_fsai_matches_oracle_entry_by_entry(eh, which):
    A = gen.tet_lap3d(N=10) if which == "tet" else gen.hex_elast3d(N=6, clamp_minz=True)
    P = eh.Plan(A, slice_rows=300)
    M = eh.Fsai(P, A)
    rp, col, val = M.export()
    n2o = P.export()["new_to_old"]
    G = of.fsai(A, n2o)
    G.sort_indices()
    assert np.array_equal(rp, G.indptr) and np.array_equal(col, G.indices)
    assert np.allclose(val, G.data, rtol=1e-11, atol=1e-14)
    assert M.info()["nnz_g"] == G.nnz


def test_pcg_history_matches_oracle_pcg(eh):
    A = gen.tet_lap3d(N=12)
    P = eh.Plan(A, slice_rows=400)
    M = eh.Fsai(P, A)
    xs = gen.uniform(A.n, 7)
    b = oracle.spmv(A, xs)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, info = P.pcg(M, torch.from_numpy(b).cuda(), x, rtol=1e-10)
    assert st == 0 and info["converged"]
    hist = M.history()
    # the oracle's PCG on P A P^T with the oracle's G, b permuted the same way
    n2o = P.export()["new_to_old"]
    _, k, rr, _ = of.pcg(_permuted(A, n2o), of.fsai(A, n2o), b[n2o], rtol=1e-10)
    assert abs(info["iterations"] - k) <= 1
    m = min(20, len(hist), len(rr))
    assert np.allclose(hist[:m], rr[:m], rtol=1e-7, atol=0)
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - oracle.spmv(A, xh)) <= 1.01e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("lowp", [0, 1, 2])
@pytest.mark.parametrize("which", ["tet", "hex"])
def test_pcg_reaches_1e10_with_fewer_iterations_than_cg(eh, lowp, which):
    A = gen.tet_lap3d(N=20) if which == "tet" else gen.hex_elast3d(N=10, clamp_minz=True)
    P = eh.Plan(A)
    M = eh.Fsai(P, A, lowp=lowp)
    b = oracle.spmv(A, gen.uniform(A.n, 24))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, info = P.pcg(M, bd, x, rtol=1e-10)
    assert st == 0 and info["converged"] and info["relres"] <= 1.01e-10
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - oracle.spmv(A, xh)) <= 1.01e-10 * np.linalg.norm(b)
    x2 = torch.zeros_like(bd)
    _, cg = P.cg(bd, x2, rtol=1e-10)
    assert info["iterations"] < 0.7 * cg["iterations"], (info["iterations"], cg["iterations"])


def test_pcg_full_size_tet(eh):
    A = gen.tet_lap3d()
    P = eh.Plan(A)
    M = eh.Fsai(P, A)
    b = oracle.spmv(A, gen.uniform(A.n, 23))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, info = P.pcg(M, bd, x, rtol=1e-10)
    assert st == 0 and info["converged"]
    assert np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) <= 1.01e-10 * np.linalg.norm(b)


def test_pcg_errors(eh):
    A = gen.tet_lap3d(N=6)
    P, Q = eh.Plan(A), eh.Plan(A)
    M = eh.Fsai(P, A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(eh.EhybError) as e:
        Q.pcg(M, b, torch.zeros_like(b))
    assert e.value.status == 1                       # the preconditioner belongs to another plan
    N = gen.CSR(A.n, A.row_ptr, A.col, -A.val)       # negative definite: a principal block fails Cholesky
    R = eh.Plan(N)
    with pytest.raises(eh.EhybError) as e:
        eh.Fsai(R, N)
    assert e.value.status == 1
    st, info = P.pcg(M, b, torch.zeros_like(b), rtol=1e-14, max_iter=3)
    assert st == eh.EHYB_ERR_NOT_CONVERGED and info["iterations"] == 3


@pytest.mark.parametrize("lowp_g", [1, 2])
@pytest.mark.parametrize("which", ["tet", "hex"])
def test_refined_pcg_reaches_1e10(eh, lowp_g, which):
    # A's values in FP32 (BF16 values of A are too coarse for elasticity: u_bf16 * cond(A) > 1), G's values in
    # FP32 or BF16
    A = gen.tet_lap3d(N=20) if which == "tet" else gen.hex_elast3d(N=10, clamp_minz=True)
    P = eh.Plan(A, lowp=1)
    M = eh.Fsai(P, A, lowp=lowp_g)
    xs = gen.uniform(A.n, 25)
    b = oracle.spmv(A, xs)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, info = P.pcg_refined(M, bd, x, rtol=1e-10)
    assert st == 0 and info["converged"] and info["refinements"] >= 2
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - oracle.spmv(A, xh)) <= 1.01e-10 * np.linalg.norm(b)   # the oracle's FP64 residual
    x2 = torch.zeros_like(bd)
    _, pinfo = P.pcg(M, bd, x2, rtol=1e-10)
    assert info["iterations"] <= 1.5 * pinfo["iterations"] + 10, (info, pinfo)


def test_refined_pcg_needs_low_precision_values(eh):
    A = gen.tet_lap3d(N=6)
    P = eh.Plan(A)                       # no FP32 copy of A
    M = eh.Fsai(P, A, lowp=1)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(eh.EhybError) as e:
        P.pcg_refined(M, b, torch.zeros_like(b))
    assert e.value.status == 7


def test_pcg_from_a_nonzero_start_and_empty_matrix(eh):
    A = gen.tet_lap3d(N=12)
    P = eh.Plan(A, lowp=1)
    M = eh.Fsai(P, A, lowp=1)
    xs = gen.uniform(A.n, 31)
    b = oracle.spmv(A, xs)
    bd = torch.from_numpy(b).cuda()
    x0 = torch.from_numpy(xs + 1e-3 * gen.uniform(A.n, 32)).cuda()      # close to the solution
    for solve in (P.pcg, P.pcg_refined):
        x = x0.clone()
        st, info = solve(M, bd, x, rtol=1e-10)
        assert st == 0 and info["converged"]
        assert np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) <= 1.01e-10 * np.linalg.norm(b)
    x = torch.zeros_like(bd)                                            # b = 0 and x0 = 0: converged at once
    st, info = P.pcg(M, torch.zeros_like(bd), x, rtol=1e-10)
    assert st == 0 and info["iterations"] == 0 and torch.count_nonzero(x) == 0
    E = gen.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    PE = eh.Plan(E)
    ME = eh.Fsai(PE, E)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")[:0]
    st, info = PE.pcg(ME, z, z.clone())
    assert st == 0 and info["converged"]


def test_fsai_missing_diagonal_is_refused(eh):
    A = gen.tet_lap3d(N=6)
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).tolil()
    S[5, 5] = 0.0
    S = S.tocsr()
    S.eliminate_zeros()                                                 # row 5 loses its diagonal entry
    B = gen.CSR(A.n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.copy())
    P = eh.Plan(B)
    with pytest.raises(eh.EhybError) as e:
        eh.Fsai(P, B)
    assert e.value.status == 1
