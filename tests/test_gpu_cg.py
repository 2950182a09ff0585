"""GPU conjugate gradients and mixed-precision refinement (ehyb_cg, C ABI) against the CPU oracle.

FP64 CG follows the same recurrences as the oracle's textbook CG, so the residual histories agree to
rounding for the first iterations and the iteration counts agree to a few; every returned x is checked
by recomputing its residual with the oracle SpMV.  Refinement results state their error against the
FP64 oracle solution.
"""
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


def _csr_from_dense(D):
    n = D.shape[0]
    rows, cols = np.nonzero(D)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return gen.CSR(n, np.cumsum(rp), cols.astype(np.int32), D[rows, cols].astype(np.float64))


def _solve(eh, A, b, x0=None, **kw):
    P = eh.Plan(A, **{k: v for k, v in kw.items() if k in ("lowp", "slice_rows", "er_layout")})
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.from_numpy(np.ascontiguousarray(x0)).cuda()
    st, info = P.cg(bd, xd, **{k: v for k, v in kw.items() if k in ("rtol", "max_iter", "refine", "inner_rtol")})
    return P, st, info, xd.cpu().numpy()


def _true_relres(A, b, x):
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


def test_cg_small_spd_matches_lapack(eh):
    rng = np.random.default_rng(0)
    n = 40
    M = rng.standard_normal((n, n))
    D = M @ M.T
    D[np.abs(D) < 2.0] = 0.0
    D = (D + D.T) / 2 + np.diag(np.abs(D).sum(1) + 1.0)
    A = _csr_from_dense(D)
    b = rng.uniform(-1, 1, n)
    P, st, info, x = _solve(eh, A, b, rtol=1e-13, max_iter=400)
    assert st == 0 and info["converged"] == 1
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_cg_1d_laplacian_history_matches_oracle(eh):
    n = 64
    D = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = _csr_from_dense(D)
    xstar = np.sin(np.arange(1, n + 1) * 3 * np.pi / (n + 1)) + np.linspace(0, 1, n)
    b = oracle.spmv(A, xstar)
    P, st, info, x = _solve(eh, A, b, rtol=1e-12, max_iter=10 * n)
    xo, ok, it_o, rel_o, hist_o = oracle.cg(A, b, rtol=1e-12, max_iter=10 * n, history=True)
    assert st == 0 and ok
    assert info["iterations"] <= n + 2 and abs(info["iterations"] - it_o) <= 2
    hist = np.sqrt(P.cg_history()) / np.linalg.norm(b)
    k = min(20, len(hist), len(hist_o))
    assert np.allclose(hist[:k], hist_o[:k], rtol=1e-8, atol=0)
    assert _true_relres(A, b, x) <= 1e-11
    assert np.linalg.norm(x - xstar) <= 1e-9 * np.linalg.norm(xstar)


@pytest.mark.parametrize("name", ["tet", "hex"])
def test_cg_known_solution_fem(eh, name):
    A = gen.tet_lap3d(N=24) if name == "tet" else gen.hex_elast3d(N=10, clamp_minz=True)
    xstar = gen.uniform(A.n, 23)
    b = oracle.spmv(A, xstar)
    P, st, info, x = _solve(eh, A, b, rtol=1e-10, max_iter=5000)
    xo, ok, it_o, rel_o = oracle.cg(A, b, rtol=1e-10, max_iter=5000)
    assert st == 0 and info["converged"] == 1 and ok
    rel = _true_relres(A, b, x)
    assert rel <= 1.5e-10                         # recomputed independently by the oracle
    assert abs(info["relres"] - rel) <= 1e-12     # the library's own FP64 residual agrees
    assert abs(info["iterations"] - it_o) <= max(3, it_o // 50)
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_cg_warm_start_and_determinism(eh):
    A = gen.tet_lap3d(N=16)
    xstar = gen.uniform(A.n, 5)
    b = oracle.spmv(A, xstar)
    x0 = xstar + 1e-3 * gen.uniform(A.n, 6)
    P, st, info, x1 = _solve(eh, A, b, x0=x0, rtol=1e-10)
    _, _, info2, x2 = _solve(eh, A, b, x0=x0, rtol=1e-10)
    assert st == 0 and np.array_equal(x1, x2) and info["iterations"] == info2["iterations"]
    _, _, info_cold, _ = _solve(eh, A, b, rtol=1e-10)
    assert info["iterations"] < info_cold["iterations"]
    assert _true_relres(A, b, x1) <= 1.5e-10


def test_cg_not_converged_status(eh):
    A = gen.tet_lap3d(N=20)
    b = oracle.spmv(A, gen.uniform(A.n, 1))
    P, st, info, x = _solve(eh, A, b, rtol=1e-12, max_iter=7)
    assert st == eh.EHYB_ERR_NOT_CONVERGED and info["iterations"] == 7 and info["converged"] == 0
    assert abs(info["relres"] - _true_relres(A, b, x)) <= 1e-12
    # zero right-hand side: converged before the first iteration
    P, st, info, x = _solve(eh, A, np.zeros(A.n), rtol=1e-10)
    assert st == 0 and info["iterations"] == 0 and np.all(x == 0)


@pytest.mark.parametrize("refine,lowp", [(1, 1), (2, 2), (3, 1), (4, 2), (5, 1), (6, 2)])
def test_refined_cg_reaches_fp64_accuracy(eh, refine, lowp):
    A = gen.tet_lap3d(N=24)
    xstar = gen.uniform(A.n, 23)
    b = oracle.spmv(A, xstar)
    P, st, info, x = _solve(eh, A, b, rtol=1e-10, max_iter=20000, refine=refine, lowp=lowp)
    rel = _true_relres(A, b, x)
    assert abs(info["relres"] - rel) <= 1e-12
    assert st == 0 and info["converged"] == 1 and rel <= 1.5e-10, info
    assert info["refinements"] >= 2
    xo = oracle.cg(A, b, rtol=1e-12, max_iter=20000)[0]
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)   # stated error against the FP64 oracle solution
    assert err <= 1e-7


@pytest.mark.parametrize("refine", [6, 4])
def test_bf16_values_on_clamped_elasticity_reach_1e10(eh, refine):
    # clamped Q1 elasticity: u_bf16 kappa(A) is not small, so refinement around a BF16 solve can stall; the
    # flexible FP64 CG (refine 6, or taking over refine 4) keeps the BF16 solve as a preconditioner only
    A = gen.hex_elast3d(N=14, clamp_minz=True)
    xstar = gen.uniform(A.n, 24)
    b = oracle.spmv(A, xstar)
    P, st, info, x = _solve(eh, A, b, rtol=1e-10, max_iter=40000, refine=refine, lowp=2)
    rel = _true_relres(A, b, x)                          # the FP64 residual, recomputed by the oracle
    assert st == 0 and info["converged"] == 1 and rel <= 1e-10, info
    assert abs(info["relres"] - rel) <= 1e-12
    if refine == 6:
        assert info["flexible"] == 1 and info["refinements"] >= 2
    xo = oracle.cg(A, b, rtol=1e-12, max_iter=40000)[0]
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6   # stated error against the FP64 oracle solve


def test_flexible_cg_is_deterministic(eh):
    A = gen.tet_lap3d(N=16)
    b = oracle.spmv(A, gen.uniform(A.n, 3))
    P = eh.Plan(A, lowp=2)
    bd = torch.from_numpy(b).cuda()
    outs = []
    for _ in range(2):
        xd = torch.zeros_like(bd)
        st, info = P.cg(bd, xd, rtol=1e-10, max_iter=20000, refine=6)
        assert st == 0
        outs.append((xd.cpu().numpy(), info["iterations"], info["refinements"]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]


def test_cg_option_errors(eh):
    A = gen.tet_lap3d(N=10)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    P = eh.Plan(A)
    with pytest.raises(eh.EhybError) as e:
        P.cg(b, x, refine=1)          # no FP32 value copy in this plan
    assert e.value.status == 7
    with pytest.raises(eh.EhybError) as e:
        P.cg(b, x, refine=6)          # no BF16 value copy either
    assert e.value.status == 7
    with pytest.raises(eh.EhybError) as e:
        P.cg(b, x, refine=7)
    assert e.value.status == 1
    Q = eh.Plan(A, er_layout=1)
    with pytest.raises(eh.EhybError) as e:
        Q.cg(b, x)                    # the fused dot needs the sliced ER layout
    assert e.value.status == 7
