"""Implicit time stepping through the C ABI (one plan and one FSAI preconditioner reused for every step,
b = (c I) u_t by the library's SpMV on a diagonal plan, a warm-started solve per step) against the same steps
taken by the oracle's CG to a tighter tolerance."""
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


def _system(K):
    rows = np.repeat(np.arange(K.n), np.diff(K.row_ptr))
    c = 0.1 * float(K.val[K.col.astype(np.int64) == rows].mean())
    return c, gen.shifted(K, c), gen.scaled_identity(K.n, c)


@pytest.mark.parametrize("which", ["tet", "hex"])
@pytest.mark.parametrize("solver", ["cg", "pcg", "pcg_refined"])
def test_transient_steps_match_the_oracle(eh, which, solver):
    K = gen.tet_lap3d(N=14) if which == "tet" else gen.hex_elast3d(N=7)   # hex: Neumann K, K + cI is SPD
    c, S, R = _system(K)
    u0 = gen.uniform(K.n, 5)
    PS, PR = eh.Plan(S, lowp=1), eh.Plan(R)
    M = None if solver == "cg" else eh.Fsai(PS, S, lowp=0 if solver == "pcg" else 2)
    u = torch.from_numpy(u0).cuda()
    b = torch.empty_like(u)
    steps = 5
    for _ in range(steps):
        PR.spmv(u, b)
        if solver == "cg":
            st, info = PS.cg(b, u, rtol=1e-10)
        elif solver == "pcg":
            st, info = PS.pcg(M, b, u, rtol=1e-10)
        else:
            st, info = PS.pcg_refined(M, b, u, rtol=1e-10)
        assert st == 0 and info["converged"]
    bh, uh = b.cpu().numpy(), u.cpu().numpy()
    assert np.linalg.norm(bh - oracle.spmv(S, uh)) <= 1.01e-10 * np.linalg.norm(bh)   # last step's FP64 residual
    uo = u0.copy()
    for _ in range(steps):
        bo = oracle.spmv(R, uo)
        uo, ok, _, _ = oracle.cg(S, bo, x0=uo, rtol=1e-13)
        assert ok
    assert np.linalg.norm(uh - uo) <= 1e-8 * np.linalg.norm(uo)
