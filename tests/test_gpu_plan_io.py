"""Plan files on the GPU: a plan saved (from device arrays or kept host arrays) and loaded again computes
bit-identical results, in FP64 and with FP32 values made from the stored FP64 ones."""
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


def _y(P, x):
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, np.nan)
    P.spmv(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("opt", [dict(), dict(keep_host=1), dict(er_layout=1), dict(ell_tpr=2, slice_rows=700)])
def test_saved_plan_loads_bit_identical(eh, tmp_path, opt):
    A = gen.hex_elast3d(N=16)
    x = gen.uniform(A.n, 4)
    P = eh.Plan(A, **opt)
    y = _y(P, x)
    f = str(tmp_path / "hex.ehyb")
    P.save(f)
    Q = eh.Plan.load(f)
    assert Q.info()["partition_ms"] == 0.0 and Q.info()["nparts"] == P.info()["nparts"]
    assert np.array_equal(_y(Q, x), y)
    ref = oracle.spmv(A, x)
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    assert Q.check() == 0


def test_loaded_plan_low_precision_copies(eh, tmp_path):
    A = gen.tet_lap3d(N=20)
    P = eh.Plan(A, lowp=1)
    f = str(tmp_path / "tet.ehyb")
    P.save(f)
    Q = eh.Plan.load(f, lowp=1)
    x = torch.from_numpy(gen.uniform(A.n, 8).astype(np.float32)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    P.spmv_lowp(x, y1)
    Q.spmv_lowp(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_loaded_plan_solves_like_the_saved_one(eh, tmp_path):
    # CG on a loaded plan (FP64 and FP32 residual replacement) gives the iterations and bits of the original
    A = gen.tet_lap3d(N=14)
    P = eh.Plan(A, lowp=1)
    f = str(tmp_path / "tet.ehyb")
    P.save(f)
    Q = eh.Plan.load(f, lowp=1)
    b = torch.from_numpy(oracle.spmv(A, gen.uniform(A.n, 5))).cuda()
    for refine in (0, 3):
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        _, i1 = P.cg(b, x1, rtol=1e-10, refine=refine)
        _, i2 = Q.cg(b, x2, rtol=1e-10, refine=refine)
        assert i1["iterations"] == i2["iterations"] and torch.equal(x1, x2)
