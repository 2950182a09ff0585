"""Batched EHYB SpMV (one persistent launch over many plans, replayed from a CUDA graph).

The batch runs every partition with the same per-row summation as ehyb_spmv, so its results must
equal the per-plan results bit for bit; integer-valued inputs also equal the oracle exactly.
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


def _single(P, x):
    y = torch.full_like(x, np.nan)
    P.spmv(x, y)
    return y


def test_batch_equals_single_plans_bitwise(eh):
    mats = [gen.random_csr(2000 + 37 * i, i, mean_row=9, int_values=True, empty_frac=0.05, long_rows=2,
                           long_len=700, duplicates=True) for i in range(4)]
    mats += [gen.fem2d_p1(N=90), gen.hex_elast3d(N=11), gen.tet_lap3d(N=17), gen.hex_lap3d(N=13)]
    plans = [eh.Plan(A, slice_rows=sr) for A, sr in zip(mats, (100, 333, 0, 1000, 0, 500, 0, 250))]
    B = eh.Batch(plans)
    xs_np = [gen.int_vector(A.n, i) if i < 4 else gen.uniform(A.n, i) for i, A in enumerate(mats)]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    ys = [torch.full_like(x, np.nan) for x in xs]
    B.spmv(xs, ys)
    torch.cuda.synchronize()
    for i, (P, A) in enumerate(zip(plans, mats)):
        ref = _single(P, xs[i])
        torch.cuda.synchronize()
        assert torch.equal(ys[i], ref), i
        if i < 4:
            assert np.array_equal(ys[i].cpu().numpy(), oracle.spmv(A, xs_np[i]))
    # replay with new vectors in new buffers
    xs2 = [torch.from_numpy(gen.uniform(A.n, 100 + i)).cuda() for i, A in enumerate(mats)]
    ys2 = [torch.empty_like(x) for x in xs2]
    for _ in range(3):
        B.spmv(xs2, ys2)
    torch.cuda.synchronize()
    for i, P in enumerate(plans):
        assert torch.equal(ys2[i], _single(P, xs2[i]))
    assert all(p.check() == 0 for p in plans)
    info = B.info()
    assert info["tiles"] == sum(P.info()["nparts"] for P in plans) and info["grid"] >= 152


def test_batch_of_generated_fem_matrices(eh):
    mats = gen.fem_batch(count=16, seed=31, n_max=60000)
    plans = [eh.Plan(A) for A in mats]
    B = eh.Batch(plans)
    xs = [torch.from_numpy(gen.uniform(A.n, 32 + i)).cuda() for i, A in enumerate(mats)]
    ys = [torch.empty_like(x) for x in xs]
    B.spmv(xs, ys)
    torch.cuda.synchronize()
    for i, (P, A) in enumerate(zip(plans, mats)):
        assert torch.equal(ys[i], _single(P, xs[i]))
    # and against the oracle, within the FP64 bar, for two of them
    for i in (0, 7):
        ref = oracle.spmv(mats[i], xs[i].cpu().numpy())
        y = ys[i].cpu().numpy()
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)


def test_batch_errors(eh):
    A = gen.fem2d_p1(N=20)
    with pytest.raises(eh.EhybError) as e:
        eh.Batch([eh.Plan(A, er_layout=1)])
    assert e.value.status == 7
    with pytest.raises(eh.EhybError) as e:
        eh.Batch([])
    assert e.value.status == 1
