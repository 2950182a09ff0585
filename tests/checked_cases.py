"""Parity cases run against the bounds-checked library (EHYB_LIBRARY points at libehyb_checked.so) by
test_gpu_checked.py: the SpMV in every layout (the halo layout included) and precision (low-precision copies in
both slot layouts), SpMM, the batched launch, CG (also flexible), PCG, plan files and row shards, each followed by
a read of the status word, which must not report a bounds violation."""
import os
import sys
import tempfile

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
import gen  # noqa: E402
import oracle  # noqa: E402
import paper_2204_06666_gb300 as eh  # noqa: E402

assert os.path.basename(eh.lib_path()) == "libehyb_checked.so", eh.lib_path()
torch.cuda.set_device(0)


def ok(P):
    st = P.check()
    assert st == 0, eh.STATUS.get(st, st)


# the check itself: an index outside its buffer is reported, one inside is not
assert eh.ehyb_test_bounds_probe(5, 5) == 12 and eh.ehyb_test_bounds_probe(-1, 5) == 12
assert eh.ehyb_test_bounds_probe(4, 5) == 0

A = gen.random_csr(3001, 1, mean_row=11, int_values=True, empty_frac=0.05, long_rows=5, long_len=1500, duplicates=True)
x = gen.int_vector(A.n, 101)
ref = oracle.spmv(A, x)
for opt in (dict(), dict(ell_tpr=4), dict(ell_tpr=32), dict(ell_width_cap=6), dict(slice_rows=37, block_threads=64),
            dict(er_layout=1, ell_tpr=2, er_tpr=4), dict(lowp=1), dict(lowp=2), dict(lowp=1, lowp_group=4),
            dict(lowp=2, lowp_group=4, ell_tpr=2), dict(er_layout=2, lowp=1), dict(er_layout=2, lowp=2, ell_tpr=4),
            dict(er_layout=2, slice_rows=37, block_threads=64)):
    P = eh.Plan(A, **opt)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    P.spmv(xd, y)
    assert np.array_equal(y.cpu().numpy(), ref), opt
    xp, yp = torch.empty_like(xd), torch.empty_like(xd)
    P.permute(True, xd, xp)
    P.spmv_permuted(xp, yp)
    if opt.get("lowp"):
        y32 = torch.empty(A.n, dtype=torch.float32, device="cuda")
        P.spmv_lowp(xd.float(), y32)
        assert np.array_equal(y32.cpu().numpy().astype(np.float64), ref), opt
    ok(P)

H = gen.hex_elast3d(N=14)
P = eh.Plan(H)
X = torch.from_numpy(np.stack([gen.uniform(H.n, 40 + j) for j in range(8)], axis=1).copy()).cuda()
Y = torch.empty_like(X)
P.spmm(X, Y)
assert np.linalg.norm(Y.cpu().numpy() - oracle.spmm(H, X.cpu().numpy())) <= 1e-13 * np.linalg.norm(Y.cpu().numpy())
ok(P)

mats = [gen.fem2d_p1(N=40), gen.tet_lap3d(N=12, dirichlet=False), H]
plans = [eh.Plan(M, part_nnz=20000) for M in mats]
xs = [torch.from_numpy(gen.uniform(M.n, 7 + i)).cuda() for i, M in enumerate(mats)]
ys = [torch.empty_like(v) for v in xs]
B = eh.Batch(plans)
B.spmv(xs, ys)
torch.cuda.synchronize()
for M, v, w, Q in zip(mats, xs, ys, plans):
    r = oracle.spmv(M, v.cpu().numpy())
    assert np.linalg.norm(w.cpu().numpy() - r) <= 1e-13 * np.linalg.norm(r)
    ok(Q)

T = gen.tet_lap3d(N=12)
for lay in (2,):  # the halo layout inside the FP64 CG (plan numbering, fused dot)
    Ph = eh.Plan(T, er_layout=lay)
    bh = torch.from_numpy(oracle.spmv(T, gen.uniform(T.n, 9))).cuda()
    xh = torch.zeros_like(bh)
    st, info = Ph.cg(bh, xh, rtol=1e-10)
    assert st == 0, info
    ok(Ph)
P = eh.Plan(T, lowp=1)
b = torch.from_numpy(oracle.spmv(T, gen.uniform(T.n, 9))).cuda()
for refine in (0, 3):
    xx = torch.zeros_like(b)
    st, info = P.cg(b, xx, rtol=1e-10, refine=refine)
    assert st == 0, (refine, info)
xx = torch.zeros_like(b)
st, info = P.cg(b, xx, rtol=1e-10, refine=5)        # flexible CG, FP32 inner solve
assert st == 0 and info["flexible"] == 1, info
M = eh.Fsai(P, T, lowp=1)
for solve in (P.pcg, P.pcg_refined):
    xx = torch.zeros_like(b)
    st, info = solve(M, b, xx, rtol=1e-10)
    assert st == 0, info
ok(P)
with tempfile.TemporaryDirectory() as d:
    f = os.path.join(d, "t.ehyb")
    P.save(f)
    Q = eh.Plan.load(f)
    y1, y2 = torch.empty_like(b), torch.empty_like(b)
    P.spmv(b, y1)
    Q.spmv(b, y2)
    assert torch.equal(y1, y2)
    ok(Q)
# row shards: each rank's product on [own rows | halo], the halo filled from the plan-numbering x directly
Pn = eh.Plan(T)
n2o = Pn.export()["new_to_old"]
xp = torch.from_numpy(gen.uniform(T.n, 4)[n2o]).cuda()
yp = torch.empty_like(xp)
assert eh.ehyb_spmv_permuted(Pn.handle, xp.data_ptr(), yp.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
for r in range(3):
    S = eh.Shard(Pn, 3, r)
    L = S.lists()
    xe = torch.cat([xp[S.row_begin:S.row_end], xp[torch.from_numpy(L["halo_rows"].astype(np.int64)).cuda()]])
    y = torch.empty(S.n_local, dtype=torch.float64, device="cuda")
    S.spmv(xe, y)
    send = torch.empty(max(S.send_total, 1), dtype=torch.float64, device="cuda")
    S.pack(xe[:S.n_local], send)
    torch.cuda.synchronize()
    assert torch.equal(y, yp[S.row_begin:S.row_end])
    assert S.info()["device_status"] == 0
print("CHECKED OK")
