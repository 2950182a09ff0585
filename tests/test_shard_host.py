"""Row shards for several GPUs (ehyb_shard_*), host side: the exchange lists, the renumbered extra-row
columns, and the exchange and CG reductions over real gloo ranks (world size 2 and 4) on the CPU.

A shard's product is evaluated here by decoding its exported arrays with the oracle's independent decoder
(the GPU product is tested in test_gpu_shard.py); every result is compared with the oracle SpMV / CG of the
whole matrix."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import gen
import oracle
from oracle import ehyb_format as ef


def _plan(A, **kw):
    import paper_2204_06666_gb300 as eh
    return eh.Plan(A, host_only=1, **kw)


def _shard_matrix(S):
    """(rows, cols, vals) of a shard: local rows, columns into x_ext = [x_local | halo]."""
    import scipy.sparse as sp
    i = S.info()
    e = S.export()
    e["new_to_old"] = np.arange(i["n_local"] + i["n_halo"])     # identity: keep local / x_ext numbering
    r, c, v = ef.decode(e)
    return sp.csr_matrix((v, (r, c)), shape=(i["n_local"], i["n_local"] + i["n_halo"]))


MATS = {"tet": lambda: gen.tet_lap3d(N=12), "hex": lambda: gen.hex_elast3d(N=8, clamp_minz=True),
        "ragged": lambda: gen.random_csr(3000, 4, mean_row=9, long_rows=3, long_len=400, empty_frac=0.05,
                                         symmetric=True)}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("R", [1, 2, 3, 4, 7])
def test_shard_lists_and_products(name, R):
    import paper_2204_06666_gb300 as eh
    A = MATS[name]()
    P = _plan(A, slice_rows=256)
    ex = P.export()
    n2o = ex["new_to_old"]
    x = gen.uniform(A.n, 5)
    xp = x[n2o]                                   # x in the plan numbering
    yp = oracle.spmv(A, x)[n2o]
    shards = [eh.Shard(P, R, r) for r in range(R)]
    infos = [S.info() for S in shards]
    lists = [S.lists() for S in shards]
    # the ranks' rows and partitions tile the plan in order
    assert infos[0]["row_begin"] == 0 and infos[-1]["row_end"] == A.n
    assert infos[0]["part_begin"] == 0 and infos[-1]["part_end"] == ex["nparts"]
    for a, b in zip(infos, infos[1:]):
        assert a["row_end"] == b["row_begin"] and a["part_end"] == b["part_begin"]
    assert sum(i["slab_stored"] for i in infos) == ex["ell_col"].size
    for r, (S, i, L) in enumerate(zip(shards, infos, lists)):
        lo, hi = i["row_begin"], i["row_end"]
        h = L["halo_rows"]
        assert np.all(np.diff(h) > 0) and not np.any((h >= lo) & (h < hi))      # ascending, all remote
        for q in range(R):
            # what q receives from r is what r sends to q, in the same order
            qi, ql = infos[q], lists[q]
            recv = ql["halo_rows"][ql["recv_ptr"][r]:ql["recv_ptr"][r + 1]]
            sent = lo + L["send_idx"][L["send_ptr"][q]:L["send_ptr"][q + 1]]
            assert np.array_equal(recv, sent), (r, q)
            assert np.all((recv >= lo) & (recv < hi))
        # the shard's product on x_ext = [x_local | x at the halo rows] gives the plan's rows
        xe = np.concatenate([xp[lo:hi], xp[h]])
        y = _shard_matrix(S) @ xe
        ref = yp[lo:hi]
        assert np.allclose(y, ref, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(ref).max(initial=0.0)))
    if R > ex["nparts"]:
        assert any(i["n_local"] == 0 for i in infos)


def _gloo_rank(rank, world, port, name, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        import paper_2204_06666_gb300 as eh
        A = MATS[name]()             # the CG cases use the SPD matrices (tet: Dirichlet, hex: clamped)
        P = _plan(A, slice_rows=256)
        n2o = P.export()["new_to_old"]
        S = eh.Shard(P, world, rank)
        comm = eh.TorchComm()
        i = S.info()
        lo, hi, nl = i["row_begin"], i["row_end"], i["n_local"]
        L = S.lists()
        M = _shard_matrix(S)
        # ---- one exchange: the halo arrives in x_ext[nl:] in the halo list's order
        x = gen.uniform(A.n, 5)
        xp = x[n2o]
        xe = torch.zeros(nl + i["n_halo"], dtype=torch.float64)
        xe[:nl] = torch.from_numpy(xp[lo:hi])
        send = xe[:nl][torch.from_numpy(L["send_idx"].astype(np.int64))] if i["send_total"] else torch.zeros(1)
        comm.exchange(S, send, xe)
        halo_ok = bool(np.array_equal(xe[nl:].numpy(), xp[L["halo_rows"]]))
        y_ok = bool(np.allclose(M @ xe.numpy(), oracle.spmv(A, x)[n2o][lo:hi], rtol=1e-13, atol=1e-12))
        # ---- CG over the ranks (the communication pattern of ehyb_shard_cg: one exchange of p and the sums
        # of p.q and r.r per iteration), against the oracle's CG on the whole matrix
        b = oracle.spmv(A, gen.uniform(A.n, 23))[n2o][lo:hi]
        xl = np.zeros(nl)
        r = b.copy()
        pe = torch.zeros(nl + i["n_halo"], dtype=torch.float64)
        pe[:nl] = torch.from_numpy(r)
        rr, bb = comm.allreduce([float(r @ r), float(b @ b)])
        hist = [np.sqrt(rr / bb)]
        it = 0
        while hist[-1] > 1e-10 and it < 2000:
            sidx = torch.from_numpy(L["send_idx"].astype(np.int64))
            send = pe[:nl][sidx] if i["send_total"] else torch.zeros(1)
            comm.exchange(S, send, pe)
            q = M @ pe.numpy()
            p = pe[:nl].numpy().copy()
            (pq,) = comm.allreduce([float(p @ q)])
            alpha = rr / pq
            xl += alpha * p
            r -= alpha * q
            (rr_new,) = comm.allreduce([float(r @ r)])
            pe[:nl] = torch.from_numpy(r + (rr_new / rr) * p)
            rr = rr_new
            it += 1
            hist.append(np.sqrt(rr / bb))
        out[rank] = (halo_ok, y_ok, lo, hi, xl, it, hist)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name,port", [(2, "tet", 29611), (4, "tet", 29612), (4, "hex", 29613)])
def test_gloo_ranks_exchange_and_cg(world, name, port):
    out = mp.Manager().dict()
    mp.spawn(_gloo_rank, args=(world, port, name, out), nprocs=world, join=True)
    A = MATS[name]()
    n2o = _plan(A, slice_rows=256).export()["new_to_old"]
    b = oracle.spmv(A, gen.uniform(A.n, 23))
    xo, ok, it_o, rel_o, hist_o = oracle.cg(A, b, rtol=1e-10, max_iter=2000, history=True)
    xg = np.zeros(A.n)
    its = set()
    for r in range(world):
        halo_ok, y_ok, lo, hi, xl, it, hist = out[r]
        assert halo_ok and y_ok, r
        xg[n2o[lo:hi]] = xl
        its.add(it)
    assert len(its) == 1                      # every rank took the same decisions
    (it,) = its
    assert ok and abs(it - it_o) <= 2
    assert np.linalg.norm(b - oracle.spmv(A, xg)) <= 1e-10 * np.linalg.norm(b)
    # the residual histories agree to rounding over the first iterations (on the clamped hex, CG runs in
    # another summation order separate after about 22 iterations, whatever computes them)
    m = min(20, it)
    assert np.allclose(out[0][6][:m], hist_o[:m], rtol=1e-8)


def test_shard_edge_cases():
    import paper_2204_06666_gb300 as eh
    # no rows at all: every rank's shard is empty and has nothing to exchange
    Z = gen.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    P = _plan(Z)
    for r in range(3):
        i = eh.Shard(P, 3, r).info()
        assert i["n_local"] == 0 and i["n_halo"] == 0 and i["send_total"] == 0
    # one row: rank 0 owns it, the others are empty
    one = gen.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.0]))
    P = _plan(one)
    infos = [eh.Shard(P, 4, r).info() for r in range(4)]
    assert sum(i["n_local"] for i in infos) == 1 and all(i["n_halo"] == 0 for i in infos)
    # a rank outside [0, nranks) and a plan with CSR-line extra rows are refused
    A = gen.tet_lap3d(N=6)
    with pytest.raises(eh.EhybError):
        eh.Shard(_plan(A), 2, 2)
    with pytest.raises(eh.EhybError) as e:
        eh.Shard(_plan(A, er_layout=1), 2, 0)
    assert e.value.status == 7
