"""Row shards on the GPU (ehyb_shard_*): every rank's shard runs on the one GPU of this machine.

The ranks are host threads of one process, each on its own CUDA stream.  Their communicator (ThreadComm
below) stands in for NCCL: the halo exchange copies each peer's packed send buffer into the receiver's
x_ext on the device, and the scalar sums add the ranks' values in rank order; the threads meet at host
barriers, never inside a kernel, so no kernel waits on another.  The shards' products concatenated must equal
the plan's product bit for bit (same per-row summation order) and the oracle's within the FP64 bound; the
distributed CG must reach 1e-10 with the residual recomputed by the oracle.
"""
import threading

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


class ThreadComm:
    """Communicator of `world` threads in one process (device-to-device copies, host-side sums)."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)   # a failing rank breaks the barrier, not the test run
        self.send = [None] * world     # (shard, send buffer) of each rank during an exchange
        self.vals = [None] * world

    def bind(self, rank):
        comm = self

        class _Rank:
            def exchange(self, shard, send_buf, x_ext):
                comm.send[rank] = (shard, send_buf)
                torch.cuda.synchronize()
                comm.bar.wait()                         # every rank has packed its send buffer
                nl = shard.n_local
                recv_ptr = np.concatenate([[0], np.cumsum(shard.recv_counts)])
                for q in range(comm.world):
                    if recv_ptr[q + 1] == recv_ptr[q]:
                        continue
                    sq, bq = comm.send[q]
                    sp = np.concatenate([[0], np.cumsum(sq.send_counts)])
                    x_ext[nl + recv_ptr[q]:nl + recv_ptr[q + 1]].copy_(bq[sp[rank]:sp[rank + 1]])
                torch.cuda.synchronize()
                comm.bar.wait()                         # every rank has read the others' buffers

            def allreduce(self, values):
                comm.vals[rank] = list(values)
                comm.bar.wait()
                out = [0.0] * len(values)
                for q in range(comm.world):             # rank order: every rank gets the same bits
                    out = [a + b for a, b in zip(out, comm.vals[q])]
                comm.bar.wait()
                return out
        return _Rank()


def _run_ranks(world, fn):
    errs = [None] * world
    res = [None] * world

    def body(r):
        try:
            torch.cuda.set_device(0)
            with torch.cuda.stream(torch.cuda.Stream()):
                res[r] = fn(r)
        except BaseException as e:      # noqa: BLE001 -- re-raised below
            errs[r] = e
            raise
    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for e in errs:
        if e is not None:
            raise e
    return res


@pytest.mark.parametrize("world", [1, 2, 3, 4])
@pytest.mark.parametrize("name", ["hex", "tet", "ragged_int"])
def test_shard_products_equal_the_plan_bit_for_bit(eh, world, name):
    if name == "hex":
        A = gen.hex_elast3d(N=16)
    elif name == "tet":
        A = gen.tet_lap3d(N=24)
    else:
        A = gen.random_csr(20000, 11, mean_row=10, int_values=True, long_rows=4, long_len=700, empty_frac=0.03)
    P = eh.Plan(A, slice_rows=500)
    n2o = P.export()["new_to_old"]
    x = gen.int_vector(A.n, 2) if name == "ragged_int" else gen.uniform(A.n, 2)
    xp = torch.from_numpy(x[n2o]).cuda()
    yp = torch.empty_like(xp)
    assert eh.ehyb_spmv_permuted(P.handle, xp.data_ptr(), yp.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    comm = ThreadComm(world)

    def rank_fn(r):
        S = eh.Shard(P, world, r)
        c = comm.bind(r)
        xe = torch.zeros(S.n_local + S.n_halo, dtype=torch.float64, device="cuda")
        xe[:S.n_local].copy_(xp[S.row_begin:S.row_end])
        send = torch.zeros(max(S.send_total, 1), dtype=torch.float64, device="cuda")
        S.pack(xe[:S.n_local], send)
        torch.cuda.synchronize()
        c.exchange(S, send, xe)
        y = torch.full((max(S.n_local, 1),), np.nan, dtype=torch.float64, device="cuda")
        if S.n_local:
            S.spmv(xe, y)
        torch.cuda.synchronize()
        assert S.info()["device_status"] == 0
        return S.row_begin, S.row_end, y[:S.n_local].cpu().numpy(), S.n_halo
    out = _run_ranks(world, rank_fn)
    y = np.concatenate([o[2] for o in out])
    assert out[0][0] == 0 and out[-1][1] == A.n
    assert np.array_equal(y, yp.cpu().numpy())                     # the plan's product, bit for bit
    ref = oracle.spmv(A, x)[n2o]
    if name == "ragged_int":
        assert np.array_equal(y, ref)
    else:
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    if world > 1:
        assert sum(o[3] for o in out) > 0                         # the shards did exchange a halo


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("name", ["tet", "hex_clamped"])
def test_shard_cg_reaches_1e10(eh, world, name):
    A = gen.tet_lap3d(N=20) if name == "tet" else gen.hex_elast3d(N=12, clamp_minz=True)
    P = eh.Plan(A, slice_rows=400)
    n2o = P.export()["new_to_old"]
    b = oracle.spmv(A, gen.uniform(A.n, 23))
    bp = torch.from_numpy(b[n2o]).cuda()
    # the single-GPU FP64 CG on the same plan, for the iteration count
    xs = torch.zeros_like(bp)
    st1, info1 = P.cg(torch.from_numpy(b).cuda(), xs, rtol=1e-10, max_iter=5000)
    comm = ThreadComm(world)

    def rank_fn(r):
        S = eh.Shard(P, world, r)
        xl = torch.zeros(max(S.n_local, 1), dtype=torch.float64, device="cuda")
        st, info = S.cg(bp[S.row_begin:S.row_end].contiguous(), xl, comm.bind(r), rtol=1e-10, max_iter=5000)
        torch.cuda.synchronize()
        return st, info, S.row_begin, S.row_end, xl[:S.n_local].cpu().numpy()
    out = _run_ranks(world, rank_fn)
    x = np.zeros(A.n)
    for st, info, lo, hi, xl in out:
        assert st == 0 and info["converged"] == 1
        x[n2o[lo:hi]] = xl
    assert len({o[1]["iterations"] for o in out}) == 1             # every rank took the same decisions
    its = out[0][1]["iterations"]
    assert abs(its - info1["iterations"]) <= max(3, info1["iterations"] // 50)
    rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert rel <= 1e-10 and abs(out[0][1]["relres"] - rel) <= 1e-12


def test_shard_errors(eh):
    A = gen.tet_lap3d(N=8)
    P = eh.Plan(A)
    with pytest.raises(eh.EhybError) as e:
        eh.Shard(P, 2, 2)
    assert e.value.status == 1
    Q = eh.Plan(A, er_layout=1)
    with pytest.raises(eh.EhybError) as e:
        eh.Shard(Q, 2, 0)
    assert e.value.status == 7
