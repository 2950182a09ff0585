"""GPU parity of the EHYB SpMV (C ABI) against the CPU oracle.

Bars: bit-exact on integer-valued inputs (every partial sum is an exact integer in FP64, so the
summation order cannot matter); on FEM inputs rel-L2 <= 1e-13 AND, row by row,
|y_gpu - y_oracle| <= 2 gamma_{k+6} (|A||x|)_i with u = 2^-53 -- the recursive-summation bound of
both sides (k = row length; +6 covers the shuffle-reduction depth and the slab + ER combination).
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


def _run(eh, A, x, **opt):
    P = eh.Plan(A, **opt)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, np.nan)
    P.spmv(xd, yd)
    torch.cuda.synchronize()
    assert P.check() == 0
    return P, yd.cpu().numpy()


def _row_bound(A, x):
    k = np.diff(A.row_ptr).astype(np.float64)
    return 2 * oracle.gamma(k + 6) * oracle.abs_spmv(A, x)


def _check_fp(A, x, y):
    ref = oracle.spmv(A, x)
    err = np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-300)
    assert err <= 1e-13, err
    assert np.all(np.abs(y - ref) <= _row_bound(A, x)), np.max(np.abs(y - ref) - _row_bound(A, x))
    return err


OPTS = [dict(), dict(ell_tpr=2), dict(ell_tpr=4), dict(ell_tpr=32), dict(ell_width_cap=6),
        dict(slice_rows=37, block_threads=64), dict(slice_rows=1), dict(slice_rows=2000, block_threads=1024),
        dict(slice_rows=33, block_threads=32),
        dict(er_layout=1, ell_tpr=2, er_tpr=1), dict(er_layout=1, ell_tpr=4, er_tpr=32),
        dict(er_layout=1, ell_tpr=32, er_tpr=8), dict(er_layout=1, ell_width_cap=6, er_tpr=4),
        dict(er_layout=1, slice_rows=37, block_threads=64),
        dict(er_layout=2), dict(er_layout=2, ell_tpr=4), dict(er_layout=2, ell_width_cap=6, slice_rows=300),
        dict(er_layout=2, slice_rows=1), dict(er_layout=2, slice_rows=33, block_threads=32)]


@pytest.mark.parametrize("opt", OPTS)
@pytest.mark.parametrize("seed", [0, 1])
def test_integer_bit_exact_ragged(eh, opt, seed):
    A = gen.random_csr(3001 + seed, seed, mean_row=11, int_values=True, empty_frac=0.05, long_rows=5,
                       long_len=1500, duplicates=True)
    x = gen.int_vector(A.n, seed + 100)
    _, y = _run(eh, A, x, **opt)
    assert np.array_equal(y, oracle.spmv(A, x))


@pytest.mark.parametrize("slice_rows", [28922, 4000])
def test_integer_bit_exact_with_and_without_slice_table(eh, slice_rows):
    # 28,922 rows (the largest partition the tuner offers): the FP64 slice of x takes 231,392 of the block's
    # 231,424 bytes of shared memory, so the launch has no room for the partition's slice table (904 slices
    # x 32 B) and reads each slice's position from global memory; with 4,000 rows the table is staged.  Both
    # must give the oracle's sums exactly.
    A = gen.random_csr(61000, 9, mean_row=10, int_values=True, empty_frac=0.05, long_rows=3, long_len=700,
                       duplicates=True)
    x = gen.int_vector(A.n, 109)
    P, y = _run(eh, A, x, slice_rows=slice_rows)
    assert P.info()["slice_rows"] == slice_rows
    assert np.array_equal(y, oracle.spmv(A, x))


@pytest.mark.parametrize("er_layout", [0, 1, 2])
@pytest.mark.parametrize("name,N,slice_rows", [("fem2d", 200, 0), ("hex", 16, 0), ("hex", 16, 700),
                                               ("tet", 20, 0), ("tet", 20, 1000)])
def test_fem_parity(eh, name, N, slice_rows, er_layout):
    A = {"fem2d": gen.fem2d_p1, "hex": gen.hex_elast3d, "tet": gen.tet_lap3d}[name](N=N)
    x = gen.uniform(A.n, 13)
    _, y = _run(eh, A, x, slice_rows=slice_rows, er_layout=er_layout)
    _check_fp(A, x, y)


def test_hex70_full_size_as_benchmarked(eh):
    # the benchmarked workload, default plan (Eq. 1) and launch configuration
    A = gen.hex_elast3d()
    x = gen.uniform(A.n, 13)
    P, y = _run(eh, A, x)
    err = _check_fp(A, x, y)
    info = P.info()
    assert info["nparts"] == 152 and info["device_status"] == 0
    # run-to-run bit reproducibility
    xd = torch.from_numpy(x).cuda()
    y2 = torch.empty_like(xd)
    for _ in range(3):
        P.spmv(xd, y2)
    torch.cuda.synchronize()
    assert np.array_equal(y2.cpu().numpy(), y)
    assert err <= 1e-13


def test_tet126_full_size(eh):
    A = gen.tet_lap3d()
    x = gen.uniform(A.n, 23)
    _, y = _run(eh, A, x)
    _check_fp(A, x, y)
    # the halo layout: the extra entries after each row's own in the slab slices, x staged at the halo; every
    # row summed in the same slot order, so the same bits
    P2, y2 = _run(eh, A, x, er_layout=2)
    assert P2.info()["er_layout"] == 2 and P2.info()["n_halo"] > 0
    assert np.array_equal(y2, y)


@pytest.mark.parametrize("name", ["tet126", "hex70"])
def test_lowp_full_size_as_benchmarked(eh, name):
    # the FP32 / BF16 products of the mixed-precision solvers on the benchmarked workloads, in the automatic
    # layout (runs of four held packed) and launch configuration that bench.py --lowp times: every row within
    # the FP32 rounding bound of the oracle's product with the same rounded values and x
    A = gen.tet_lap3d() if name == "tet126" else gen.hex_elast3d()
    x = gen.uniform(A.n, 29)
    k = np.diff(A.row_ptr).astype(np.float64)
    bound = 2 * oracle.gamma(k + 6, 2.0 ** -24) * oracle.abs_spmv(A, x)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    for lowp in (1, 2):
        P = eh.Plan(A, lowp=lowp)
        assert P.info()["lowp_group"] == 4
        yd = torch.full_like(xd, np.nan)
        P.spmv_lowp(xd, yd)
        torch.cuda.synchronize()
        assert P.check() == 0
        y = yd.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - oracle.spmv_low(A, x, bf16=(lowp == 2))) <= bound), lowp
        del P


@pytest.mark.parametrize("make", [lambda: gen.tet_lap3d(N=30), lambda: gen.hex_elast3d(N=16),
                                  lambda: gen.fem2d_p1(N=150),
                                  lambda: gen.random_csr(5000, 3, mean_row=12, empty_frac=0.05, long_rows=4,
                                                         long_len=1200, duplicates=True)],
                         ids=["tet", "hex", "fem2d", "ragged"])
@pytest.mark.parametrize("slice_rows", [0, 500])
def test_halo_layout_bit_identical_to_sliced(eh, make, slice_rows):
    # er_layout 2 against er_layout 0 on the same partition: the fused-permutation entry, the plan-numbering
    # entry, the allocation-free entry and the FP32 / BF16 products give the same bits
    A = make()
    x = gen.uniform(A.n, 31)
    out = {}
    for lay in (0, 2):
        P = eh.Plan(A, slice_rows=slice_rows, er_layout=lay, lowp=1)
        P16 = eh.Plan(A, slice_rows=slice_rows, er_layout=lay, lowp=2)
        xd = torch.from_numpy(x).cuda()
        y = torch.full_like(xd, np.nan)
        P.spmv(xd, y)
        xp, yp = torch.empty_like(xd), torch.full_like(xd, np.nan)
        P.permute(True, xd, xp)
        P.spmv_permuted(xp, yp)
        yn = torch.full_like(xd, np.nan)
        P.spmv_noalloc(xd, yn)
        x32 = xd.float()
        y32, y16 = torch.full_like(x32, np.nan), torch.full_like(x32, np.nan)
        P.spmv_lowp(x32, y32)
        P16.spmv_lowp(x32, y16)
        torch.cuda.synchronize()
        assert P.check() == 0 and P16.check() == 0
        out[lay] = [t.cpu().numpy() for t in (y, yp, yn, y32, y16)]
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a, b)
    _check_fp(A, x, out[2][0])


def test_halo_layout_cg_matches_sliced(eh):
    # the CG's fused p.q runs in the same kernel epilogue: identical residual histories
    A = gen.tet_lap3d(N=24)
    b = torch.from_numpy(oracle.spmv(A, gen.uniform(A.n, 5))).cuda()
    hist = {}
    for lay in (0, 2):
        P = eh.Plan(A, er_layout=lay)
        x = torch.zeros_like(b)
        st, info = P.cg(b, x, rtol=1e-10)
        assert st == 0, info
        hist[lay] = (P.cg_history(info["iterations"]), x.cpu().numpy())
    assert np.array_equal(hist[0][0], hist[2][0]) and np.array_equal(hist[0][1], hist[2][1])


def test_halo_layout_unsupported_paths(eh):
    A = gen.tet_lap3d(N=12)
    P = eh.Plan(A, er_layout=2)
    with pytest.raises(eh.EhybError):
        P.spmm(torch.zeros(A.n, 8, dtype=torch.float64, device="cuda"), torch.zeros(A.n, 8, dtype=torch.float64,
                                                                                     device="cuda"))
    with pytest.raises(eh.EhybError):
        eh.Batch([P])
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        with pytest.raises(eh.EhybError):
            P.save(os.path.join(d, "p.ehyb"))


@pytest.mark.parametrize("name", ["hex", "tet", "powerlaw", "ragged_int"])
def test_multilevel_partition_parity(eh, name):
    # plans whose PartVec comes from the multilevel partitioner (equal parts, supervariables split across parts)
    if name == "ragged_int":
        A = gen.random_csr(3001, 4, mean_row=11, int_values=True, empty_frac=0.05, long_rows=5, long_len=1500,
                           duplicates=True)
        x = gen.int_vector(A.n, 104)
        _, y = _run(eh, A, x, partitioner=1, slice_rows=37, block_threads=64)
        assert np.array_equal(y, oracle.spmv(A, x))
        return
    A = {"hex": lambda: gen.hex_elast3d(N=16), "tet": lambda: gen.tet_lap3d(N=20),
         "powerlaw": lambda: gen.tuner_matrix(1)}[name]()
    x = gen.uniform(A.n, 13)
    P, y = _run(eh, A, x, partitioner=1)
    _check_fp(A, x, y)
    G = eh.Plan(A)
    assert P.info()["er_nnz"] < G.info()["er_nnz"]


def test_multilevel_hex70_full_size(eh):
    A = gen.hex_elast3d()
    x = gen.uniform(A.n, 13)
    P, y = _run(eh, A, x, partitioner=1)
    _check_fp(A, x, y)
    info = P.info()
    assert info["nparts"] == 152 and info["er_nnz"] < 0.135 * A.nnz


def test_permuted_entry_and_permute(eh):
    A = gen.hex_elast3d(N=10)
    x = gen.uniform(A.n, 5)
    P, y = _run(eh, A, x, slice_rows=500)
    n2o = P.export()["new_to_old"]
    xd = torch.from_numpy(x).cuda()
    xp = torch.empty_like(xd)
    P.permute(True, xd, xp)
    assert np.array_equal(xp.cpu().numpy(), x[n2o])
    yp = torch.empty_like(xd)
    P.spmv_permuted(xp, yp)
    back = torch.empty_like(xd)
    P.permute(False, yp, back)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), y)
    # an x that is not 16-byte aligned takes the plain-load staging path and gives the same bits
    big = torch.zeros(A.n + 1, dtype=torch.float64, device="cuda")
    big[1:] = xp
    yp2 = torch.empty_like(xd)
    P.spmv_permuted(big[1:], yp2)
    torch.cuda.synchronize()
    assert np.array_equal(yp2.cpu().numpy(), yp.cpu().numpy())


@pytest.mark.parametrize("opt", [dict(), dict(ell_tpr=4, slice_rows=300), dict(er_layout=1)])
def test_fused_permutation_matches_permute_then_plan_numbering(eh, opt):
    # ehyb_spmv reads x through new_to_old while staging (sliced ER) and must give the bits of the
    # explicit route permute -> plan-numbering SpMV -> permute back, also for an x that is not 16-byte aligned
    A = gen.tet_lap3d(N=18, dirichlet=False)
    x = gen.uniform(A.n, 77)
    P, y = _run(eh, A, x, **opt)
    xd = torch.from_numpy(x).cuda()
    xp, yp, back = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
    P.permute(True, xd, xp)
    P.spmv_permuted(xp, yp)
    P.permute(False, yp, back)
    big = torch.zeros(A.n + 1, dtype=torch.float64, device="cuda")
    big[1:] = xd
    y2 = torch.empty_like(xd)
    P.spmv(big[1:], y2)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), y)
    assert np.array_equal(y2.cpu().numpy(), y)
    _check_fp(A, x, y)


def test_back_to_back_launches_respect_the_stream_order(eh):
    # consecutive launches may be scheduled early (programmatic dependent launch): a chain in which each
    # SpMV reads the previous one's output, with no host synchronisation, must still see finished inputs
    A = gen.hex_elast3d(N=14)
    x = gen.uniform(A.n, 3)
    P = eh.Plan(A)
    v = [torch.from_numpy(x).cuda()] + [torch.empty(A.n, dtype=torch.float64, device="cuda") for _ in range(6)]
    for k in range(6):
        P.spmv(v[k], v[k + 1])
    xp = [torch.empty_like(v[0]) for _ in range(4)]
    P.permute(True, v[6], xp[0])
    for k in range(3):
        P.spmv_permuted(xp[k], xp[k + 1])
    back = torch.empty_like(v[0])
    P.permute(False, xp[3], back)
    torch.cuda.synchronize()
    ref = x.copy()
    for k in range(6):
        ref = oracle.spmv(A, ref)
        got = v[k + 1].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), k
    for k in range(3):
        ref = oracle.spmv(A, ref)
    assert np.linalg.norm(back.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


def test_host_entry_matches_device_entry(eh):
    A = gen.fem2d_p1(N=80)
    x = gen.uniform(A.n, 9)
    P, y = _run(eh, A, x)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    P.spmv_host(xh, yh)
    assert np.array_equal(yh.numpy(), y)
    yn = np.zeros(A.n)
    P.spmv_host(np.ascontiguousarray(x), yn)   # pageable numpy buffers work too
    assert np.array_equal(yn, y)


@pytest.mark.parametrize("count", [1, 2, 5])
def test_pipelined_host_entry_matches_device_entry(eh, count):
    # x_{i+1} in and y_{i-1} out overlap product i; each result must equal the device entry's bits
    A = gen.hex_elast3d(N=12)
    P = eh.Plan(A)
    xs = [torch.from_numpy(gen.uniform(A.n, 40 + i)).pin_memory() for i in range(count)]
    ys = [torch.full((A.n,), np.nan, dtype=torch.float64).pin_memory() for _ in range(count)]
    P.spmv_host_many(xs, ys)
    for i in range(count):
        xd = xs[i].cuda()
        yd = torch.empty_like(xd)
        P.spmv(xd, yd)
        torch.cuda.synchronize()
        assert np.array_equal(ys[i].numpy(), yd.cpu().numpy()), i
        _check_fp(A, xs[i].numpy(), ys[i].numpy())
    outs = [torch.empty_like(xs[0]).pin_memory() for _ in range(3)]
    P.spmv_host_many([xs[0]] * 3, outs)                                # one input three times
    assert all(np.array_equal(o.numpy(), outs[0].numpy()) for o in outs)
    P.spmv_host_many([], [])                                            # count 0: nothing to do
    import ctypes
    null = (ctypes.c_void_p * 1)(None)
    assert eh._lib.ehyb_spmv_host_many(P._h, 1, null, null, None) == 1  # a NULL entry: EHYB_ERR_INVALID_ARG


@pytest.mark.parametrize("lowp", [1, 2])
def test_lowp_integer_exact_and_fem_bound(eh, lowp):
    A = gen.random_csr(2000, 4, mean_row=12, int_values=True, empty_frac=0.05, long_rows=2, long_len=600)
    x = gen.int_vector(A.n, 6)
    P = eh.Plan(A, lowp=lowp, slice_rows=300)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty_like(xd)
    P.spmv_lowp(xd, yd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy().astype(np.float64), oracle.spmv(A, x))
    B = gen.tet_lap3d(N=20)
    xb = gen.uniform(B.n, 3)
    P = eh.Plan(B, lowp=lowp)
    xd = torch.from_numpy(xb.astype(np.float32)).cuda()
    yd = torch.empty_like(xd)
    P.spmv_lowp(xd, yd)
    torch.cuda.synchronize()
    ref = oracle.spmv_low(B, xb, bf16=(lowp == 2))
    k = np.diff(B.row_ptr).astype(np.float64)
    bound = 2 * oracle.gamma(k + 6, 2.0 ** -24) * oracle.abs_spmv(B, xb)
    assert np.all(np.abs(yd.cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("lowp", [1, 2])
@pytest.mark.parametrize("make", [lambda: gen.hex_elast3d(N=14), lambda: gen.tet_lap3d(N=20),
                                  lambda: gen.random_csr(3000, 7, mean_row=40, int_values=True, long_rows=3,
                                                         long_len=900, empty_frac=0.02)],
                         ids=["hex", "tet", "ragged_int"])
def test_lowp_runs_layout_bit_identical_to_column_major(eh, lowp, make):
    # the copies in runs of four slots (lowp_group 4) sum every row in the same slot order as the column-major
    # copies (lowp_group 1): identical bits, for the fused-permutation entry and inside the FP32 CG
    A = make()
    x = gen.uniform(A.n, 4).astype(np.float32)
    out = {}
    for grp in (1, 4):
        P = eh.Plan(A, lowp=lowp, lowp_group=grp, slice_rows=400)
        assert P.info()["lowp_group"] == grp
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, np.nan)
        P.spmv_lowp(xd, yd)
        torch.cuda.synchronize()
        assert P.check() == 0
        out[grp] = yd.cpu().numpy()
    assert np.array_equal(out[1], out[4])


def test_lowp_group_auto(eh):
    # the sliced and halo extra-row layouts get the copies in runs of four, wide (elasticity) and narrow (tet)
    # slices alike; the CSR-line layout keeps column-major copies
    assert eh.Plan(gen.hex_elast3d(N=14), lowp=2).info()["lowp_group"] == 4
    assert eh.Plan(gen.tet_lap3d(N=20), lowp=2).info()["lowp_group"] == 4
    assert eh.Plan(gen.hex_elast3d(N=14), lowp=2, er_layout=1).info()["lowp_group"] == 1
    assert eh.Plan(gen.tet_lap3d(N=20), lowp=1, er_layout=2).info()["lowp_group"] == 4
    with pytest.raises(eh.EhybError) as e:
        eh.Plan(gen.tet_lap3d(N=8), lowp=1, lowp_group=2)
    assert e.value.status == 1


def test_lowp_requires_lowp_plan(eh):
    A = gen.fem2d_p1(N=20)
    P = eh.Plan(A)
    x = torch.zeros(A.n, dtype=torch.float32, device="cuda")
    with pytest.raises(eh.EhybError) as e:
        P.spmv_lowp(x, torch.empty_like(x))
    assert e.value.status == 7


@pytest.mark.parametrize("tpr", [1, 2, 4, 8, 32])
def test_csr_baseline_parity(eh, tpr):
    A = gen.random_csr(2500, 8, mean_row=10, int_values=True, empty_frac=0.05, long_rows=3, long_len=900,
                       duplicates=True)
    x = gen.int_vector(A.n, 1)
    M = eh.CsrBaseline(A, tpr=tpr)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    M.spmv(xd, yd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), oracle.spmv(A, x))
    B = gen.hex_elast3d(N=12)
    xb = gen.uniform(B.n, 2)
    M = eh.CsrBaseline(B, tpr=tpr)
    xd = torch.from_numpy(xb).cuda()
    yd = torch.empty_like(xd)
    M.spmv(xd, yd)
    torch.cuda.synchronize()
    _check_fp(B, xb, yd.cpu().numpy())


@pytest.mark.parametrize("er_layout", [0, 2])
def test_edge_cases(eh, er_layout):
    for n in (1, 2, 31, 32, 33, 65):
        A = gen.random_csr(n, n, mean_row=3, int_values=True, empty_frac=0.3)
        x = gen.int_vector(n, n)
        _, y = _run(eh, A, x, slice_rows=16, er_layout=er_layout)
        assert np.array_equal(y, oracle.spmv(A, x)), n
    Z = gen.CSR(40, np.zeros(41, np.int64), np.zeros(0, np.int32), np.zeros(0))   # no entries at all
    _, y = _run(eh, Z, np.ones(40), er_layout=er_layout)
    assert np.all(y == 0)
    E = gen.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    P = eh.Plan(E, er_layout=er_layout)
    P.spmv(torch.zeros(1, dtype=torch.float64, device="cuda")[:0], torch.zeros(1, dtype=torch.float64, device="cuda")[:0])
    assert P.check() == 0
    # every row's entries outside its one-row partition: the halo holds all of them
    n = 64
    rp = np.arange(n + 1, dtype=np.int64) * 3
    col = np.stack([(np.arange(n) + k) % n for k in (7, 19, 41)], axis=1).ravel().astype(np.int32)
    D = gen.CSR(n, rp, col, np.arange(1, 3 * n + 1, dtype=np.float64))
    x = gen.int_vector(n, 3)
    P, y = _run(eh, D, x, slice_rows=1, er_layout=er_layout)
    assert np.array_equal(y, oracle.spmv(D, x))
    if er_layout == 2:
        assert P.info()["n_halo"] == 3 * n and P.info()["max_stage_rows"] == 4


def test_staging_wait_timeout_is_reported_and_context_survives(eh):
    A = gen.fem2d_p1(N=30)
    x = gen.uniform(A.n, 1)
    # the wait is given a copy that is never issued: it must run out after 2 ms and report (the bulk
    # staging copy is the one of the plan-numbering entry; ehyb_spmv gathers x with plain loads)
    P = eh.Plan(A, slice_rows=100, inject_wait_fault=1, wait_timeout_ns=2_000_000)
    xd = torch.from_numpy(x).cuda()
    xp = torch.empty_like(xd)
    P.permute(True, xd, xp)
    yd = torch.zeros_like(xd)
    P.spmv_permuted(xp, yd)
    assert P.check() == eh.EHYB_ERR_TIMEOUT
    assert P.check() == 0   # reading clears the word
    # the context is intact: a normal plan still computes correctly
    Q, y = _run(eh, A, x, slice_rows=100)
    _check_fp(A, x, y)


def test_oom_hook(eh):
    A = gen.fem2d_p1(N=30)
    eh.ehyb_test_fail_allocs_after(0)
    try:
        with pytest.raises(eh.EhybError) as e:
            eh.Plan(A)
        assert e.value.status == 5
    finally:
        eh.ehyb_test_fail_allocs_after(-1)
    eh.Plan(A)


def test_profile_counts_main_kernel(eh):
    A = gen.fem2d_p1(N=50)
    P = eh.Plan(A)
    xd = torch.from_numpy(gen.uniform(A.n, 1)).cuda()
    yd = torch.empty_like(xd)
    P.profile_enable(True)
    for _ in range(5):
        P.spmv(xd, yd)
    ms, cnt = P.profile_read()
    assert cnt == 5 and ms > 0
