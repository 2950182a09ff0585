#!/usr/bin/env python3
"""EHYB FP64 SpMV benchmark on GB300.

One step = one y = A x through the C ABI (ehyb_spmv: one fused launch that gathers x through the
permutation into shared memory, runs the slab and the ER entries and writes y in the original
numbering) on the 3D Q1 hex elasticity matrix (70^3 nodes x 3 dof: n = 1,029,000,
nnz = 80,990,208), x ~ U[-1, 1) seeded.

Prints ONE JSON line (rank 0).  value = whole-job GFLOP/s (2 nnz per SpMV, padding excluded)
timed with CUDA events on the launching stream.  A workload larger than L2 (the 3D meshes) runs
back to back; one that fits L2 (the 2D mesh) is timed cold, a 512 MB write before every step,
with the warm time in `warm`.  Also reported:
  * roofline of the fused kernel (achieved / peak, the bound, DRAM traffic from the committed
    ncu record while the kernel sources and the plan's layout match it); the FP64 roof is the FMA
    rate ehyb_fp64_fma_peak measures on the device after the timed region;
  * long_window: when fewer than 200 steps are requested, the same product over 2000 more steps;
  * plan_numbering: the same product with x and y kept in the plan's numbering (ehyb_spmv_permuted, the
    form a solver iterates in; the permutations happen once, outside the window), back to back, and
    whether its result permuted back equals the fused entry's bit for bit;
  * the plain vector-CSR kernel on the same GPU (original and EHYB-reordered row order, best
    lanes-per-row of 1..32);
  * preprocessing (plan build) time as a multiple of one SpMV;
  * e2e: the same metric through the host-vector entries, x copied in and y out every step:
    ehyb_spmv_host_many (copies overlapping neighbouring products) and, under `sync`, one
    synchronous ehyb_spmv_host call per step;
  * cpu_baseline: the CPU oracle (plain C CSR SpMV) on one core over a bounded row sample, and
    under `multicore` whole products split over every host core.

Other modes: --partitioner 1 (multilevel partition), --lowp (FP32 / BF16 SpMVs), --solver (CG,
mixed precision, flexible CG, FSAI-PCG to 1e-10), --transient (implicit time steps reusing one plan),
--batch, --spmm, --plan-io, --shard (row shards with a halo exchange per product across the torchrun
ranks: strong scaling of one matrix).  --impl reference times the oracle on the host cores as the reference
arm (there is no runnable reference code).  Multi-GPU (torchrun): by default independent replicas, one
full product per rank (weak scaling, max time over ranks); with --shard one matrix split into row shards,
its halo moved by an NCCL all-to-all every product (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EHYB SpMV GFLOP/s & % of HBM roofline vs plain CSR kernel on same GB300"
HBM_FALLBACK_GBS = 6800.0
# FP64 FMA pipe, nominal: 2 DFMA/clk/SM x 2 flops x 152 SMs x 2.07 GHz (context only: the roofline of the
# FP64 kernels is taken against the rate ehyb_fp64_fma_peak measures on the device at hand)
FP64_NOMINAL_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
LONG_WINDOW_STEPS = 2000  # a requested window shorter than 200 steps is repeated over this many steps too

WORKLOADS = {
    "hex_elast3d_70": dict(kind="hex", N=70, seed_x=13,
                           desc="3D Q1 hex elasticity, 70^3 nodes x 3 dof, jitter 0.2h, node relabelling"),
    "hex_elast3d_48": dict(kind="hex", N=48, seed_x=13,
                           desc="3D Q1 hex elasticity, 48^3 nodes x 3 dof (profiling size, 0.27 GB slab)"),
    "fem2d_p1_200": dict(kind="fem2d", N=200, seed_x=3, desc="2D P1 Laplacian, 200^2 nodes, jitter 0.3h"),
    "tet_lap3d_126": dict(kind="tet", N=126, seed_x=23, desc="3D P1 tet Laplacian, 126^3 nodes, Dirichlet"),
    "hex_elast3d_70_clamped": dict(kind="hex", N=70, seed_x=24, clamp=True,
                                   desc="3D Q1 hex elasticity, 70^3 nodes x 3 dof, min-z face clamped (SPD)"),
}


def make_matrix(w):
    import gen
    if w["kind"] == "hex":
        return gen.hex_elast3d(N=w["N"], clamp_minz=w.get("clamp", False))
    if w["kind"] == "fem2d":
        return gen.fem2d_p1(N=w["N"])
    return gen.tet_lap3d(N=w["N"])


FLUSH_BYTES = 512 << 20  # written before each timed step of an L2-resident workload


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            time.sleep(0.15)
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if len(r) > 3 and r[3].strip()[:1].isdigit())
                if rows else None}


def cpu_multicore(A, x, budget_s: float = 5.0):
    """The same oracle routine on every host core: whole SpMVs, row range t of T on thread t (the C call
    releases the interpreter lock), repeated until budget."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    n, T = A.n, max(1, os.cpu_count() or 1)
    y = np.zeros(n)
    cuts = [n * t // T for t in range(T + 1)]
    passes = 0
    with ThreadPoolExecutor(T) as ex:
        t0 = time.perf_counter()
        while passes == 0 or time.perf_counter() - t0 < budget_s:
            list(ex.map(lambda t: oracle.spmv_rows(A, x, cuts[t], cuts[t + 1], y), range(T)))
            passes += 1
        dt = time.perf_counter() - t0
    return {"value": 2.0 * A.nnz * passes / dt / 1e9, "unit": "GFLOP/s", "cores": T, "kind": "oracle",
            "sample": f"{passes} whole SpMVs, rows split over {T} threads ({dt:.1f} s)"}


def cpu_baseline(A, x, budget_s: float = 10.0, y_gpu=None):
    """The oracle CSR SpMV (plain C, one thread) on a bounded sample: whole row blocks until budget.  With the
    GPU result y_gpu, also the relative L2 error of y_gpu on the rows the oracle computed."""
    import oracle
    n = A.n
    y = np.zeros(n)
    done = np.zeros(n, bool)
    block = max(1, n // 16)
    t0 = time.perf_counter()
    rows = flops = 0
    r = 0
    while time.perf_counter() - t0 < budget_s:
        r1 = min(n, r + block)
        oracle.spmv_rows(A, x, r, r1, y)
        done[r:r1] = True
        flops += 2 * int(A.row_ptr[r1] - A.row_ptr[r])
        rows += r1 - r
        r = 0 if r1 >= n else r1
    dt = time.perf_counter() - t0
    out = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
           "sample": f"{rows} rows in blocks of {block} of the same matrix (plain C CSR, 1 thread, {dt:.1f} s)"}
    out["multicore"] = cpu_multicore(A, x, budget_s / 2)
    if y_gpu is not None:
        ref = y[done]
        out["parity"] = {"rows_checked": int(done.sum()),
                         "rel_l2": float(np.linalg.norm(y_gpu[done] - ref) / max(np.linalg.norm(ref), 1e-300)),
                         "tolerance": 1e-13}
    return out


KERNEL_SOURCES = ("paper_2204_06666_gb300/csrc/ehyb_core.cuh", "paper_2204_06666_gb300/csrc/spmv_kernels.cu")


def kernel_source_sha() -> str:
    """Hash of the sources of the fused kernel and its launch."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def layout_signature(info: dict) -> str:
    """The plan's byte layout as the kernel reads it: partitions, slices, stored slab and ER slots, ER entries."""
    return "/".join(str(info[k]) for k in ("nparts", "nslices", "ell_stored", "er_stored", "er_nnz"))


def recorded_traffic(workload: str, layout: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu capture, or None when the kernel's
    sources or the plan's layout differ from the captured ones (or no capture exists for this workload)."""
    p = os.path.join(ROOT, "profiles", "ehyb_kernel_dram.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        rec = json.load(f)
    r = rec.get(workload)
    if not r or r.get("source_sha") != kernel_source_sha() or r.get("layout") != layout:
        return None, None
    return float(r["dram_bytes_per_launch"]), r.get("note")


def _busy(stream, cycles: int = 4_000_000):
    """Queue about 2 ms of device-side waiting on `stream` before a timed window's start event, so the GPU is
    still busy while the host enqueues the event and the window's first launches: otherwise an idle stream
    puts the host's launch latency of the first kernel inside the window.  Nothing of the window's work runs
    before its start event."""
    import torch
    if hasattr(torch.cuda, "_sleep"):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(cycles)


def aggregate(local_ms: float, world: int, units_per_rank: float, reduce_max=None):
    """Whole-job throughput: the max of the ranks' times, all ranks' units.  reduce_max(x) returns the max of
    x over ranks (identity for one rank).  Returns (value in units/s, max ms)."""
    ms_max = reduce_max(local_ms) if reduce_max else local_ms
    return units_per_rank * world / (ms_max / 1e3), ms_max


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    w = WORKLOADS[args.workload]
    A = make_matrix(w)
    import gen
    x = gen.uniform(A.n, w["seed_x"])
    y = np.zeros(A.n)
    oracle.build()
    # each step: one contiguous row block of the matrix, split over every host core (the oracle's C routine
    # on threads; the call releases the interpreter lock), sized so the whole run takes about 60 s
    from concurrent.futures import ThreadPoolExecutor
    T = max(1, os.cpu_count() or 1)
    steps = args.steps + args.warmup
    t0 = time.perf_counter()
    oracle.spmv_rows(A, x, 0, min(A.n, 4096), y)
    per_row = (time.perf_counter() - t0) / min(A.n, 4096)
    rows_per_step = int(max(64 * T, min(A.n, 60.0 * T / max(steps, 1) / max(per_row, 1e-9))))
    # threads only where a step has work for them (about 500k entries each): thread dispatch would dominate
    # the small 2D matrix
    T = int(max(1, min(T, (A.nnz * rows_per_step // max(A.n, 1)) // 500000)))
    r = 0
    flops = 0
    t_total = 0.0
    with ThreadPoolExecutor(T) as ex:
        for i in range(steps):
            r1 = min(A.n, r + rows_per_step)
            cuts = [r + (r1 - r) * t // T for t in range(T + 1)]
            t = time.perf_counter()
            list(ex.map(lambda k: oracle.spmv_rows(A, x, cuts[k], cuts[k + 1], y), range(T)))
            dt = time.perf_counter() - t
            if i >= args.warmup:
                t_total += dt
                flops += 2 * int(A.row_ptr[r1] - A.row_ptr[r])
            r = 0 if r1 >= A.n else r1
    value = flops / t_total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "desc": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": T, "kind": "oracle",
                             "sample": f"row blocks of {rows_per_step} rows per step (plain C CSR, rows split "
                                       f"over {T} thread{'s' if T > 1 else ''})"},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ehyb(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import gen
    import paper_2204_06666_gb300 as eh

    w = WORKLOADS[args.workload]
    A = make_matrix(w)
    x = gen.uniform(A.n, w["seed_x"])
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = eh.Plan(A, partitioner=args.partitioner, er_layout=args.er_layout, slice_rows=args.slice_rows,
                   block_threads=args.block_threads)
    plan_ms = (time.perf_counter() - t0) * 1e3
    info = plan.info()
    xd = torch.from_numpy(x).to(dev)
    yd = torch.empty_like(xd)
    flops_per_step = 2.0 * A.nnz

    for _ in range(args.warmup):
        plan.spmv(xd, yd)
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the launching stream).  A workload larger than L2 runs
    # back to back; one that fits L2 is timed cold: before every step a 512 MB write evicts the plan, x and y
    # from L2, and only the SpMV between its two events counts (the warm back-to-back time is kept beside it)
    l2_bytes = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 128 << 20)
    l2_resident = float(info["bytes_effective"]) <= l2_bytes
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    warm = None
    if l2_resident:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            plan.spmv(xd, yd)
        e1.record(stream)
        torch.cuda.synchronize()
        warm_ms = e0.elapsed_time(e1) / args.steps
        warm = {"ms_per_step": warm_ms, "value": flops_per_step / (warm_ms / 1e3) / 1e9}
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        if l2_resident:
            for i in range(args.steps):
                flush.fill_(i & 255)
                evs[i][0].record(stream)
                plan.spmv(xd, yd)
                evs[i][1].record(stream)
        else:
            _busy(stream)
            e0.record(stream)
            for _ in range(args.steps):
                plan.spmv(xd, yd)
            e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs) if l2_resident else e0.elapsed_time(e1)
    clocks = clk.summary()
    # a short requested window (20 steps of the hex product are about 3 ms) is repeated over a long one, so
    # the spread of the requested window's figure can be read beside it; the line's value stays the requested
    # window's
    long_window = None
    if args.steps < 200 and not l2_resident:
        with ClockSampler(local) as clk_long:
            torch.cuda.synchronize()
            _busy(stream)
            e0.record(stream)
            for _ in range(LONG_WINDOW_STEPS):
                plan.spmv(xd, yd)
            e1.record(stream)
            torch.cuda.synchronize()
        lw_ms = e0.elapsed_time(e1) / LONG_WINDOW_STEPS
        long_window = {"steps": LONG_WINDOW_STEPS, "ms_per_step": lw_ms,
                       "value": flops_per_step / (lw_ms / 1e3) / 1e9, "clocks": clk_long.summary()}
    # the same product in the plan numbering (ehyb_spmv_permuted: x and y permuted once, outside the window, as
    # a solver keeps its vectors): back to back beside the line's caller's-numbering figure, and its result,
    # permuted back, compared bit for bit with the fused entry's
    plan_numbering = None
    if not l2_resident:
        xp, yp, yb = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
        plan.permute(True, xd, xp)
        for _ in range(max(3, args.warmup)):
            plan.spmv_permuted(xp, yp)
        pn_steps = args.steps if args.steps >= 200 else LONG_WINDOW_STEPS
        torch.cuda.synchronize()
        _busy(stream)
        e0.record(stream)
        for _ in range(pn_steps):
            plan.spmv_permuted(xp, yp)
        e1.record(stream)
        torch.cuda.synchronize()
        pn_ms = e0.elapsed_time(e1) / pn_steps
        plan.permute(False, yp, yb)
        torch.cuda.synchronize()
        pn_gbs = float(info["bytes_effective"]) / (pn_ms / 1e3) / 1e9
        plan_numbering = {"api": "ehyb_spmv_permuted", "steps": pn_steps, "ms_per_step": pn_ms,
                          "value": flops_per_step / (pn_ms / 1e3) / 1e9, "unit": "GFLOP/s", "effective_gbs": pn_gbs,
                          "nominal_8tbs_frac": pn_gbs / 8000.0,
                          "bit_identical_after_permutation": bool(torch.equal(yb, yd))}
    # the FP64 FMA pipe's rate on this device, measured now (the FP64 kernels' ALU roof)
    fp64_peak, fp64_probe_ms = eh.fp64_fma_peak(iters=2048, reps=5)
    # the fused kernel timed alone: events around every launch (they keep consecutive launches from
    # overlapping, so this is the isolated duration, not the back-to-back one)
    plan.profile_enable(True)
    for _ in range(max(20, min(args.steps, 500))):
        plan.spmv(xd, yd)
    torch.cuda.synchronize()
    kern_ms, kern_n = plan.profile_read()
    plan.profile_enable(False)

    def reduce_max(v):
        t = torch.tensor([v], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())
    value, ms_max = aggregate(ms, world, flops_per_step * args.steps, reduce_max if pg else None)
    value /= 1e9
    ms_per_step = ms_max / args.steps

    # ---- roofline of the fused kernel.  With the permutation fused (one launch per step) its average
    # duration in the timed region is the step time; otherwise its isolated event-timed duration.
    hbm_peak, peak_src = measured_peaks()
    fused = info["er_layout"] != 1
    kern_iso_s = kern_ms / 1e3 / max(kern_n, 1)
    kern_s = ms_per_step / 1e3 if fused else kern_iso_s
    bytes_alg = float(info["bytes_effective"])
    gbs = bytes_alg / kern_s / 1e9
    fp64_tf = flops_per_step / kern_s / 1e12
    fp64_src = (f"measured: ehyb_fp64_fma_peak, 2-4 independent DFMA chains acc = u*w + acc per thread, 4 x 512 "
                f"threads per SM, best launch {fp64_probe_ms:.2f} ms, run after the timed region")
    t_hbm = bytes_alg / (hbm_peak * 1e9)
    t_alu = flops_per_step / (fp64_peak * 1e12)
    if t_alu > t_hbm:
        roof = {"bound": "alu", "achieved": fp64_tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": fp64_tf / fp64_peak,
                "traffic": None, "peak_source": fp64_src, "peak_nominal": FP64_NOMINAL_TFLOPS,
                "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "peak_source": f"{peak_src} copy bandwidth"}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": None, "peak_source": f"{peak_src} copy bandwidth",
                "alu": {"achieved": fp64_tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": fp64_tf / fp64_peak,
                        "peak_source": fp64_src, "peak_nominal": FP64_NOMINAL_TFLOPS}}
    traffic, tnote = recorded_traffic(args.workload + ("_multilevel" if args.partitioner else ""),
                                      layout_signature(info))
    roof["traffic"] = traffic
    if traffic is not None:
        roof["traffic_over_algorithmic"] = traffic / bytes_alg
        roof["traffic_source"] = tnote
    roof["kernel"] = "ehyb_kernel<double,double,gather+scatter>" if fused else "ehyb_kernel<double,double,scatter>"
    roof["kernel_ms"] = kern_s * 1e3
    roof["kernel_ms_isolated"] = kern_iso_s * 1e3
    roof["duration_source"] = ("timed region / launches (one launch per step, back to back)" if fused
                               else "per-launch CUDA events")
    roof["bytes_per_launch"] = bytes_alg
    roof["nominal_8tbs_frac"] = gbs / 8000.0

    # ---- plain CSR kernel on the same GPU (original order and EHYB order), best tpr
    csr = {}
    if not args.skip_csr:
        n2o = plan.export()["new_to_old"]
        o2n = np.empty(A.n, np.int64)
        o2n[n2o] = np.arange(A.n)
        for label, M in (("original_order", A), ("ehyb_order", _reorder(A, n2o, o2n))):
            base = eh.CsrBaseline(M)
            xx = xd if label == "original_order" else torch.from_numpy(x[n2o]).to(dev)
            best = None
            for tpr in (1, 2, 4, 8, 16, 32):
                base.set_tpr(tpr)
                for _ in range(3):
                    base.spmv(xx, yd)
                torch.cuda.synchronize()
                reps = max(20, min(args.steps, 200))
                e0.record(stream)
                for _ in range(reps):
                    base.spmv(xx, yd)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / reps
                if best is None or t < best[1]:
                    best = (tpr, t)
            csr_bytes = A.nnz * 12 + (A.n + 1) * 8 + 16 * A.n
            csr[label] = {"tpr": best[0], "ms": best[1], "gflops": flops_per_step / best[1] / 1e6,
                          "gbs": csr_bytes / best[1] / 1e6}
            base.close()
        csr["ehyb_speedup_vs_best_csr"] = min(c["ms"] for c in csr.values() if isinstance(c, dict)) / ms_per_step

    # ---- plan file: save once, load (no partitioning / encoding), same bits
    plan_io = None
    if args.plan_io:
        import tempfile as _tf
        d = _tf.mkdtemp()
        path = os.path.join(d, "plan.ehyb")
        t0 = time.perf_counter()
        plan.save(path)
        save_ms = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        loaded = eh.Plan.load(path)
        load_ms = (time.perf_counter() - t0) * 1e3
        y2 = torch.empty_like(yd)
        loaded.spmv(xd, y2)
        plan.spmv(xd, yd)
        torch.cuda.synchronize()
        plan_io = {"file_bytes": os.path.getsize(path), "save_ms": save_ms, "load_ms": load_ms,
                   "x_spmv_loaded": load_ms / ms_per_step, "bit_identical": bool(torch.equal(y2, yd))}
        loaded.close()
        os.unlink(path)
        os.rmdir(d)

    # ---- e2e through the public host entries, every step copying its x in from pinned host memory and its
    # y back out: the pipelined ehyb_spmv_host_many (the copies of neighbouring steps overlap each product;
    # host buffers in a ring of 4) and, beside it, one synchronous ehyb_spmv_host call per step
    ring = 4
    xhs = [torch.from_numpy(x).pin_memory() for _ in range(ring)]
    yhs = [torch.empty_like(xhs[0]).pin_memory() for _ in range(ring)]
    e2e_steps = max(10, min(args.steps, 200))
    xs_list = [xhs[i % ring] for i in range(e2e_steps)]
    ys_list = [yhs[i % ring] for i in range(e2e_steps)]
    plan.spmv_host_many(xs_list[:ring], ys_list[:ring])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.spmv_host_many(xs_list, ys_list)
    e2e_s = time.perf_counter() - t0
    plan.spmv(xd, yd)
    torch.cuda.synchronize()
    y_dev = yd.cpu()
    e2e = {"value": flops_per_step * e2e_steps * world / e2e_s / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(x.nbytes),
           "steps": e2e_steps, "api": "ehyb_spmv_host_many (pipelined)",
           "bit_identical_to_device_entry": all(bool(torch.equal(y, y_dev)) for y in yhs)}
    for _ in range(2):
        plan.spmv_host(xhs[0], yhs[0])
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.spmv_host(xhs[0], yhs[0])
    sync_s = time.perf_counter() - t0
    e2e["sync"] = {"value": flops_per_step * e2e_steps * world / sync_s / 1e9, "unit": "GFLOP/s",
                   "api": "ehyb_spmv_host (one synchronous call per step)"}

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "desc": w["desc"],
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": (f"inputs larger than L2 ({bytes_alg / 1e9:.2f} GB streamed from HBM every step)"
                              if not l2_resident else
                              f"L2-resident ({bytes_alg / 1e6:.1f} MB): every timed SpMV follows a "
                              f"{FLUSH_BYTES >> 20} MB write that flushes L2 (cold); warm back-to-back steps "
                              f"in 'warm'"),
                       "partitioner": ["greedy growing", "multilevel"][args.partitioner],
                       "er_layout": info["er_layout"], "block_threads": info["block_threads"],
                       "nparts": info["nparts"], "slice_rows": info["slice_rows"],
                       "er_fraction": info["er_nnz"] / A.nnz, "er_tpr": info["er_tpr"],
                       "block_threads": info["block_threads"]},
            "effective_gbs": bytes_alg * args.steps * world / (ms_max / 1e3) / 1e9,
            "roofline": roof, "csr_baseline": csr,
            "preprocessing": {"plan_ms": plan_ms, "partition_ms": info["partition_ms"],
                              "reorder_ms": info["reorder_ms"], "upload_ms": info["upload_ms"],
                              "x_spmv": plan_ms / ms_per_step, "plan_file": plan_io},
            "e2e": e2e, "gpu_launches": (1 if fused else 2) * args.steps, "clocks": clocks}
    if warm:
        line["warm"] = warm
    if plan_numbering:
        plan_numbering["hbm_frac"] = plan_numbering["effective_gbs"] / measured_peaks()[0]
        line["plan_numbering"] = plan_numbering
    if long_window:
        line["long_window"] = long_window
    if rank == 0 and not args.no_cpu_baseline:
        plan.spmv(xd, yd)
        torch.cuda.synchronize()
        line["cpu_baseline"] = cpu_baseline(A, x, args.cpu_seconds, yd.cpu().numpy())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def run_transient(args):
    """Many right-hand sides over time steps: implicit Euler for the heat equation on the Dirichlet tet
    Laplacian, (K + c I) u_{t+1} = c u_t (lumped mass, c = 0.1 x the mean diagonal of K, about ten times
    the explicit step), from u_0 ~ U[-1, 1) (seeded).  The plan and the preconditioner are built once; every
    step forms b = (c I) u_t with the library's SpMV on a diagonal plan and solves to a 1e-10 relative
    residual from u_t (warm start).  Per method: setup seconds, seconds and iterations per step, and how
    many steps one setup costs.  The line's value is steps per second of the fastest method.
    """
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    K = make_matrix(w)
    rows = np.repeat(np.arange(K.n), np.diff(K.row_ptr))
    c = 0.1 * float(K.val[K.col.astype(np.int64) == rows].mean())
    S = gen.shifted(K, c)
    u0 = torch.from_numpy(gen.uniform(K.n, w["seed_x"])).cuda()
    t0 = time.perf_counter()
    PS = eh.Plan(S, lowp=1)
    plan_s = time.perf_counter() - t0
    PR = eh.Plan(gen.scaled_identity(K.n, c))
    out, finals = {}, {}
    for name in ("fp64_cg", "fsai_pcg", "fsai_pcg_bf16_refined_0.01"):
        t0 = time.perf_counter()
        M = None if name == "fp64_cg" else eh.Fsai(PS, S, lowp=0 if name == "fsai_pcg" else 2)
        setup_s = plan_s + time.perf_counter() - t0
        u, b = u0.clone(), torch.empty_like(u0)
        secs, iters = [], []
        for step in range(args.transient_steps + 1):   # step 0 is untimed (first-use allocations)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            PR.spmv(u, b)
            if name == "fp64_cg":
                st, info = PS.cg(b, u, rtol=1e-10, max_iter=args.solver_max_iter)
            elif name == "fsai_pcg":
                st, info = PS.pcg(M, b, u, rtol=1e-10, max_iter=args.solver_max_iter)
            else:
                st, info = PS.pcg_refined(M, b, u, rtol=1e-10, max_iter=args.solver_max_iter, inner_rtol=0.01)
            torch.cuda.synchronize()
            if st != 0:
                raise RuntimeError(f"{name} step {step}: {eh.STATUS.get(st, st)}")
            if step > 0:
                secs.append(time.perf_counter() - t1)
                iters.append(info["iterations"])
        step_s = statistics.median(secs)
        finals[name] = u.cpu().numpy()
        out[name] = {"setup_s": setup_s, "step_s": step_s, "steps_per_s": 1.0 / step_s,
                     "iterations_per_step": float(np.mean(iters)), "iterations_first": iters[0],
                     "setup_in_steps": setup_s / step_s,
                     "total_s": setup_s + sum(secs)}
        if M is not None:
            M.close()
    ref = finals["fp64_cg"]
    for k in out:
        out[k]["rel_diff_vs_fp64_cg"] = float(np.linalg.norm(finals[k] - ref) / np.linalg.norm(ref))
    best = min(out, key=lambda k: out[k]["step_s"])
    line = {"metric": "implicit time steps per second (heat equation, PCG to 1e-10 per step, warm start)",
            "unit": "steps/s", "value": out[best]["steps_per_s"], "method": best, "higher_is_better": True,
            "n_gpus": 1, "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": args.workload, "n": K.n, "nnz": K.nnz, "desc": w["desc"], "shift_c": c,
                       "steps": args.transient_steps},
            "methods": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_solver(args):
    """Time to a 1e-10 relative residual: FP64 CG vs FP64 refinement around FP32 / BF16 inner CG, as
    restarted refinement (refine 1 / 2), as residual replacement that keeps the direction (refine 3 / 4) and as
    flexible FP64 CG with the inner solve as its preconditioner (refine 5 / 6),
    and FSAI-preconditioned CG (G in FP64 / FP32 / BF16; FP64 PCG and FP32 PCG with FP64 residual
    replacement every 10x or 100x).  The line's value is the FP32 PCG with BF16 G and replacement every 100x.

    b = A x* with x* ~ U[-1, 1) (seeded), computed by the library's FP64 SpMV.  Each method solves from
    x0 = 0; one untimed solve, then the median of `--solver-reps` timed solves (host wall clock around
    the synchronous ehyb_cg call).  Reported per method: iterations, refinements, seconds, the library's
    FP64 true residual and the error against x* and against the FP64 CG solution.
    """
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    A = make_matrix(w)
    xstar = gen.uniform(A.n, w["seed_x"])
    P32 = eh.Plan(A, lowp=1)
    ex = P32.export()
    pv = np.empty(A.n, np.int32)
    for p in range(len(ex["part_ptr"]) - 1):
        pv[ex["new_to_old"][ex["part_ptr"][p]:ex["part_ptr"][p + 1]]] = p
    P16 = eh.Plan(A, lowp=2, part_vec=pv)   # same partition, BF16 value copy
    xs = torch.from_numpy(xstar).cuda()
    b = torch.empty_like(xs)
    P32.spmv(xs, b)
    torch.cuda.synchronize()
    out = {}
    x_ref = None
    for name, plan, refine in (("fp64_cg", P32, 0), ("refined_fp32", P32, 1), ("refined_bf16", P16, 2),
                               ("replaced_fp32", P32, 3), ("replaced_bf16", P16, 4),
                               ("flexible_fp32", P32, 5), ("flexible_bf16", P16, 6)):
        times, res = [], None
        for rep in range(args.solver_reps + 1):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info = plan.cg(b, x, rtol=1e-10, max_iter=args.solver_max_iter, refine=refine)
            dt = time.perf_counter() - t0
            if rep > 0:
                times.append(dt)
            res = (st, info, x)
        st, info, x = res
        xh = x.cpu().numpy()
        if refine == 0:
            x_ref = xh
        out[name] = {"status": eh.STATUS.get(st, st), "converged": bool(info["converged"]),
                     "iterations": info["iterations"], "refinements": info["refinements"],
                     "flexible": bool(info["flexible"]),
                     "seconds": statistics.median(times), "relres_fp64": info["relres"],
                     "err_vs_xstar": float(np.linalg.norm(xh - xstar) / np.linalg.norm(xstar)),
                     "err_vs_fp64_cg": float(np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)),
                     "ms_per_iteration": 1e3 * statistics.median(times) / max(info["iterations"], 1)}
    # FSAI-preconditioned CG: G and G^T as two more EHYB plans on the same partition; G applied in FP64,
    # FP32 or BF16 values (M^-1 only has to be a fixed SPD operator); setup time reported beside the solve
    for name, lowp in (("fsai_pcg", 0), ("fsai_pcg_fp32", 1), ("fsai_pcg_bf16", 2)):
        t0 = time.perf_counter()
        M = eh.Fsai(P32, A, lowp=lowp)
        setup_s = time.perf_counter() - t0
        times, res = [], None
        for rep in range(args.solver_reps + 1):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info = P32.pcg(M, b, x, rtol=1e-10, max_iter=args.solver_max_iter)
            dt = time.perf_counter() - t0
            if rep > 0:
                times.append(dt)
            res = (st, info, x)
        st, info, x = res
        xh = x.cpu().numpy()
        out[name] = {"status": eh.STATUS.get(st, st), "converged": bool(info["converged"]),
                     "iterations": info["iterations"], "refinements": 0,
                     "seconds": statistics.median(times), "relres_fp64": info["relres"],
                     "err_vs_xstar": float(np.linalg.norm(xh - xstar) / np.linalg.norm(xstar)),
                     "err_vs_fp64_cg": float(np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)),
                     "ms_per_iteration": 1e3 * statistics.median(times) / max(info["iterations"], 1),
                     "setup_s": setup_s, "nnz_g": M.info()["nnz_g"]}
        if lowp:   # the same preconditioner in an all-FP32 PCG with FP64 residual replacement every `irt`
            for irt in (0.1, 0.01):
                times, res = [], None
                for rep in range(args.solver_reps + 1):
                    x = torch.zeros_like(b)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    st, info = P32.pcg_refined(M, b, x, rtol=1e-10, max_iter=args.solver_max_iter, inner_rtol=irt)
                    dt = time.perf_counter() - t0
                    if rep > 0:
                        times.append(dt)
                    res = (st, info, x)
                st, info, x = res
                xh = x.cpu().numpy()
                out[f"{name}_refined_{irt:g}"] = {
                    "status": eh.STATUS.get(st, st), "converged": bool(info["converged"]),
                    "iterations": info["iterations"], "refinements": info["refinements"],
                    "seconds": statistics.median(times), "relres_fp64": info["relres"],
                    "err_vs_xstar": float(np.linalg.norm(xh - xstar) / np.linalg.norm(xstar)),
                    "err_vs_fp64_cg": float(np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)),
                    "ms_per_iteration": 1e3 * statistics.median(times) / max(info["iterations"], 1),
                    "setup_s": setup_s, "nnz_g": M.info()["nnz_g"]}
        M.close()
    base = out["fp64_cg"]["seconds"]
    best = "fsai_pcg_bf16_refined_0.01"
    line = {"metric": "CG time to 1e-10 relative residual (FP64 CG vs mixed-precision and preconditioned solvers)",
            "unit": "s", "value": out[best]["seconds"], "method": best,
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64+f32+bf16",
            "data": "synthetic", "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "desc": w["desc"],
                                             "reps": args.solver_reps},
            "methods": out,
            "speedup_vs_fp64": {k: base / v["seconds"] for k, v in out.items() if v["converged"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _event_time(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_batch(args):
    """64 generated FEM matrices (n log-uniform in [5k, 300k], four element kinds): one persistent batch
    launch (graph replay) vs the same 64 SpMVs issued one by one."""
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    mats = gen.fem_batch(count=args.batch_count, seed=31)
    plans = [eh.Plan(A, part_nnz=args.part_nnz, smem_budget=args.batch_smem) for A in mats]
    xs = [torch.from_numpy(gen.uniform(A.n, 32 + i)).cuda() for i, A in enumerate(mats)]
    ys = [torch.empty_like(x) for x in xs]
    B = eh.Batch(plans)
    for _ in range(args.warmup):
        B.spmv(xs, ys)
    t_batch = _event_time(lambda: B.spmv(xs, ys), args.steps, stream)

    def one_by_one():
        for P, x, y in zip(plans, xs, ys):
            P.spmv(x, y)
    for _ in range(args.warmup):
        one_by_one()
    t_seq = _event_time(one_by_one, max(3, args.steps // 4), stream)
    nnz = sum(A.nnz for A in mats)
    byts = sum(P.info()["bytes_effective"] for P in plans)
    line = {"metric": "batched EHYB SpMV GFLOP/s (64 FEM matrices, one persistent graph-captured launch)",
            "unit": "GFLOP/s", "value": 2 * nnz / t_batch / 1e6, "higher_is_better": True, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"fem_batch_{args.batch_count}", "matrices": len(mats),
                       "rows": sum(A.n for A in mats), "nnz": nnz, "n_min": min(A.n for A in mats),
                       "n_max": max(A.n for A in mats), "kinds": sorted(set(A.name.split("_N")[0] for A in mats)),
                       "tiles": B.info()["tiles"], "grid": B.info()["grid"], "threads": B.info()["threads"],
                       "part_nnz": args.part_nnz, "smem_budget": args.batch_smem},
            "batch": {"ms": t_batch, "gflops": 2 * nnz / t_batch / 1e6, "effective_gbs": byts / t_batch / 1e6},
            "one_by_one": {"ms": t_seq, "gflops": 2 * nnz / t_seq / 1e6, "effective_gbs": byts / t_seq / 1e6,
                           "launches": len(mats)},
            "speedup": t_seq / t_batch, "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_spmm(args):
    """SpMM with k = 8 and 32 right-hand sides on the 70^3 hex matrix vs k separate SpMVs."""
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    A = make_matrix(WORKLOADS["hex_elast3d_70"])
    P1 = eh.Plan(A)                                   # the SpMV's plan, for the k-SpMV comparison
    x = torch.from_numpy(gen.uniform(A.n, 13)).cuda()
    y = torch.empty_like(x)
    t_spmv = _event_time(lambda: P1.spmv(x, y), 50, stream)
    fp64_peak, _ = eh.fp64_fma_peak(iters=2048, reps=5)
    out = {}
    for k in args.spmm_k:
        # a plan built for k right-hand sides (Eq. 1 with an 8-column slice of X per row), or a given VecSize
        P = eh.Plan(A, slice_rows=args.spmm_slice_rows, spmm_rhs=k)
        X = torch.from_numpy(np.stack([gen.uniform(A.n, 32 + j) for j in range(k)], axis=1)).cuda()
        Y = torch.empty_like(X)
        for _ in range(args.warmup):
            P.spmm(X, Y)
        t = _event_time(lambda: P.spmm(X, Y), max(5, args.steps // 50), stream)
        flops = 2.0 * A.nnz * k
        out[f"k{k}"] = {"ms": t, "gflops": flops / t / 1e6, "fp64_roof_frac": flops / t / 1e9 / fp64_peak,
                        "vs_k_spmv": (k * t_spmv) / t, "slice_rows": P.info()["slice_rows"],
                        "nparts": P.info()["nparts"], "er_fraction": P.info()["er_nnz"] / A.nnz}
    line = {"metric": "EHYB SpMM GFLOP/s (FP64, k right-hand sides, 3D hex 70^3)", "unit": "GFLOP/s",
            "value": out[f"k{args.spmm_k[0]}"]["gflops"], "higher_is_better": True, "n_gpus": 1, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "hex_elast3d_70", "n": A.n, "nnz": A.nnz},
            "spmv_ms": t_spmv, "fp64_peak_tflops": fp64_peak, "fp64_peak_source": "measured (ehyb_fp64_fma_peak)",
            "spmm": out}
    print(json.dumps(line), flush=True)
    return 0


def run_lowp(args):
    """The low-precision SpMVs of the mixed-precision solvers (`ehyb_spmv_lowp`: FP32 or BF16 values, FP32 x, y,
    FP32 accumulation, one fused launch) against the FP64 one on the same partition.  Algorithmic bytes per
    SpMV: FP32 6 per slab entry (value + 16-bit column), 8 per ER entry, 4n (x) + 4n (y); BF16 4 / 6 per entry."""
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    A = make_matrix(w)
    hbm, hbm_src = measured_peaks()
    P32 = eh.Plan(A, lowp=1, lowp_group=args.lowp_group, er_layout=args.er_layout)
    ex = P32.export()
    pv = np.empty(A.n, np.int32)
    for p in range(len(ex["part_ptr"]) - 1):
        pv[ex["new_to_old"][ex["part_ptr"][p]:ex["part_ptr"][p + 1]]] = p
    P16 = eh.Plan(A, lowp=2, part_vec=pv, lowp_group=args.lowp_group, er_layout=args.er_layout)
    info = P32.info()
    slab, er, n = info["ell_nnz"], info["er_nnz"], A.n
    xh = gen.uniform(A.n, w["seed_x"])
    x64 = torch.from_numpy(xh).cuda()
    y64 = torch.empty_like(x64)
    x32 = x64.float()
    y32 = torch.empty_like(x32)
    reps = max(50, args.steps // 10)
    out = {}
    for name, fn, nbytes in (("f64", lambda: P32.spmv(x64, y64), 10 * slab + 12 * er + 16 * n),
                             ("f32", lambda: P32.spmv_lowp(x32, y32), 6 * slab + 8 * er + 8 * n),
                             ("bf16", lambda: P16.spmv_lowp(x32, y32), 4 * slab + 6 * er + 8 * n)):
        for _ in range(args.warmup):
            fn()
        t = _event_time(fn, reps, stream)
        gbs = nbytes / t / 1e6
        out[name] = {"us": t * 1e3, "gflops": 2.0 * A.nnz / t / 1e6, "bytes": nbytes, "gbs": gbs,
                     "hbm_frac": gbs / hbm}
    P32.spmv_lowp(x32, y32)
    torch.cuda.synchronize()
    y = y32.double().cpu().numpy()
    P32.spmv(x64, y64)
    torch.cuda.synchronize()
    ref = y64.cpu().numpy()
    line = {"metric": "EHYB low-precision SpMV effective GB/s (FP32 values, FP32 x/y)", "unit": "GB/s",
            "value": out["f32"]["gbs"], "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "hbm_peak_gbs": hbm,
                       "hbm_peak_source": hbm_src, "reps": reps, "lowp_group": [P32.info()["lowp_group"],
                                                                            P16.info()["lowp_group"]]},
            "spmv": out,
            "f32_vs_f64_rel_l2": float(np.linalg.norm(y - ref) / np.linalg.norm(ref))}
    print(json.dumps(line), flush=True)
    return 0


def run_shard(args):
    """The halo-exchange form of the product across ranks (one GPU each, launched by torchrun): every rank
    builds the plan of the whole matrix, keeps its shard (a contiguous group of partitions), and a step is
    pack -> all_to_all of the halo (NCCL) -> the shard's product.  Strong scaling: the same matrix over N GPUs;
    value = 2 nnz per step / the slowest rank's time.  One rank runs the same path with an empty exchange."""
    import torch
    import gen
    import paper_2204_06666_gb300 as eh
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOADS[args.workload]
    A = make_matrix(w)
    P = eh.Plan(A)
    n2o = P.export()["new_to_old"]
    S = eh.Shard(P, world, rank)
    x = gen.uniform(A.n, w["seed_x"])[n2o]
    xe = torch.zeros(S.n_local + S.n_halo, dtype=torch.float64, device=dev)
    xe[:S.n_local] = torch.from_numpy(x[S.row_begin:S.row_end]).to(dev)
    send = torch.zeros(max(S.send_total, 1), dtype=torch.float64, device=dev)
    y = torch.empty(max(S.n_local, 1), dtype=torch.float64, device=dev)
    halo = xe[S.n_local:]

    def step():
        S.pack(xe[:S.n_local], send)
        if world > 1:
            dist.all_to_all_single(halo, send[:S.send_total], output_split_sizes=S.recv_counts,
                                   input_split_sizes=S.send_counts)
        S.spmv(xe, y)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        _busy(stream)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)

    def reduce_max(v):
        t = torch.tensor([v], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    ms_max = reduce_max(ms) if world > 1 else ms
    value = 2.0 * A.nnz * args.steps / (ms_max / 1e3) / 1e9
    line = {"metric": METRIC + " (row shards, halo exchange over NCCL)", "value": value, "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "desc": w["desc"],
                       "parallelism": f"row shards x{world}", "n_local": S.n_local, "n_halo": S.n_halo,
                       "send_total": S.send_total},
            "gpu_launches": (2 if S.send_total else 1) * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _reorder(A, n2o, o2n):
    """P A P^T in CSR, rows in the plan numbering (columns relabelled, order kept)."""
    import gen
    lens = np.diff(A.row_ptr)[n2o]
    rp = np.zeros(A.n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    idx = _gather_rows(A.row_ptr, n2o, rp)
    return gen.CSR(A.n, rp, o2n[A.col[idx]].astype(np.int32), A.val[idx], A.name + "_ehyb_order")


def _gather_rows(row_ptr, n2o, rp_new):
    starts = row_ptr[n2o]
    lens = np.diff(rp_new)
    out = np.repeat(starts - rp_new[:-1], lens) + np.arange(rp_new[-1])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ehyb", choices=["ehyb", "reference"])
    ap.add_argument("--workload", default="hex_elast3d_70", choices=sorted(WORKLOADS))
    ap.add_argument("--skip-csr", action="store_true")
    ap.add_argument("--er-layout", type=int, default=0, choices=[0, 1, 2],
                    help="extra-row layout of the SpMV and --lowp plans (options.er_layout)")
    ap.add_argument("--slice-rows", type=int, default=0,
                    help="rows per partition of the SpMV plan (options.slice_rows; 0 = Eq. 1)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="threads per block of the SpMV plan (options.block_threads; 0 = automatic)")
    ap.add_argument("--partitioner", type=int, default=0, choices=[0, 1],
                    help="PartVec of the SpMV plan: 0 greedy graph growing, 1 multilevel")
    ap.add_argument("--plan-io", action="store_true", help="also time saving the plan to a file and loading it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--solver", action="store_true", help="time CG / refined CG instead of the SpMV")
    ap.add_argument("--batch", action="store_true", help="time the batched launch over generated FEM matrices")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--part-nnz", type=int, default=640000, help="entries per partition of batched plans")
    ap.add_argument("--batch-smem", type=int, default=50000,
                    help="shared-memory budget per block of batched plans in bytes (caps partition rows; 0 = device max)")
    ap.add_argument("--spmm", action="store_true", help="time SpMM with --spmm-k right-hand sides")
    ap.add_argument("--spmm-k", type=int, nargs="+", default=[8, 32])
    ap.add_argument("--spmm-slice-rows", type=int, default=0,
                    help="VecSize of the SpMM plans (0: Eq. 1 for k right-hand sides)")
    ap.add_argument("--lowp", action="store_true", help="time the FP32 / BF16 SpMVs of the mixed-precision solvers")
    ap.add_argument("--lowp-group", type=int, default=0, choices=[0, 1, 4],
                    help="slot layout of the FP32 / BF16 copies: 0 automatic, 1 column-major, 4 runs of four")
    ap.add_argument("--shard", action="store_true",
                    help="row shards across the torchrun ranks with a halo exchange per product (strong scaling)")
    ap.add_argument("--solver-reps", type=int, default=3)
    ap.add_argument("--transient", action="store_true",
                    help="time implicit-Euler steps (one plan and preconditioner, a PCG solve per step)")
    ap.add_argument("--transient-steps", type=int, default=20)
    ap.add_argument("--solver-max-iter", type=int, default=50000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.solver:
        return run_solver(args)
    if args.transient:
        return run_transient(args)
    if args.batch:
        return run_batch(args)
    if args.spmm:
        return run_spmm(args)
    if args.lowp:
        return run_lowp(args)
    if args.shard:
        return run_shard(args)
    return run_ehyb(args)


if __name__ == "__main__":
    sys.exit(main())
