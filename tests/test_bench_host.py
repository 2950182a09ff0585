"""bench.py host logic without a GPU: the whole-job aggregation over ranks (gloo, world size 2), the
traffic record's invalidation, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    local_ms = [120.0, 150.0][rank]                     # the slower rank sets the time
    value, ms_max = bench.aggregate(local_ms, world, 1e9, reduce_max)
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_over_ranks_gloo():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, 29517, out), nprocs=world, join=True)
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1e9 / 0.150)   # all ranks' units over the slowest rank's time


def test_aggregate_single_rank():
    assert bench.aggregate(100.0, 1, 5e8) == (5e8 / 0.1, 100.0)


def test_traffic_record_tied_to_kernel_sources_and_layout(tmp_path, monkeypatch):
    lay = "152/32208/411238400/12930000/11921367"
    rec = {"hex_elast3d_70": {"source_sha": bench.kernel_source_sha(), "layout": lay, "dram_bytes_per_launch": 9.0e8,
                              "note": "x"}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ehyb_kernel_dram.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is computed over ROOT's sources: copy them so the record matches
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    assert bench.recorded_traffic("hex_elast3d_70", lay)[0] == 9.0e8
    assert bench.recorded_traffic("fem2d_p1_200", lay)[0] is None
    assert bench.recorded_traffic("hex_elast3d_70", "152/1/2/3/4")[0] is None     # another plan layout
    (tmp_path / "paper_2204_06666_gb300/csrc/ehyb_core.cuh").write_text("// changed kernel")
    assert bench.recorded_traffic("hex_elast3d_70", lay)[0] is None                # kernel changed: no stale traffic
    info = {"nparts": 152, "nslices": 32208, "ell_stored": 411238400, "er_stored": 12930000, "er_nnz": 11921367}
    assert bench.layout_signature(info) == lay


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "fem2d_p1_200", "--steps", "20", "--warmup", "3"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baselines_compute_the_product():
    # the single-thread sample and the all-core run use the oracle's row routine; the all-core run's rows
    # together are one whole product
    import numpy as np
    import gen
    import oracle
    A = gen.fem2d_p1(N=60)
    x = gen.uniform(A.n, 3)
    one = bench.cpu_baseline(A, x, 0.2, oracle.spmv(A, x))
    assert one["value"] > 0 and one["cores"] == 1 and one["parity"]["rel_l2"] == 0.0
    multi = one["multicore"]
    assert multi["value"] > 0 and multi["cores"] >= 1 and multi["kind"] == "oracle"


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29563", os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "fem2d_p1_200", "--steps", "10", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
