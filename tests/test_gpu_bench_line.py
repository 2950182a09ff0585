"""The benchmark's JSON line on a GPU: every key of the contract is present with the right type, the roofline
block names its bound and a fraction in range, the end-to-end block counts its copies, and the cold timing of
an L2-resident workload keeps the warm time beside it; a workload larger than L2 also reports the product in the
plan's numbering, bit-identical to the fused entry after the permutation."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_default_workload_line_keeps_the_contract():
    d = _line("--steps", "20", "--warmup", "3", "--skip-csr", "--cpu-seconds", "1")
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("roofline", dict), ("e2e", dict),
                 ("gpu_launches", int), ("clocks", dict), ("cpu_baseline", dict)):
        assert isinstance(d[k], t), k
    assert d["vs_baseline"] is None and d["n_gpus"] == 1 and d["steps"] == 20 and d["dtype"] == "f64"
    assert d["config"]["workload"] == "hex_elast3d_70" and d["value"] > 0
    r = d["roofline"]
    assert r["bound"] in ("alu", "hbm") and 0 < r["frac"] < 1.2 and r["peak"] > 0 and r["unit"] in ("TFLOP/s", "GB/s")
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9
    fp64 = r if r["bound"] == "alu" else r["alu"]
    assert fp64["peak_source"].startswith("measured") and 0.3 < fp64["peak"] / fp64["peak_nominal"] < 1.1
    lw = d["long_window"]                   # a 20-step window is repeated over 2000 steps beside it
    assert lw["steps"] == 2000 and 0.5 < lw["ms_per_step"] / d["ms_per_step"] < 2.0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 8 * d["config"]["n"]
    assert e["bit_identical_to_device_entry"] and e["sync"]["value"] > 0
    assert d["gpu_launches"] == d["steps"]
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] == 1 and c["value"] > 0 and c["multicore"]["cores"] >= 1
    assert c["parity"]["rel_l2"] <= c["parity"]["tolerance"]
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    pn = d["plan_numbering"]                # the same product with the vectors kept in the plan's numbering
    assert pn["api"] == "ehyb_spmv_permuted" and pn["steps"] == 2000 and pn["bit_identical_after_permutation"]
    assert 0.5 < pn["ms_per_step"] / d["ms_per_step"] < 1.5 and 0 < pn["hbm_frac"] < 1.2


def test_l2_resident_workload_is_timed_cold():
    d = _line("--workload", "fem2d_p1_200", "--steps", "200", "--warmup", "3", "--skip-csr", "--no-cpu-baseline")
    assert "flushes L2" in d["config"]["l2"]
    assert d["warm"]["ms_per_step"] > 0 and d["warm"]["value"] > 0
    assert d["ms_per_step"] >= 0.8 * d["warm"]["ms_per_step"]     # a flushed step is not faster than a warm one
    assert "plan_numbering" not in d                                # timed only where inputs exceed L2


def test_fp64_probe_measures_a_plausible_rate():
    import torch
    import paper_2204_06666_gb300 as eh
    torch.cuda.set_device(0)
    tf, ms = eh.fp64_fma_peak(iters=1024, reps=3)
    nominal = 2 * 2 * torch.cuda.get_device_properties(0).multi_processor_count * 2.07e9 / 1e12
    assert ms > 0 and 0.3 * nominal < tf < 1.1 * nominal     # at most the nominal rate, well above a stall
    with pytest.raises(eh.EhybError):
        eh.fp64_fma_peak(iters=0)


def test_shard_mode_line_on_one_rank():
    # one rank: the shard is the whole plan, no halo, one launch per step; the same time as the plan's product
    d = _line("--shard", "--steps", "50", "--warmup", "3")
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["n_halo"] == 0 and d["config"]["n_local"] == d["config"]["n"]
    assert d["gpu_launches"] == 50 and set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
