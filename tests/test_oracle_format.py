"""Pins of the independent EHYB format checks: a hand-derived example, Eq. 1 closed form, Sec. 3.4 byte model."""
import json
import math
import os

import numpy as np
import pytest

import gen
from oracle import ehyb_format as ef

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ehyb_tiny.json")
GROUPED = os.path.join(os.path.dirname(__file__), "golden", "ehyb_grouped.json")


def golden_plan(path=GOLDEN):
    g = json.load(open(path))
    p = dict(g["plan"])
    size = p["slice_pos"][-1]
    col = np.zeros(size, np.uint16)
    val = np.zeros(size, np.float64)
    for pos, c, v in p.pop("ell_entries"):
        col[pos], val[pos] = c, v
    p["ell_col"], p["ell_val"] = col, val
    A = gen.CSR(g["n"], np.array(g["row_ptr"], np.int64), np.array(g["col"], np.int32),
                np.array(g["val"], np.float64))
    return g, p, A


@pytest.mark.parametrize("path", [GOLDEN, GROUPED], ids=["tiny", "grouped"])
def test_decode_hand_derived_example(path):
    g, p, A = golden_plan(path)
    assert ef.same_multiset(ef.decode(p), ef.triplets(A))


@pytest.mark.parametrize("path", [GOLDEN, GROUPED], ids=["tiny", "grouped"])
def test_decode_hand_derived_example_sliced_extra_rows(path):
    g, p, A = golden_plan(path)
    q = {k: v for k, v in p.items() if not k.startswith("er_")}
    q["er_layout"] = 0
    q["er_slice_pos"] = p["er_slice_pos"]
    size = p["er_slice_pos"][-1]
    q["er_scol"] = np.full(size, p["er_slice_pad_col"][0], np.int32)
    q["er_sval"] = np.zeros(size)
    for pos, c, v in p["er_slice_entries"]:
        q["er_scol"][pos], q["er_sval"][pos] = c, v
    assert ef.same_multiset(ef.decode(q), ef.triplets(A))
    q["row_er_count"] = np.roll(np.asarray(p["row_er_count"]), 1)   # extra entries attributed to the wrong row
    assert not ef.same_multiset(ef.decode(q), ef.triplets(A))


def test_slot_index_runs_and_tail():
    # group 1 is Alg. 2's column-major order
    assert [ef.slot_index(0, 6, k, 5) for k in range(6)] == [5, 37, 69, 101, 133, 165]
    # group 4, width 6: slots 0..3 of a lane are four consecutive words, the 32 lanes' runs side by side;
    # slots 4, 5 are column-major behind the runs
    assert [ef.slot_index(0, 6, k, 0, 4) for k in range(6)] == [0, 1, 2, 3, 128, 160]
    assert [ef.slot_index(0, 6, k, 5, 4) for k in range(6)] == [20, 21, 22, 23, 133, 165]
    # narrower than a run: column-major in both layouts
    assert [ef.slot_index(32, 3, k, 7, 4) for k in range(3)] == [39, 71, 103]
    # every run is aligned to four slots, so a 4-slot vector load of it is aligned to its own size
    assert all(ef.slot_index(0, 9, 4 * q, lane, 4) % 4 == 0 for q in range(2) for lane in range(32))


@pytest.mark.parametrize("group", [1, 4])
@pytest.mark.parametrize("width", range(0, 11))
def test_slot_index_fills_the_slice_once_in_both_layouts(width, group):
    got = sorted(ef.slot_index(64, width, k, lane, group) for lane in range(32) for k in range(width))
    assert got == list(range(64, 64 + 32 * width))


def _runs_plan():
    # the grouped golden with its FP32 copy (integer values: exact) in place of the FP64 arrays
    g, p, A = golden_plan(GROUPED)
    q = dict(p)
    size, esize = p["slice_pos"][-1], p["er_slice_pos"][-1]
    q["ell_col"], q["ell_val"] = np.zeros(size, np.uint16), np.zeros(size)
    for pos, c, v in g["runs"]["ell_entries"]:
        q["ell_col"][pos], q["ell_val"][pos] = c, v
    q["er_layout"], q["er_scol"], q["er_sval"] = 0, np.full(esize, p["er_slice_pad_col"][0], np.int32), np.zeros(esize)
    for pos, c, v in g["runs"]["er_slice_entries"]:
        q["er_scol"][pos], q["er_sval"][pos] = c, v
    return q, A


def test_decode_runs_layout_of_the_hand_derived_example():
    q, A = _runs_plan()
    assert ef.same_multiset(ef.decode(q, group=4), ef.triplets(A))
    assert not ef.same_multiset(ef.decode(q, group=1), ef.triplets(A))   # read in the wrong layout


def test_decode_detects_a_swapped_pair_inside_a_run():
    q, A = _runs_plan()
    q["ell_val"] = q["ell_val"].copy()
    q["ell_val"][[4, 128]] = q["ell_val"][[128, 4]]   # slot 0 of lane 1 swapped with slot 4 of lane 0
    assert not ef.same_multiset(ef.decode(q, group=4), ef.triplets(A))


def test_decode_detects_a_misplaced_entry():
    g, p, A = golden_plan()
    p["ell_col"] = p["ell_col"].copy()
    p["ell_col"][96] = 1          # wrong local column for entry (1,2)
    assert not ef.same_multiset(ef.decode(p), ef.triplets(A))
    g, p, A = golden_plan()
    p["new_to_old"] = [3, 0, 4, 1, 2]   # rows swapped
    assert not ef.same_multiset(ef.decode(p), ef.triplets(A))


@pytest.mark.parametrize("n,tau,P,shm", [(1029000, 8, 152, 232448 - 1024), (40000, 8, 152, 231424),
                                         (2000376, 4, 152, 231424), (10 ** 7, 8, 80, 98304),
                                         (1, 8, 152, 1000), (5_000_000, 8, 148, 65536)])
def test_eq1_closed_form(n, tau, P, shm):
    K, vec = ef.eq1(n, tau, P, shm)
    # smallest integer K with n*tau/(K*P) < SHM  <=>  K = floor(n*tau/(P*SHM)) + 1, unless the 2^16 cap binds
    K0 = n * tau // (P * shm) + 1
    assert K >= K0
    if math.ceil(n / (K0 * P)) <= 1 << 16:
        assert K == K0
    assert vec == math.ceil(n / (K * P)) and vec <= 1 << 16
    assert n * tau / (K * P) < shm
    if K > 1:
        assert not (n * tau / ((K - 1) * P) < shm and math.ceil(n / ((K - 1) * P)) <= 1 << 16)


def test_eq1_hex_config_is_one_partition_per_sm():
    K, vec = ef.eq1(1029000, 8, 152, 227 * 1024)
    assert K == 1 and vec == 6770


def test_footprint_savings_of_16bit_columns():
    # Sec. 3.4: a 16-bit column index instead of 32-bit saves 25% of the ELL bytes in FP32;
    # in FP64 the same arithmetic gives 1 - 10/12 = 16.7% (the text prints 13.3%)
    assert 1 - ef.ell_bytes_per_entry(4, 2) / ef.ell_bytes_per_entry(4, 4) == 0.25
    assert abs(1 - ef.ell_bytes_per_entry(8, 2) / ef.ell_bytes_per_entry(8, 4) - 1 / 6) < 1e-15
