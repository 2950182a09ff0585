"""Pins of the independent EHYB format checks: a hand-derived example, Eq. 1 closed form, Sec. 3.4 byte model."""
import json
import math
import os

import numpy as np
import pytest

import gen
from oracle import ehyb_format as ef

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ehyb_tiny.json")


def golden_plan():
    g = json.load(open(GOLDEN))
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


def test_decode_hand_derived_example():
    g, p, A = golden_plan()
    assert ef.same_multiset(ef.decode(p), ef.triplets(A))


def test_decode_hand_derived_example_sliced_extra_rows():
    g, p, A = golden_plan()
    q = {k: v for k, v in p.items() if not k.startswith("er_")}
    q["er_layout"] = 0
    q["er_slice_pos"] = p["er_slice_pos"]
    size = p["er_slice_pos"][-1]
    q["er_scol"] = np.full(size, p["er_slice_pad_col"][0], np.int32)
    q["er_sval"] = np.zeros(size)
    for pos, c, v in p["er_slice_entries"]:
        q["er_scol"][pos], q["er_sval"][pos] = c, v
    assert ef.same_multiset(ef.decode(q), ef.triplets(A))
    q["row_er_count"] = [0, 1, 0, 0, 0]   # the extra entry attributed to the wrong row is dropped
    assert not ef.same_multiset(ef.decode(q), ef.triplets(A))


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
