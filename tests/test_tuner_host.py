"""Tuner host logic without a GPU: features against an independent numpy statement, the knob grid."""
import math

import numpy as np
import pytest

import gen
from oracle import ehyb_format as ef
from oracle import features as of


def _pinned(name):
    # matrices whose oracle features are pinned to closed forms in test_oracle_features.py
    n = 300
    if name == "lower_triangle":
        rows = [np.arange(i + 1) for i in range(n)]
    else:
        rows = [np.array([n - 1 - i]) for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    return gen.CSR(n, rp, col, np.ones(col.size))


@pytest.mark.parametrize("make", [lambda: gen.fem2d_p1(N=40), lambda: gen.hex_elast3d(N=6),
                                  lambda: gen.random_csr(900, 3, mean_row=7, long_rows=4, long_len=300,
                                                         empty_frac=0.05, symmetric=True),
                                  lambda: gen.random_csr(500, 4, mean_row=12, duplicates=True),
                                  lambda: _pinned("lower_triangle"), lambda: _pinned("anti_diagonal")])
def test_features_match_independent_statement(make):
    import paper_2204_06666_gb300 as eh
    A = make()
    f = eh.features(A)
    ref = of.features(A)
    assert np.allclose(f, ref.astype(np.float32), rtol=2e-6, atol=1e-6), np.c_[f, ref]


def test_features_closed_forms():
    import paper_2204_06666_gb300 as eh
    n = 64
    D = 4 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)   # tridiagonal, strictly dominant, symmetric
    r, c = np.nonzero(D)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    A = gen.CSR(n, np.cumsum(rp), c.astype(np.int32), D[r, c])
    f = eh.features(A)
    assert f[0] == pytest.approx(math.log2(65)) and f[1] == pytest.approx(math.log2(n * 3 - 2 + 1))
    assert f[2] == pytest.approx((3 * n - 2) / n) and f[5] == 2 and f[6] == 3
    assert f[13] == 1.0 and f[14] == 1.0 and f[9] == 0.0
    assert f[12] == 1.0                 # every entry within one band of the diagonal


def test_tune_grid_values():
    import paper_2204_06666_gb300 as eh
    A = gen.random_csr(20000, 9, mean_row=10, long_rows=50, long_len=2000)
    g = eh.tune_grid(A)
    assert len(g) == 112
    K, vec = ef.eq1(A.n, 8, 152, 232448 - 1024 - 32)
    slices = sorted({e["slice_rows"] for e in g})
    assert set(slices) == {vec, 1024, 2048, 4096, 8192, 16384, (232448 - 1024 - 32) // 8 - 2}
    lens = np.sort(np.diff(A.row_ptr))
    caps = {e["ell_width_cap"] for e in g}
    assert caps == {0} | {int(lens[int(q * (A.n - 1))]) for q in (0.99, 0.9, 0.75)}
    assert {e["ell_tpr"] for e in g} == {1, 2, 4, 8}
    # entry order: VecSize index g // 16, cap index (g // 4) % 4 (none, p99, p90, p75), lanes index g % 4
    assert g[0]["slice_rows"] == vec and g[0]["ell_width_cap"] == 0 and g[0]["ell_tpr"] == 1
    assert g[4 * 3 + 3]["ell_width_cap"] == int(lens[int(0.75 * (A.n - 1))]) and g[15]["ell_tpr"] == 8
    assert g[111]["slice_rows"] == (232448 - 1024 - 32) // 8 - 2 and g[111]["ell_tpr"] == 8
