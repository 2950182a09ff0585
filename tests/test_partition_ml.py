"""The multilevel partitioner (options.partitioner = 1) on the CPU: the plans it gives decode to the input and
keep every partition under the cap with ceil(n / cap) parts of equal size, it finds the known optimum on
graphs whose best cut is fixed by their structure, it is deterministic (seed, thread count), and it cuts
fewer entries than the greedy partitioner on the generated FEM and power-law matrices (measured quality,
not a parity pin)."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
from oracle import ehyb_format as ef
from test_plan_host import _invariants


def _plan(A, **kw):
    import paper_2204_06666_gb300 as eh
    return eh.Plan(A, host_only=1, **kw)


def _csr(S, name=""):
    S = sp.csr_matrix(S)
    S.sort_indices()
    return gen.CSR(S.shape[0], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(float), name)


def _permuted(S, seed):
    p = np.random.default_rng(seed).permutation(S.shape[0])
    return sp.csr_matrix(S)[p][:, p]


def _er_fraction(A, **kw):
    info = _plan(A, **kw).info()
    return info["er_nnz"] / max(A.nnz, 1)


@pytest.mark.parametrize("name", ["fem2d", "hex", "tet", "random"])
@pytest.mark.parametrize("cap", [200, 57])
def test_multilevel_plan_decodes_with_equal_parts_under_the_cap(name, cap):
    A = {"fem2d": lambda: gen.fem2d_p1(N=40), "hex": lambda: gen.hex_elast3d(N=8),
         "tet": lambda: gen.tet_lap3d(N=12),
         "random": lambda: gen.random_csr(3000, 5, mean_row=9, empty_frac=0.1, long_rows=3, long_len=400,
                                          duplicates=True)}[name]()
    P = _plan(A, slice_rows=cap, partitioner=1)
    ex = P.export()
    assert ef.same_multiset(ef.decode(ex), ef.triplets(A))
    _invariants(A, ex, cap=cap)
    k = -(-A.n // cap)
    sizes = np.diff(ex["part_ptr"])
    assert P.info()["nparts"] == k and sizes.max() <= cap
    assert sizes.max() - sizes.min() <= 1          # every part holds its share of the rows


def test_disjoint_cliques_are_found_exactly():
    # 12 cliques of 40 rows in a random numbering: the optimum cuts nothing
    S = sp.block_diag([sp.csr_matrix(np.ones((40, 40)))] * 12, format="csr")
    A = _csr(_permuted(S, 1))
    assert _er_fraction(A, slice_rows=40, partitioner=1) == 0.0


def test_path_is_cut_into_contiguous_runs():
    # a path of 16 x 100 vertices in a random numbering: 15 cut edges (30 entries) is optimal
    n, cap = 1600, 100
    S = sp.diags([np.ones(n - 1), 2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1], format="csr")
    A = _csr(_permuted(S, 2))
    info = _plan(A, slice_rows=cap, partitioner=1).info()
    assert info["er_nnz"] == 2 * (n // cap - 1)


def test_grid_is_bisected_across_its_short_side():
    # 5-point 64 x 32 grid into two parts: the optimum cuts the 32 edges of a column line (64 entries)
    nx, ny = 64, 32
    T = lambda m: sp.diags([np.ones(m - 1), np.ones(m - 1)], [-1, 1])
    S = (sp.kron(sp.identity(ny), T(nx)) + sp.kron(T(ny), sp.identity(nx)) + 4 * sp.identity(nx * ny)).tocsr()
    A = _csr(_permuted(S, 3))
    info = _plan(A, slice_rows=nx * ny // 2, partitioner=1).info()
    assert info["er_nnz"] <= 1.25 * 2 * ny, info["er_nnz"]


def test_supervariable_larger_than_the_cap_is_split():
    # a dense 10 x 10 block is one supervariable of 10 rows; cap 3 needs four parts and three splits
    A = _csr(np.ones((10, 10)))
    ex = _plan(A, slice_rows=3, partitioner=1).export()
    assert ef.same_multiset(ef.decode(ex), ef.triplets(A))
    assert list(np.diff(ex["part_ptr"])) in ([3, 2, 3, 2], [2, 3, 2, 3], [3, 3, 2, 2], [2, 2, 3, 3])


def test_edge_cases():
    for n in (0, 1, 2, 31, 33):
        A = gen.random_csr(n, 3, mean_row=2, empty_frac=0.3)
        ex = _plan(A, slice_rows=16, partitioner=1).export()
        assert ef.same_multiset(ef.decode(ex), ef.triplets(A))
    D = _csr(sp.identity(1000))                                   # no edges at all
    ex = _plan(D, slice_rows=64, partitioner=1).export()
    assert ef.same_multiset(ef.decode(ex), ef.triplets(D)) and np.diff(ex["part_ptr"]).max() <= 64
    A = gen.fem2d_p1(N=20)                                        # one part holds everything
    ex = _plan(A, slice_rows=A.n, partitioner=1).export()
    assert list(ex["part_ptr"]) == [0, A.n] and ex["row_er_count"].sum() == 0


def test_invalid_partitioner_is_refused():
    import paper_2204_06666_gb300 as eh
    A = gen.fem2d_p1(N=10)
    for bad in (-1, 2):
        with pytest.raises(eh.EhybError) as e:
            _plan(A, partitioner=bad)
        assert e.value.status == 1


@pytest.mark.parametrize("which", ["hex", "tet", "random"])
def test_multilevel_is_deterministic(which):
    A = {"hex": lambda: gen.hex_elast3d(N=12), "tet": lambda: gen.tet_lap3d(N=16, dirichlet=False),
         "random": lambda: gen.random_csr(20000, 9, mean_row=9, empty_frac=0.02, long_rows=3, long_len=900,
                                          duplicates=True)}[which]()
    keys = ("new_to_old", "part_ptr", "slice_pos", "ell_col", "er_scol")
    ref = _plan(A, slice_rows=900, partitioner=1, host_threads=1).export()
    for kw in (dict(host_threads=3), dict(host_threads=8), dict()):
        ex = _plan(A, slice_rows=900, partitioner=1, **kw).export()
        for k in keys:
            assert np.array_equal(np.asarray(ref[k]), np.asarray(ex[k])), (kw, k)
    other = _plan(A, slice_rows=900, partitioner=1, seed=12345).export()
    assert ef.same_multiset(ef.decode(other), ef.triplets(A))


def test_multilevel_cuts_fewer_entries_than_greedy_growing():
    cases = [(gen.hex_elast3d(N=20), -(-24000 // 152)), (gen.tet_lap3d(N=30, dirichlet=False), None)]
    for i in (1, 3, 5):
        cases.append((gen.tuner_matrix(i), None))
    for A, cap in cases:
        kw = dict(slice_rows=cap) if cap else dict()
        g, m = _er_fraction(A, **kw), _er_fraction(A, partitioner=1, **kw)
        assert m < g, (A.name, g, m)


def test_very_many_parts_fall_back_to_greedy_growing():
    # 20,000 rows in parts of one row: far more parts than the multilevel scheme is meant for
    A = gen.random_csr(20000, 8, mean_row=5, empty_frac=0.0)
    ex = _plan(A, slice_rows=1, partitioner=1).export()
    assert ef.same_multiset(ef.decode(ex), ef.triplets(A))
    assert np.all(np.diff(ex["part_ptr"]) == 1)
    g = _plan(A, slice_rows=1).export()
    assert np.array_equal(np.asarray(ex["new_to_old"]), np.asarray(g["new_to_old"]))
