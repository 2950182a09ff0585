"""The FSAI factor computed by the library's host code, for host-only plans (no GPU), against the oracle:
same pattern, same values; a matrix that is not SPD is refused."""
import numpy as np
import pytest

import gen
from oracle import fsai as of


@pytest.fixture(scope="module")
def eh():
    import paper_2204_06666_gb300 as m
    return m


@pytest.mark.parametrize("which", ["tet", "hex", "random"])
def test_fsai_factor_matches_oracle(eh, which):
    if which == "tet":
        A = gen.tet_lap3d(N=9)
    elif which == "hex":
        A = gen.hex_elast3d(N=5, clamp_minz=True)
    else:   # symmetric, diagonally dominant, duplicates and unsorted columns
        R = gen.random_csr(900, 3, mean_row=7, symmetric=True)
        import scipy.sparse as sp
        S = sp.csr_matrix((np.abs(R.val), R.col, R.row_ptr), shape=(R.n, R.n))
        S = (S + S.T).tocsr()
        d = np.asarray(abs(S).sum(axis=1)).ravel() + 1.0
        S = (S + sp.diags(d)).tocsr()
        A = gen.CSR(R.n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.copy())
    P = eh.Plan(A, host_only=1, num_sms=16, keep_host=1)
    M = eh.Fsai(P, A)
    rp, col, val = M.export()
    G = of.fsai(A, P.export()["new_to_old"])
    G.sort_indices()
    assert np.array_equal(rp, G.indptr) and np.array_equal(col, G.indices)
    assert np.allclose(val, G.data, rtol=1e-11, atol=1e-14)


def test_not_spd_is_refused(eh):
    A = gen.tet_lap3d(N=5)
    N = gen.CSR(A.n, A.row_ptr, A.col, -A.val)
    P = eh.Plan(N, host_only=1, num_sms=16)
    with pytest.raises(eh.EhybError) as e:
        eh.Fsai(P, N)
    assert e.value.status == 1


def test_host_only_preconditioner_closes_without_a_device():
    # a host-only plan's preconditioner holds no device memory: releasing it must not touch CUDA, and the
    # handle is gone after the first close (a second close and the destructor do nothing)
    import paper_2204_06666_gb300 as eh
    A = gen.tet_lap3d(N=6)
    P = eh.Plan(A, host_only=1, num_sms=4)
    M = eh.Fsai(P, A)
    M.close()
    M.close()
    P.close()
    P.close()
