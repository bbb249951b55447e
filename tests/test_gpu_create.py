"""pdnqp_create's host preparation (validation, explicit diagonal, row
ordering, transpose, all parallel over row ranges): errors on bad input, and
unsorted rows give the same result as sorted ones."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2609_19557_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_19557_gb300 import build as B
    from paper_2609_19557_gb300 import pdnqp
    B.build()
    pdnqp.load()
    return pdnqp


def _create(P, inst, **over):
    d = dict(inst)
    d.update(over)
    return P.pdnqp_create(d["Q"], d["c"], d["A"], d["l_c"], d["u_c"], d["l_x"], d["u_x"])


def _expect(P, code, inst, **over):
    with pytest.raises(P.PdnqpError) as e:
        _create(P, inst, **over)
    assert f"pdnqp error {code}:" in str(e.value), str(e.value)


def test_rejects_bad_input(P):
    inst = I.small_qp(0)
    Q = inst["Q"].tolil()
    Q[0, 5] = Q[0, 5] + 1.0  # breaks symmetry
    _expect(P, -3, inst, Q=Q.tocsr())
    A = inst["A"].copy()
    A.indices[1] = A.indices[0]  # duplicate column in row 0
    A.has_sorted_indices = False
    _expect(P, -1, inst, A=A)
    A = inst["A"].copy()
    A.indices[0] = inst["Q"].shape[0] + 3  # column out of range
    _expect(P, -1, inst, A=A)
    lc = inst["l_c"].copy()
    lc[2] = inst["u_c"][2] + 1.0
    _expect(P, -2, inst, l_c=lc)
    Qn = inst["Q"].copy()
    Qn.data[0] = np.nan
    _expect(P, -2, inst, Q=Qn)


def test_unsorted_rows_match_sorted(P):
    inst = I.mid_qp(1, n=6000, m=3000, replica_n=3000)
    rng = np.random.default_rng(0)

    def shuffled(M):
        M = M.copy()
        for i in range(M.shape[0]):
            b, e = M.indptr[i], M.indptr[i + 1]
            p = rng.permutation(e - b) + b
            M.indices[b:e] = M.indices[p]
            M.data[b:e] = M.data[p]
        M.has_sorted_indices = False
        return M

    res = []
    for Q, A in ((inst["Q"], inst["A"]), (shuffled(inst["Q"]), shuffled(inst["A"]))):
        h = _create(P, inst, Q=Q, A=A)
        P.pdnqp_set_param(h, "iter_budget", 500)
        P.pdnqp_solve(h, 1e-4, 1e-4)
        res.append(P.pdnqp_get(h)[:2])
        h.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
