"""Dense coupling rows (rows of A longer than the split threshold): products
split evenly over the blocks of the row pass and combined in block order.
Per-step parity of Algorithm 4 against the FP64 oracle in both loop forms
(persistent cooperative launch and graph replay), on the paper's soft-label
and SVM families (capacity rows, y'alpha = 0) and on an instance with more
dense rows than the split takes (the rest stay row-wise)."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2609_19557_gb300 import instances as I
from test_gpu_parity import P, compare_snaps  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

CK = [1, 2, 5, 10, 64, 100, 128, 200]


def many_dense_rows(seed=5, n=1500, dense=70, length=1100, sparse_rows=30):
    """small_qp's Q with A = `dense` rows of `length` entries plus sparse rows."""
    base = I.small_qp(seed, n=n, m=sparse_rows)
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n, size=length, replace=False)) for _ in range(dense)]
    D = sp.csr_matrix((rng.standard_normal(dense * length), np.concatenate(rows), np.arange(dense + 1) * length),
                      shape=(dense, n))
    A = sp.vstack([base["A"], D]).tocsr()
    x0 = base["x0"]
    ax = A @ x0
    lo, hi = ax - rng.uniform(0.1, 1.0, A.shape[0]), ax + rng.uniform(0.1, 1.0, A.shape[0])
    eq = rng.random(A.shape[0]) < 0.2
    hi[eq] = lo[eq] = ax[eq]
    return I._pack(base["Q"], base["c"], A, lo, hi, base["l_x"], base["u_x"], x0, workload="dense_rows")


CASES = {
    "svm": lambda: I.svm_qp(101, n_target=3000),
    "softlabel": lambda: I.softlabel_qp(104, n_target=12000),
    "many": many_dense_rows,
}


@pytest.fixture(scope="module")
def refs(oracle):
    out = {}
    for k, f in CASES.items():
        inst = f()
        out[k] = (inst, oracle.debug_inner(inst, CK)[0])
    return out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("persistent", [1, 0])
def test_dense_rows_per_step_parity(P, refs, case, persistent):
    inst, ref = refs[case]
    assert np.diff(inst["A"].indptr).max() > 1024  # the split is exercised
    h = P.create_from_instance(inst)
    P.pdnqp_set_param(h, "persistent", persistent)
    compare_snaps(P.pdnqp_debug_inner(h, CK), ref)
    h.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_dense_rows_deterministic(P, precision):
    """Two solves of the same instance give the same bits (fixed combination order)."""
    inst = I.svm_qp(102, n_target=4000)
    res = []
    for _ in range(2):
        h = P.create_from_instance(inst, precision=precision)
        P.pdnqp_set_param(h, "time_limit", 20.0)
        P.pdnqp_set_param(h, "k_out", 5)
        P.pdnqp_solve(h, 1e-6, 1e-6)
        x, y, r = P.pdnqp_get(h)
        res.append((x, y, r["inner_iters"]))
        h.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]


@pytest.mark.parametrize("precision", [64, 32])
def test_flow_end_to_end(P, oracle, precision):
    inst = I.flow_qp(101, n_target=1500)
    h = P.create_from_instance(inst, precision=precision)
    P.pdnqp_set_param(h, "time_limit", 60.0)
    st = P.pdnqp_solve(h, 1e-4, 1e-4)
    x, y, r = P.pdnqp_get(h)
    h.close()
    assert P.STATUS_NAMES[st] == "SOLVED", r
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
