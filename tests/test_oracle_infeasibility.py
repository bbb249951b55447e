"""Infeasibility detection of the oracle (Sec. "Infeasibility detection"),
pinned to facts outside the oracle: an LP solver confirms that the primal
instances have an empty constraint set and that the dual instances have a
feasible point and an explicit ray of negative curvature."""
import numpy as np
import pytest
from scipy.optimize import linprog

from paper_2609_19557_gb300 import instances as I


def _lp_feasible(inst):
    A = inst["A"].toarray()
    n = A.shape[1]
    lc, uc = inst["l_c"], inst["u_c"]
    rows_ub, rhs = [], []
    for i in range(A.shape[0]):
        if np.isfinite(uc[i]):
            rows_ub.append(A[i]); rhs.append(uc[i])
        if np.isfinite(lc[i]):
            rows_ub.append(-A[i]); rhs.append(-lc[i])
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(inst["l_x"], inst["u_x"])]
    r = linprog(np.zeros(n), A_ub=np.array(rows_ub), b_ub=np.array(rhs), bounds=bounds, method="highs")
    return r.status == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_primal_infeasible_detected(oracle, seed):
    inst = I.primal_infeasible_qp(seed)
    assert not _lp_feasible(inst)  # ground truth: empty constraint set
    x, y, info = oracle.solve(inst, eps_abs=1e-6, eps_rel=1e-6, time_limit=60)
    assert info["status_name"] == "PRIMAL_INFEASIBLE", info


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dual_infeasible_detected(oracle, seed):
    inst = I.dual_infeasible_qp(seed)
    assert _lp_feasible(inst)  # a feasible point exists ...
    e0 = np.zeros(inst["Q"].shape[0]); e0[0] = 1.0
    assert e0 @ (inst["Q"] @ e0) < 0 and np.abs(inst["A"] @ e0).max() == 0  # ... and a descent ray along x_0
    x, y, info = oracle.solve(inst, eps_abs=1e-6, eps_rel=1e-6, time_limit=60)
    assert info["status_name"] == "DUAL_INFEASIBLE", info


@pytest.mark.parametrize("seed", [0, 1])
def test_feasible_instances_not_flagged(oracle, seed):
    inst = I.small_qp(seed)
    x, y, info = oracle.solve(inst, eps_abs=1e-6, eps_rel=1e-6, time_limit=60)
    assert info["status_name"] == "SOLVED"
