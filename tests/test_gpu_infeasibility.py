"""Infeasibility detection on the GPU (Sec. "Infeasibility detection"): the
same status as the oracle, at the same outer iteration, on instances whose
infeasibility an LP solver confirms (tests/test_oracle_infeasibility.py)."""
import pytest

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


@pytest.mark.parametrize("kind,seed", [("primal", 0), ("primal", 1), ("primal", 2), ("dual", 0), ("dual", 1),
                                       ("dual", 2)])
@pytest.mark.parametrize("precision", [64, 32])
def test_infeasibility_status_matches_oracle(P, oracle, kind, seed, precision):
    inst = I.primal_infeasible_qp(seed) if kind == "primal" else I.dual_infeasible_qp(seed)
    _, _, ref = oracle.solve(inst, eps_abs=1e-6, eps_rel=1e-6, time_limit=60)
    h = P.create_from_instance(inst, precision=precision)
    P.pdnqp_set_param(h, "time_limit", 60)
    st = P.pdnqp_solve(h, 1e-6, 1e-6)
    _, _, r = P.pdnqp_get(h)
    h.close()
    want = "PRIMAL_INFEASIBLE" if kind == "primal" else "DUAL_INFEASIBLE"
    assert ref["status_name"] == want
    assert P.STATUS_NAMES[st] == want, (P.STATUS_NAMES[st], r)
    if precision == 64:
        assert r["outer_iters"] == ref["outer_iters"], (r["outer_iters"], ref["outer_iters"])
