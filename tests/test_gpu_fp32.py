"""FP32-bulk form: SpMVs, vector updates and the per-thread terms of the
acceptance sums in FP32; the block and grid reductions of the acceptance sums,
the check / restart / termination reductions, the multiplier and penalty
updates and the base point of each inner solve in FP64.  Error against the
FP64 oracle, and end-to-end KKT acceptance."""
import numpy as np
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


def rel_err(a, b):
    return np.abs(a - b).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300)


def test_fp32_iterates_track_fp64_oracle(P, oracle):
    """Stated error of the FP32-bulk iterates vs the FP64 oracle over the first
    200 iterations of the first inner solve (n=200 workload): below 1e-4 relative."""
    inst = I.small_qp(0)
    ck = [1, 10, 50, 100, 200]
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    gpu = P.pdnqp_debug_inner(h, ck)
    ref, _ = oracle.debug_inner(inst, ck)
    errs = []
    for s, r in zip(gpu, ref):
        assert s["t_total"] == r["t_total"]
        e = max(rel_err(s[k], r[k]) for k in ("w", "y", "wbar", "ybar"))
        errs.append(e)
    print("fp32 vs oracle rel err at", ck, ":", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-4
    h.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_fp32_end_to_end_small(P, oracle, eps):
    inst = I.small_qp(0)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    P.pdnqp_set_param(h, "time_limit", 120)
    st = P.pdnqp_solve(h, eps, eps)
    x, y, res = P.pdnqp_get(h)
    assert st == P.PDNQP_SOLVED, (P.STATUS_NAMES[st], res)
    assert oracle.kkt_pass(inst, x, y, eps, eps)
    h.close()


def test_fp32_end_to_end_mid(P, oracle):
    inst = I.mid_qp(0)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    P.pdnqp_set_param(h, "time_limit", 300)
    st = P.pdnqp_solve(h, 1e-4, 1e-4)
    x, y, res = P.pdnqp_get(h)
    assert st == P.PDNQP_SOLVED, (P.STATUS_NAMES[st], res)
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
    h.close()


def test_fp32_tight_tolerance_escalates_to_fp64(P, oracle):
    """n = 50,000 to rel-KKT 1e-6: the FP32-bulk form alone follows the FP64
    form's trajectory for about 25 outer iterations, then its inner solves
    stop converging within K_in and it ends in NUMERICAL_ERROR (the FP32
    form's limit on this workload); with the
    default escalation the handle continues as an FP64 solve from the same
    start point and returns a point that passes the oracle's KKT test at
    1e-6, flagged as escalated."""
    inst = I.mid_qp(0)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    P.pdnqp_set_param(h, "time_limit", 240.0)
    st = P.pdnqp_solve(h, 1e-6, 1e-6)
    x, y, r = P.pdnqp_get(h)
    esc = P.pdnqp_get_param(h, "escalated")
    h.close()
    print("fp32 1e-6 mid:", P.STATUS_NAMES[st], "escalated", esc, "outer", r["outer_iters"], "inner",
          r["inner_iters"], "seconds %.1f" % r["solve_seconds"])
    assert P.STATUS_NAMES[st] == "SOLVED", (P.STATUS_NAMES[st], r)
    assert oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)


def test_fp32_escalation_flag(P):
    """Parameter escalate (FP32-bulk handles): the default is on, a solve that
    does not end in NUMERICAL_ERROR is not escalated, and the flag and the
    rebase counter are readable."""
    inst = I.small_qp(0)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    assert P.pdnqp_get_param(h, "escalate") == 1
    st = P.pdnqp_solve(h, 1e-6, 1e-6)
    assert P.STATUS_NAMES[st] == "SOLVED"
    assert P.pdnqp_get_param(h, "escalated") == 0
    assert P.pdnqp_get_param(h, "rebases") >= 0
    h.close()
