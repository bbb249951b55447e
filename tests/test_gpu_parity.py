"""GPU path vs the FP64 oracle: per-step parity of Algorithm 4 and end-to-end
KKT acceptance, through the C ABI."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import instances as I

pytestmark = pytest.mark.gpu

REL = 1e-10  # per-step parity bound for the FP64 form (relative, per vector)


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


def compare_snaps(gpu, ref, rel=REL):
    assert len(gpu) == len(ref)
    worst = 0.0
    for s, r in zip(gpu, ref):
        assert s["t_total"] == r["t_total"]
        assert s["trials"] == r["trials"], (s["t_total"], s["trials"], r["trials"])
        assert s["restarts"] == r["restarts"], s["t_total"]
        assert s["t"] == r["t"]
        assert s["kappa"] == r["kappa"]
        assert abs(s["omega"] - r["omega"]) <= rel * abs(r["omega"])
        for key in ("w", "y", "wbar", "ybar"):
            e = rel_err(s[key], r[key])
            worst = max(worst, e)
            assert e <= rel, (key, s["t_total"], e)
    return worst


def test_small_per_step_parity_200(P, oracle):
    inst = I.small_qp(0)
    ck = list(range(1, 201))
    h = P.create_from_instance(inst)
    gpu = P.pdnqp_debug_inner(h, ck)
    ref, info = oracle.debug_inner(inst, ck)
    assert abs(P.pdnqp_get_param(h, "gamma") - info["gamma"]) <= 1e-10 * info["gamma"]
    compare_snaps(gpu, ref)
    h.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_small_parity_other_seeds(P, oracle, seed):
    inst = I.small_qp(seed)
    ck = [1, 2, 3, 10, 63, 64, 65, 128, 200]
    h = P.create_from_instance(inst)
    compare_snaps(P.pdnqp_debug_inner(h, ck), oracle.debug_inner(inst, ck)[0])
    h.close()


def test_mid_per_step_parity(P, oracle):
    """n = 50,000, m = 25,000: power-law rows up to 200 nnz, free variables, equality rows."""
    inst = I.mid_qp(0)
    ck = [1, 2, 5, 10, 64, 100, 128, 200]
    h = P.create_from_instance(inst)
    gpu = P.pdnqp_debug_inner(h, ck)
    ref, info = oracle.debug_inner(inst, ck)
    assert abs(P.pdnqp_get_param(h, "gamma") - info["gamma"]) <= 1e-10 * info["gamma"]
    compare_snaps(gpu, ref)
    h.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_small_end_to_end(P, oracle, eps):
    inst = I.small_qp(0)
    h = P.create_from_instance(inst)
    st = P.pdnqp_solve(h, eps, eps)
    x, y, res = P.pdnqp_get(h)
    assert st == P.PDNQP_SOLVED, P.STATUS_NAMES[st]
    assert oracle.kkt_pass(inst, x, y, eps, eps)
    # Same algorithm, same decisions: the oracle's outer iteration count matches closely.
    xo, yo, info = oracle.solve(inst, eps_abs=eps, eps_rel=eps)
    assert info["status"] == 0
    assert abs(res["outer_iters"] - info["outer_iters"]) <= max(2, 0.1 * info["outer_iters"])
    h.close()


def test_mid_end_to_end(P, oracle):
    inst = I.mid_qp(0)
    h = P.create_from_instance(inst)
    P.pdnqp_set_param(h, "time_limit", 300)
    st = P.pdnqp_solve(h, 1e-4, 1e-4)
    x, y, res = P.pdnqp_get(h)
    assert st == P.PDNQP_SOLVED, (P.STATUS_NAMES[st], res)
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
    h.close()


def test_solve_twice_is_reproducible(P):
    inst = I.small_qp(3)
    h = P.create_from_instance(inst)
    P.pdnqp_solve(h, 1e-5, 1e-5)
    x1, y1, r1 = P.pdnqp_get(h)
    P.pdnqp_solve(h, 1e-5, 1e-5)
    x2, y2, r2 = P.pdnqp_get(h)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    assert r1["inner_iters"] == r2["inner_iters"]
    h.close()
