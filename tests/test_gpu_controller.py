"""Learned controller in the solver: the rules' path is untouched without it,
the network's proposals are judged by the rules (fallback), results still pass
the oracle's KKT test, and a small training run shows what the trained network
gains (or loses) against the method without it."""
import json

import numpy as np
import pytest

from paper_2609_19557_gb300 import instances as I
from paper_2609_19557_gb300 import mlp_data as D

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


def test_rule_path_trace(P):
    inst = I.small_qp(3)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP64)
    assert P.pdnqp_solve(h, 1e-6, 1e-6) == P.PDNQP_SOLVED
    _, _, r = P.pdnqp_get(h)
    tr = P.pdnqp_get_trace(h)
    h.close()
    assert tr.shape[1] == P.TRACE_COLS and 0 < len(tr) <= r["outer_iters"]
    assert np.array_equal(tr[:, 19:21], tr[:, 21:23])  # actions taken are the rules'
    assert not tr[:, 23].any() and r["ctrl_used"] == 0
    assert np.all(np.isfinite(tr))


def test_untrained_network_is_judged_by_the_rules(P, oracle):
    inst = I.small_qp(4)
    h = P.create_from_instance(inst, precision=P.PDNQP_FP32_BULK)
    P.pdnqp_set_controller(h, D.init_weights(5))
    P.pdnqp_set_param(h, "controller", 1)
    P.pdnqp_set_param(h, "time_limit", 120)
    st = P.pdnqp_solve(h, 1e-6, 1e-6)
    x, y, r = P.pdnqp_get(h)
    tr = P.pdnqp_get_trace(h)
    h.close()
    assert st == P.PDNQP_SOLVED, (P.STATUS_NAMES[st], r)
    assert oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)
    assert r["ctrl_used"] + r["ctrl_fallbacks"] == len(tr)
    assert r["ctrl_used"] == int(tr[:, 23].sum()) > 0
    # after a proposal that made the relative KKT residual worse, the rules decide
    for k in range(1, len(tr)):
        if tr[k - 1, 23] and tr[k, 1] > tr[k - 1, 1]:
            assert tr[k, 23] == 0 and np.array_equal(tr[k, 19:21], tr[k, 21:23])


def test_exploration_is_seeded(P):
    inst = I.small_qp(5)
    traces = []
    for _ in range(2):
        h = P.create_from_instance(inst, precision=P.PDNQP_FP64)
        P.pdnqp_set_param(h, "ctrl_explore", 0.5)
        P.pdnqp_set_param(h, "ctrl_seed", 11)
        P.pdnqp_solve(h, 1e-6, 1e-6)
        traces.append(P.pdnqp_get_trace(h))
        h.close()
    assert np.array_equal(traces[0], traces[1])
    assert not np.array_equal(traces[0][:, 19:21], traces[0][:, 21:23])


def test_trained_controller_gain(P, oracle):
    """Trains on trajectories of the mid-size generator at n = 2,000-4,000 with
    the library's kernels, then compares with the rules on fresh instances.
    The comparison is reported, not required to favour the network; every
    result must pass the oracle's KKT test."""
    from paper_2609_19557_gb300 import controller as CT
    rng = np.random.default_rng(3)
    data = []
    for i in range(24):
        n = int(rng.integers(2000, 4001))
        _, tr = CT.run(CT.make_instance(500 + i, n), eps=1e-4, explore=0.5, seed=i, time_limit=60)
        data += CT.transitions(tr)
    feats, acts, scores = zip(*data)
    theta, hist = CT.train(feats, acts, scores, epochs=1500)
    assert hist[-1][1] < hist[0][1]
    rows = []
    for j in range(6):
        n = int(rng.integers(2000, 4001))
        inst = CT.make_instance(900 + j, n)
        base, _ = CT.run(inst, eps=1e-4, time_limit=60)
        mlp, _ = CT.run(inst, eps=1e-4, controller=theta, time_limit=60)
        for res in (base, mlp):
            assert res["status"] == "SOLVED", res["status"]
            assert oracle.kkt_pass(inst, res["x"], res["y"], 1e-4, 1e-4)
        rows.append((base["outer"], mlp["outer"], base["inner"], mlp["inner"], mlp["ctrl_used"],
                     mlp["ctrl_fallbacks"]))
    R = np.array(rows, dtype=float)
    print("controller gain:", json.dumps({
        "transitions": len(data), "train_loss": hist,
        "outer_rule_vs_mlp": R[:, :2].sum(axis=0).tolist(), "inner_rule_vs_mlp": R[:, 2:4].sum(axis=0).tolist(),
        "ctrl_used": int(R[:, 4].sum()), "fallbacks": int(R[:, 5].sum())}))


def test_committed_controller_paired(P, oracle):
    """The committed network (paper_2609_19557_gb300/controller_weights.npy)
    against the paper's rules on 12 fresh instances of the mid-size generator
    at n = 10,000-20,000, paired (the same instances for both), each side
    solved to rel-KKT 1e-4 as one fused batch.  Solves are deterministic, so
    the paired counts are fixed for this library build.  Measured on the
    GB300: the network's totals are lower (outer 9,026 vs 9,595, inner
    1,089,728 vs 1,175,744), but it needs fewer outer iterations on only 6 of
    the 12 instances (exact two-sided sign test p = 1.0; inner 7 of 12,
    p = 0.77), as on the 32-instance evaluation (p = 0.60): the direction of
    the totals holds, with no confidence that it generalises instance by
    instance.  The test asserts the totals' direction and prints the test."""
    from paper_2609_19557_gb300 import controller as CT
    import os
    theta = np.load(os.path.join(os.path.dirname(CT.__file__), "controller_weights.npy")).astype(np.float32)
    rng = np.random.default_rng(11)
    ns = [int(rng.integers(10_000, 20_001)) for _ in range(12)]
    shift = CT.make_instance(71_000, ns[0])["shift"]
    insts = [CT.make_instance(71_000 + j, ns[j], shift) for j in range(12)]
    ev = CT.evaluate_batched(insts, theta, eps=1e-4, time_limit=300.0)
    for inst, e in zip(insts, ev):
        for side in ("rule", "mlp"):
            assert e[side]["status"] == "SOLVED", (side, e[side]["status"])
            assert oracle.kkt_pass(inst, e[side]["x"], e[side]["y"], 1e-4, 1e-4)
    stats = {}
    for key in ("outer", "inner"):
        d = [e["mlp"][key] - e["rule"][key] for e in ev]
        k, nn, p = CT.sign_test(d)
        stats[key] = {"rule_total": sum(e["rule"][key] for e in ev), "mlp_total": sum(e["mlp"][key] for e in ev),
                      "mlp_fewer": k, "nonzero": nn, "sign_test_p": p}
    print("committed controller, paired:", json.dumps(stats))
    assert all(e["mlp"]["ctrl_used"] > 0 for e in ev)
    assert stats["outer"]["mlp_total"] < stats["outer"]["rule_total"]
    assert stats["inner"]["mlp_total"] < stats["inner"]["rule_total"]
