"""Batched form: independent problems of uneven sizes solved together
(pdnqp_solve_batch), each with its own acceptance, restart and termination:
the fused form (all inner iterations in one launch per phase of one captured
CUDA graph) and the thread-pool form; and the row-binning autotuner of the
graph form."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import instances as I
from test_gpu_parity import P  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _batch():
    return I.batched_set(5, count=8, n_lo=1000, n_hi=3000, n_median=1800, sigma=0.4)


def _make(P, inst, precision, fused=1):
    h = P.create_from_instance(inst, precision=precision)
    P.pdnqp_set_param(h, "batch_fused", fused)
    # Bounded and deterministic (no time limit decides): 200 outer iterations
    # for the small generator, 20 for the slower Motzkin-Straus problems.
    P.pdnqp_set_param(h, "k_out", 200 if inst["workload"] == "small" else 20)
    P.pdnqp_set_param(h, "persistent", 0)
    return h


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("precision", [64, 32])
def test_batch_matches_sequential(P, oracle, precision, fused):
    """Each problem of the batch ends with the same status, bitwise the same
    iterates and the same counts as when it is solved alone in the graph form
    (the fused form gives each problem its solo block partition, so its
    reductions round the same way)."""
    insts = _batch()
    seq = []
    for inst in insts:
        h = _make(P, inst, precision)
        st = P.pdnqp_solve(h, 1e-4, 1e-4)
        x, y, r = P.pdnqp_get(h)
        seq.append((st, x, y, r["outer_iters"], r["inner_iters"]))
        h.close()
    hs = [_make(P, inst, precision, fused) for inst in insts]
    sts = P.pdnqp_solve_batch(hs, 1e-4, 1e-4, threads=4)
    solved = 0
    for k, (h, inst) in enumerate(zip(hs, insts)):
        x, y, r = P.pdnqp_get(h)
        assert sts[k] == seq[k][0]
        assert np.array_equal(x, seq[k][1]) and np.array_equal(y, seq[k][2])
        assert (r["outer_iters"], r["inner_iters"]) == seq[k][3:]
        if P.STATUS_NAMES[sts[k]] == "SOLVED":
            solved += 1
            assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
        h.close()
    assert solved >= 3  # the small-generator half solves within 200 outer iterations


def test_batch_arguments(P):
    assert P.pdnqp_solve_batch([], 1e-4, 1e-4) == []
    h = P.create_from_instance(I.small_qp(0))
    with pytest.raises(P.PdnqpError):
        P.pdnqp_solve_batch([h, h], 1e-4, 1e-4)
    h.close()


def test_autotune_graph_form(P, oracle):
    inst = I.mid_qp(1, n=20000, m=10000, replica_n=2000)
    h = P.create_from_instance(inst, precision=32)
    P.pdnqp_set_param(h, "persistent", 0)
    P.pdnqp_set_param(h, "autotune", 1)
    P.pdnqp_set_param(h, "time_limit", 60.0)
    st = P.pdnqp_solve(h, 1e-4, 1e-4)
    x, y, r = P.pdnqp_get(h)
    assert P.STATUS_NAMES[st] == "SOLVED"
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
    assert P.pdnqp_get_param(h, "lanes_rows") in (4, 8, 16)
    assert P.pdnqp_get_param(h, "lanes_cols") in (4, 8, 16)
    h.close()
