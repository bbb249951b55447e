"""Failure detection on the GPU without a fault: each bounded wait of the
persistent trial loop is made to run out (a grid barrier that one block never
reaches, a bulk-copy barrier that expects bytes nothing sends); every waiter
must give up, set the fault flag and return, and the context must stay
usable for a solve afterwards."""
import pytest

from paper_2609_19557_gb300 import instances as I
from test_gpu_parity import P  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1], ids=["grid_barrier", "bulk_copy_barrier"])
def test_bounded_wait_gives_up(P, oracle, kind):
    gave_up, seconds = P.pdnqp_selftest_wait(kind)
    assert gave_up
    assert seconds < 60.0
    inst = I.small_qp(0)
    h = P.create_from_instance(inst)
    st = P.pdnqp_solve(h, 1e-6, 1e-6)
    x, y, _ = P.pdnqp_get(h)
    h.close()
    assert P.STATUS_NAMES[st] == "SOLVED"
    assert oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)
