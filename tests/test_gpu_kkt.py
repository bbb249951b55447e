"""pdnqp_kkt_residuals (external KKT test of Sec. 4.1 on device data) vs the oracle's checker."""
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


def _points(inst, rng):
    n, m = inst["Q"].shape[0], inst["A"].shape[0]
    lx = np.where(np.isfinite(inst["l_x"]), inst["l_x"], -2.0)
    ux = np.where(np.isfinite(inst["u_x"]), inst["u_x"], 2.0)
    yield inst["x0"], np.zeros(m)
    yield rng.uniform(lx - 0.1, ux + 0.1), rng.normal(size=m)  # slightly outside the box too
    yield np.clip(rng.normal(size=n), lx, ux), rng.normal(scale=10, size=m)


@pytest.mark.parametrize("workload", ["small", "mid"])
def test_kkt_residuals_match_oracle(P, oracle, workload):
    import torch
    inst = I.small_qp(1) if workload == "small" else I.mid_qp(1)
    prob = P.DeviceProblem(inst)
    rng = np.random.default_rng(7)
    for x, y in _points(inst, rng):
        xd = torch.as_tensor(x, device="cuda", dtype=torch.float64)
        yd = torch.as_tensor(y, device="cuda", dtype=torch.float64)
        out = torch.zeros(4, device="cuda", dtype=torch.float64)
        P.pdnqp_kkt_residuals(prob, xd, yd, out)
        got = out.cpu().numpy()
        ref = np.array(oracle.kkt_check(inst, x, y))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-14), (got, ref)


def test_kkt_residuals_of_solution(P, oracle):
    import torch
    inst = I.small_qp(2)
    h = P.create_from_instance(inst)
    assert P.pdnqp_solve(h, 1e-6, 1e-6) == P.PDNQP_SOLVED
    x, y, res = P.pdnqp_get(h)
    h.close()
    prob = P.DeviceProblem(inst)
    out = torch.zeros(4, device="cuda", dtype=torch.float64)
    P.pdnqp_kkt_residuals(prob, torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), out)
    rp, rd, sp, sd = out.cpu().numpy()
    assert rp <= 1e-6 + 1e-6 * sp and rd <= 1e-6 + 1e-6 * sd
    # the solver's own report uses the same definition
    assert np.allclose([rp, rd, sp, sd], [res["r_p"], res["r_d"], res["s_p"], res["s_d"]], rtol=1e-9, atol=1e-12)


def test_kkt_residuals_rejects_bad_input(P):
    import ctypes
    prob = P.pdnqp_device_problem()  # all zero: n = 0
    rc = P.load().pdnqp_kkt_residuals(ctypes.byref(prob), None, None, None, None)
    assert rc == -1
    assert P.load().pdnqp_kkt_last_error()


@pytest.mark.parametrize("where", ["x_first", "x_mid", "x_last", "y_mid", "x_inf"])
def test_kkt_residuals_reject_nonfinite_point(P, oracle, where):
    """A point with one NaN (or infinite) entry never passes the external KKT test
    (Sec. 4.1): the maxima of Eqs. outer-residuals must not drop it, in either entry
    point, and the oracle's checker agrees."""
    import torch
    inst = I.small_qp(2)
    h = P.create_from_instance(inst)
    assert P.pdnqp_solve(h, 1e-6, 1e-6) == P.PDNQP_SOLVED
    x, y, _ = P.pdnqp_get(h)
    h.close()
    assert oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)
    x, y = x.copy(), y.copy()
    pos = {"x_first": 0, "x_mid": x.size // 2, "x_last": x.size - 1}
    if where == "y_mid":
        y[y.size // 2] = np.nan
    elif where == "x_inf":
        x[x.size // 3] = np.inf
    else:
        x[pos[where]] = np.nan
    assert not oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)
    prob = P.DeviceProblem(inst)
    for fn in (P.pdnqp_kkt_residuals, P.pdnqp_kkt_residuals_noalloc):
        out = torch.zeros(4, device="cuda", dtype=torch.float64)
        fn(prob, torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), out)
        torch.cuda.synchronize()
        rp, rd, sp, sd = out.cpu().numpy()
        assert np.isfinite(sp) and np.isfinite(sd), (fn.__name__, sp, sd)
        assert not (rp <= 1e-6 + 1e-6 * sp and rd <= 1e-6 + 1e-6 * sd), (fn.__name__, rp, rd)
