"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

No GPU.  Each test names the passage it pins.  Brute force (active-set
enumeration), closed forms, library special cases (numpy eigvalsh) and
invariants are used so that a dropped term, a wrong sign, index or operand in
the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import bruteforce as BF
from paper_2609_19557_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(Q, c, A, lc, uc, lx, ux):
    return dict(Q=sp.csr_matrix(np.atleast_2d(Q)), c=np.asarray(c, float), A=sp.csr_matrix(A, shape=np.shape(A)),
                l_c=np.asarray(lc, float), u_c=np.asarray(uc, float), l_x=np.asarray(lx, float),
                u_x=np.asarray(ux, float))


# ---------------------------------------------------------------------------
# Sec. 1.2: projection onto a box
# ---------------------------------------------------------------------------
def test_projection_idempotent_and_feasible(oracle):
    rng = np.random.default_rng(0)
    lo = rng.normal(size=500) - 1
    hi = lo + rng.uniform(0, 2, size=500)
    lo[::7], hi[::11] = -np.inf, np.inf
    v = rng.normal(scale=3, size=500)
    p = oracle.project(v, lo, hi)
    assert np.all(p >= lo) and np.all(p <= hi)
    assert np.array_equal(oracle.project(p, lo, hi), p)
    inside = (v >= lo) & (v <= hi)
    assert np.array_equal(p[inside], v[inside])
    # Euclidean projection onto a box: closest point, componentwise (library special case).
    assert np.allclose(p, np.minimum(np.maximum(v, lo), hi))


# ---------------------------------------------------------------------------
# Sec. 3.1: Ruiz equilibration and the Lanczos eigenvalue estimate
# ---------------------------------------------------------------------------
def test_ruiz_equilibrates_rows_and_columns(oracle):
    inst = I.small_qp(1)
    A = inst["A"]
    As, Dc, Dx = oracle.ruiz_outer(A, 8)
    # The returned matrix is Dc A Dx.
    assert np.allclose(As.toarray(), np.diag(Dc) @ A.toarray() @ np.diag(Dx), rtol=1e-14, atol=0)
    a = np.abs(As.toarray())
    assert np.all(np.abs(a.max(1) - 1) < 0.05)
    nz = a.max(0) > 0
    assert np.all(np.abs(a.max(0)[nz] - 1) < 0.05)
    # KKT form: columns see Q's column too.
    As, Dc, Dx = oracle.ruiz_outer(A, 12, inst["Q"])
    q = np.abs(np.diag(Dx) @ inst["Q"].toarray() @ np.diag(Dx))
    col = np.maximum(np.abs(As.toarray()).max(0), q.max(0))
    assert np.all(np.abs(col - 1) < 0.01)
    # Zero sweeps is the identity.
    _, Dc0, Dx0 = oracle.ruiz_outer(A, 0)
    assert np.all(Dc0 == 1) and np.all(Dx0 == 1)


def test_tridiagonal_min_eig_closed_form(oracle):
    # T = tridiag(-1, 2, -1) of size k has eigenvalues 2 - 2cos(j pi/(k+1)).
    for k in (1, 2, 5, 40):
        got = oracle.tridiag_min_eig(np.full(k, 2.0), np.full(k - 1, -1.0))
        assert abs(got - (2 - 2 * np.cos(np.pi / (k + 1)))) < 1e-13


def test_lanczos_matches_eigvalsh(oracle):
    inst = I.small_qp(2)
    Q = inst["Q"]
    lam = np.linalg.eigvalsh(Q.toarray())[0]
    assert abs(oracle.lanczos_min(Q, 200, 1) - lam) < 1e-10  # full Krylov space
    assert abs(oracle.lanczos_min(Q, 64, 1) - lam) < 1e-6
    assert oracle.lanczos_min(Q, 10, 1) >= lam - 1e-12  # Ritz values bound lambda_min from above


def test_gamma_makes_inner_hessian_positive_definite(oracle):
    """Eq. base-strong-convexity / R-choice: Q + gamma^-1 I > 0 on the scaled data."""
    for seed in range(3):
        inst = I.small_qp(seed)
        info = oracle.setup_info(inst)
        Dx, cs = info["Dx"], info["cs"]
        Qs = cs * np.diag(Dx) @ inst["Q"].toarray() @ np.diag(Dx)
        ev = np.linalg.eigvalsh(Qs)
        g = info["gamma"]
        assert ev[0] + 1.0 / g > 0
        assert abs(info["qnorm"] - np.abs(Qs).sum(1).max()) < 1e-12
        expect = 1.0 / (max(0.0, -ev[0]) + 1e-2 * max(1.0, info["qnorm"]))
        assert abs(g - expect) / expect < 1e-6
        assert info["qnorm"] <= 1 + 1e-12  # objective scalar c_s bounds ||Q||


# ---------------------------------------------------------------------------
# Sec. 2.2: the residual-form inner QP (Eq. prox-alm-subproblem / inner-qp)
# ---------------------------------------------------------------------------
def test_residual_form_equals_proximal_alm(oracle):
    """Eliminating r recovers Eq. base-proximal-alm (row-wise sigma, Eq. practical-multiplier-update)."""
    rng = np.random.default_rng(3)
    for seed in range(4):
        t = I.tiny_qp(seed, n=5, m=3, eq_rows=1)
        gamma, z = 0.7, rng.uniform(0, 1, 5)
        lam, sig = rng.normal(size=3), rng.uniform(0.5, 3, 3)
        D = oracle.inner_qp_dense(t, z, lam, sig, gamma, no_scaling=1)
        n, m, mE, mI = D["n"], D["m"], D["mE"], D["mI"]
        assert (mE, mI) == (1, 2) and D["dw"] == n + mI + m
        Q, A, c = t["Q"].toarray(), t["A"].toarray(), t["c"]
        for _ in range(3):
            x = rng.uniform(0, 1, n)
            s = rng.uniform(t["l_c"][1:], t["u_c"][1:])
            rE = A[:1] @ x - t["l_c"][:1]
            rI = A[1:] @ x - s
            w = np.concatenate([x, s, rE, rI])
            assert np.allclose(D["B"] @ w, D["h"], atol=1e-14)
            inner = 0.5 * w @ D["H"] @ w + D["q"] @ w
            r = np.concatenate([rE, rI])
            alm = 0.5 * x @ Q @ x + c @ x + lam @ r + 0.5 * np.sum(sig * r * r)
            prox = alm + np.sum((x - z) ** 2) / (2 * gamma)
            assert abs(inner - (prox - np.sum(z ** 2) / (2 * gamma))) < 1e-12
        # Bounds of Eq. inner-bounds with the two-sided slack box.
        assert np.array_equal(D["lo"][:n], t["l_x"]) and np.array_equal(D["hi"][:n], t["u_x"])
        assert np.array_equal(D["lo"][n:n + mI], t["l_c"][1:]) and np.array_equal(D["hi"][n:n + mI], t["u_c"][1:])
        assert np.all(np.isinf(D["lo"][n + mI:])) and np.all(np.isinf(D["hi"][n + mI:]))


def test_inner_qp_strongly_convex_on_kernel(oracle):
    """Sec. 2.2: H_k >= 0 and positive definite on ker B."""
    t = I.tiny_qp(5, n=6, m=3, eq_rows=1)
    info = oracle.setup_info(t, no_scaling=1)
    D = oracle.inner_qp_dense(t, np.zeros(6), np.zeros(3), np.full(3, 2.0), info["gamma"], no_scaling=1)
    assert np.linalg.eigvalsh(D["H"])[0] > -1e-12
    _, sv, vt = np.linalg.svd(D["B"])
    Z = vt[D["m"]:].T  # basis of ker B (B has full row rank)
    assert np.linalg.eigvalsh(Z.T @ D["H"] @ Z)[0] > 1e-8


@pytest.mark.parametrize("seed", range(6))
def test_inner_solution_matches_bruteforce(oracle, seed):
    """Algorithm 4 converges to the unique minimiser of Eq. inner-qp (active-set enumeration),
    and its dual y is the multiplier of Bw = h, so -y = lambda + sigma r (Eq. base-inner-saddle)."""
    rng = np.random.default_rng(100 + seed)
    n, m = 4 + seed % 2, 3
    t = I.tiny_qp(seed, n=n, m=m, eq_rows=seed % 3)
    info = oracle.setup_info(t, no_scaling=1)
    gamma = info["gamma"]
    z, lam, sig = rng.uniform(0, 1, n), rng.normal(size=m), rng.uniform(0.3, 5, m)
    D = oracle.inner_qp_dense(t, z, lam, sig, gamma, no_scaling=1)
    w, y = BF.inner_qp_minimizer(D["H"], D["q"], D["B"], D["h"], D["lo"], D["hi"])
    perm = D["perm"]
    x, yo, st, it = oracle.inner_solve_given(t, z, lam, sig, gamma, tol=1e-11, kin=2_000_000, no_scaling=1)
    assert st == 0
    assert np.abs(x - w[:n]).max() < 1e-8
    assert np.abs(yo - y).max() < 1e-7
    # -y = lambda + sigma * r at the minimiser (stationarity in r).
    r = w[n + D["mI"]:]
    assert np.allclose(-y, lam + sig * r, atol=1e-9)
    # Outer scaling on: same minimiser in the original coordinates.
    del perm


# ---------------------------------------------------------------------------
# Algorithm 4 step rules (Eqs. pdqp-trial, diagonal-scales, diagonal-steps)
# ---------------------------------------------------------------------------
def test_diagonal_scales_hand_example(oracle):
    """Worked example in tests/golden/diagonal_scales_1x1.json (values derived by hand)."""
    g = json.load(open(os.path.join(GOLDEN, "diagonal_scales_1x1.json")))
    t = _inst([[g["Q"]]], [g["c"]], [[g["A"]]], [g["l_c"]], [g["u_c"]], [g["l_x"]], [g["u_x"]])
    info = oracle.setup_info(t, no_scaling=1, gamma_override=g["gamma"])
    assert abs(info["sigma0"] - g["sigma0"]) < 1e-12
    st = oracle.inner_steps(t, no_scaling=1, ruiz_inner=0, gamma_override=g["gamma"])
    assert np.allclose(st["mw"], g["m_w"], rtol=1e-14)
    assert np.allclose(st["my"], g["m_y"], rtol=1e-14)


def test_averages_and_momentum_weights(oracle):
    """alpha_t = 2/(t+2), wbar_{t+1} = (1-alpha_t) wbar_t + alpha_t w_{t+1}, beta_t = t/(t+1)."""
    inst = I.small_qp(3)
    snaps, info = oracle.debug_inner(inst, [1, 2, 3, 4])
    s1, s2, s3, s4 = snaps
    assert np.array_equal(s1["wbar"], s1["w"]) and np.array_equal(s1["ybar"], s1["y"])  # alpha_0 = 1
    assert np.allclose(s2["wbar"], s1["wbar"] / 3 + 2 * s2["w"] / 3, rtol=1e-12, atol=1e-14)
    assert np.allclose(s3["wbar"], s2["wbar"] / 2 + s3["w"] / 2, rtol=1e-12, atol=1e-14)
    assert np.allclose(s4["ybar"], 0.6 * s3["ybar"] + 0.4 * s4["y"], rtol=1e-12, atol=1e-14)
    assert [s["t_total"] for s in snaps] == [1, 2, 3, 4]


def test_dual_step_extrapolation(oracle):
    """Eq. pdqp-trial (dual part) at t = 1 (beta = 1/2) without inner Ruiz (dy = 1)."""
    inst = I.small_qp(4)
    prm = dict(ruiz_inner=0)
    info = oracle.setup_info(inst, **prm)
    snaps, _ = oracle.debug_inner(inst, [1, 2], **prm)
    st = oracle.inner_steps(inst, **prm)
    D = oracle.inner_qp_dense(inst, np.zeros(200), np.zeros(100), np.full(100, info["sigma0"]), info["gamma"])
    s1, s2 = snaps
    assert s2["trials"] == 2 and s2["kappa"] == 1.0  # no rejection in this example
    eta = 0.99 * s2["omega"] * s2["kappa"] / st["my"]
    Bw1, Bw2 = D["B"] @ s1["w"], D["B"] @ s2["w"]
    pred = s1["y"] + eta * (D["h"] - Bw2 - 0.5 * (Bw2 - Bw1))
    assert np.allclose(s2["y"], pred, rtol=1e-9, atol=1e-12)
    # Primal step at t = 1: w_md = (1 - 2/3) wbar + 2/3 w, projected gradient step.
    tau = 0.99 * s2["kappa"] / (s2["omega"] * st["mw"] * st["ew"] ** -2)
    wmd = s1["wbar"] / 3 + 2 * s1["w"] / 3
    grad = D["H"] @ wmd + D["q"] - D["B"].T @ s1["y"]
    pred_w = np.clip(s1["w"] - tau * grad, D["lo"], D["hi"])
    assert np.allclose(s2["w"], pred_w, rtol=1e-9, atol=1e-12)


def test_rejections_shrink_steps(oracle):
    """Rejected trials (Eq. adaptive-condition fails) halve kappa; restarts reset it to 1."""
    inst = I.small_qp(0)
    snaps, _ = oracle.debug_inner(inst, list(range(1, 65)))
    for s in snaps:
        k = s["kappa"]
        assert k == 0.5 ** round(-np.log2(k))
    last = snaps[-1]
    assert last["trials"] >= last["t_total"]


# ---------------------------------------------------------------------------
# Outer method end to end (Algorithm 3): KKT points by brute force
# ---------------------------------------------------------------------------
def test_sign_convention_closed_forms(oracle):
    """Eq. kkt-stationarity sign convention: lambda <= 0 on an active >= row, >= 0 on an active <= row."""
    # min x  s.t. x >= 1  ->  x = 1, 1 + lambda = 0.
    t = _inst([[0.0]], [1.0], [[1.0]], [1.0], [np.inf], [-10.0], [10.0])
    x, y, info = oracle.solve(t, eps_abs=1e-9, eps_rel=1e-9)
    assert info["status"] == 0 and abs(x[0] - 1) < 1e-7 and abs(y[0] + 1) < 1e-6
    # min -x  s.t. x <= 1  ->  lambda = +1.
    t = _inst([[0.0]], [-1.0], [[1.0]], [-np.inf], [1.0], [-10.0], [10.0])
    x, y, info = oracle.solve(t, eps_abs=1e-9, eps_rel=1e-9)
    assert info["status"] == 0 and abs(x[0] - 1) < 1e-7 and abs(y[0] - 1) < 1e-6
    # min 2x  s.t. 3x = 1.5  ->  x = 0.5, 2 + 3 lambda = 0.
    t = _inst([[0.0]], [2.0], [[3.0]], [1.5], [1.5], [-10.0], [10.0])
    x, y, info = oracle.solve(t, eps_abs=1e-9, eps_rel=1e-9)
    assert info["status"] == 0 and abs(x[0] - 0.5) < 1e-7 and abs(y[0] + 2 / 3) < 1e-6


@pytest.mark.parametrize("q,c,lo,hi", [(-2.0, 0.3, 0.0, 1.0), (-1.0, -0.2, -1.0, 2.0), (-0.5, 0.0, -1.0, 1.0),
                                       (-3.0, 1.5, 0.0, 1.0), (2.0, -1.0, 0.0, 1.0)])
def test_one_dimensional_box_qp(oracle, q, c, lo, hi):
    """min 1/2 q x^2 + c x on [lo, hi]: the KKT set is {lo if q lo + c >= 0} U {hi if q hi + c <= 0}
    U {-c/q if inside}; the result must be one of them (Eq. kkt-stationarity)."""
    t = _inst([[q]], [c], np.zeros((0, 1)), [], [], [lo], [hi])
    x, y, info = oracle.solve(t, x0=np.array([0.5 * (lo + hi) + 0.1]), eps_abs=1e-10, eps_rel=1e-10)
    assert info["status"] == 0
    kkt = []
    if q * lo + c >= 0:
        kkt.append(lo)
    if q * hi + c <= 0:
        kkt.append(hi)
    if q != 0 and lo < -c / q < hi:
        kkt.append(-c / q)
    assert min(abs(x[0] - k) for k in kkt) < 1e-7


@pytest.mark.parametrize("seed", range(8))
def test_outer_kkt_point_bruteforce(oracle, seed):
    """The oracle's answer is (within tolerance) one of the KKT points found by enumerating
    every active set of bounds and rows (Eq. kkt-stationarity + feasibility + signs)."""
    n, m = 5, 3
    t = I.tiny_qp(seed, n=n, m=m, eq_rows=seed % 2)
    x, y, info = oracle.solve(t, eps_abs=1e-9, eps_rel=1e-9)
    assert info["status"] == 0
    pts = BF.qp_kkt_points(t["Q"].toarray(), t["c"], t["A"].toarray(), t["l_c"], t["u_c"], t["l_x"], t["u_x"])
    assert pts
    d = [np.abs(x - p[0]).max() for p in pts]
    k = int(np.argmin(d))
    assert d[k] < 1e-6
    assert np.abs(y - pts[k][1]).max() < 1e-5
    rp, rd, sp_, sd = oracle.kkt_check(t, x, y)
    assert rp <= 1e-9 * (1 + sp_) + 1e-9 and rd <= 1e-9 + 1e-9 * sd


@pytest.mark.parametrize("seed", range(4))
def test_convex_case_unique_solution(oracle, seed):
    """Q > 0: the QP has exactly one KKT point and the oracle finds it; zero duality gap."""
    n, m = 5, 2
    t = I.tiny_qp(seed, n=n, m=m, convex=True)
    pts = BF.qp_kkt_points(t["Q"].toarray(), t["c"], t["A"].toarray(), t["l_c"], t["u_c"], t["l_x"], t["u_x"])
    assert len(pts) == 1
    x, y, info = oracle.solve(t, eps_abs=1e-10, eps_rel=1e-10)
    assert info["status"] == 0
    assert np.abs(x - pts[0][0]).max() < 1e-7
    # Lagrangian dual value equals the primal value at the KKT point (convex: zero gap).
    Q, A, c = t["Q"].toarray(), t["A"].toarray(), t["c"]
    prim = 0.5 * x @ Q @ x + c @ x
    lam = y
    g = Q @ x + c + A.T @ lam
    mu_l, mu_u = np.maximum(g, 0), np.maximum(-g, 0)  # bound multipliers from stationarity
    lag = prim + lam @ (A @ x) - np.where(lam < 0, lam * t["l_c"], lam * t["u_c"]).sum() - mu_l @ (x - t["l_x"]) \
        - mu_u @ (t["u_x"] - x)
    assert abs(prim - lag) < 1e-7


def test_motzkin_straus_clique_bound(oracle):
    """Motzkin-Straus: min -x'A_G x over the simplex equals -(1 - 1/omega(G)); any KKT point
    has value >= that bound and the oracle's point is a KKT point."""
    import networkx as nx
    for seed in range(3):
        t = I.clique_qp(seed, n=12, p=0.4)
        G = nx.from_scipy_sparse_array(t["graph"])
        omega = max(len(c) for c in nx.find_cliques(G))
        x, y, info = oracle.solve(t, x0=t["x0"], eps_abs=1e-6, eps_rel=1e-6)
        assert info["status"] == 0
        assert np.all(x >= -1e-9) and abs(x.sum() - 1) < 1e-5
        obj = 0.5 * x @ t["Q"].toarray() @ x
        assert obj >= -(1 - 1 / omega) - 1e-5
        assert oracle.kkt_pass(t, x, y, 1e-6, 1e-6)


def test_multiplier_signs_and_complementarity(oracle):
    """lambda_I <= 0 on active lower sides, >= 0 on upper sides, 0 on strictly inactive rows
    (Eq. projected-multipliers, two-sided reading)."""
    inst = I.small_qp(5)
    x, y, info = oracle.solve(inst, eps_abs=1e-7, eps_rel=1e-7)
    assert info["status"] == 0
    ax = inst["A"] @ x
    lo, hi = inst["l_c"], inst["u_c"]
    ineq = lo != hi
    tol = 1e-5
    ytol = 1e-12 * max(1.0, np.abs(y).max())  # lambda + sigma (v - s) cancels up to rounding
    assert np.all(np.abs(y[ineq & (ax > lo + tol) & (ax < hi - tol)]) <= ytol)
    assert np.all(y[ineq & (ax > lo + tol)] >= -ytol)
    assert np.all(y[ineq & (ax < hi - tol)] <= ytol)
    assert np.abs(y[ineq & ((np.abs(ax - lo) < tol) | (np.abs(ax - hi) < tol))]).max() > 1e-3  # some rows bind


def test_kkt_checker_closed_forms(oracle):
    """External test of Sec. 4.1: zero at an exact KKT point; a bound violation of d gives r_p = d."""
    t = I.tiny_qp(0, n=5, m=3, eq_rows=1)
    pts = BF.qp_kkt_points(t["Q"].toarray(), t["c"], t["A"].toarray(), t["l_c"], t["u_c"], t["l_x"], t["u_x"])
    x, lam = pts[0]
    rp, rd, sp_, sd = oracle.kkt_check(t, x, lam)
    assert rp < 1e-12 and rd < 1e-12
    assert sp_ >= 1 and sd >= 1
    x2 = x.copy()
    x2[0] = t["u_x"][0] + 0.25
    rp2, *_ = oracle.kkt_check(t, x2, lam)
    ax = t["A"] @ x2
    viol = np.maximum(t["l_c"] - ax, 0).max(initial=0)
    viol = max(viol, np.maximum(ax - t["u_c"], 0).max(initial=0))
    assert abs(rp2 - max(0.25, viol)) < 1e-12



@pytest.mark.parametrize("where", ["x_first", "x_mid", "x_last", "y_first", "y_last", "x_inf"])
def test_kkt_checker_rejects_nonfinite_point(oracle, where):
    """External test of Sec. 4.1: a point with one NaN or infinite entry is not a KKT
    point, wherever the entry sits (a maximum built from plain comparisons keeps a
    NaN only when it comes last), while the scales stay finite."""
    t = I.tiny_qp(0, n=5, m=3, eq_rows=1)
    pts = BF.qp_kkt_points(t["Q"].toarray(), t["c"], t["A"].toarray(), t["l_c"], t["u_c"], t["l_x"], t["u_x"])
    x, lam = (np.array(v, dtype=float) for v in pts[0])
    assert oracle.kkt_pass(t, x, lam, 1e-8, 1e-8)
    if where == "x_inf":
        x[2] = np.inf
    elif where.startswith("x"):
        x[{"x_first": 0, "x_mid": 2, "x_last": 4}[where]] = np.nan
    else:
        lam[{"y_first": 0, "y_last": 2}[where]] = np.nan
    rp, rd, sp_, sd = oracle.kkt_check(t, x, lam)
    assert np.isfinite(sp_) and np.isfinite(sd)
    assert rp == np.inf or rd == np.inf
    assert not oracle.kkt_pass(t, x, lam, 1e-4, 1e-4)

def test_end_to_end_small_workload(oracle):
    """n = 200, m = 100 workload: relative KKT 1e-4 reached and verified externally."""
    inst = I.small_qp(0)
    x, y, info = oracle.solve(inst, eps_abs=1e-4, eps_rel=1e-4, time_limit=120)
    assert info["status"] == 0
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)
    assert np.all(x >= -1e-12) and np.all(x <= 1 + 1e-12)
