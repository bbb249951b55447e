"""Pins of the oracle's restart, primal-weight and outer rules (no GPU).

The oracle exports a trace of its periodic checks (the quantities of the
restart decision and the iterates before it) and of its outer iterations (the
vectors and scalars each outer rule reads and writes).  Every test below
recomputes what the rule must give from the paper's definition, with numpy,
on a representation the oracle never uses (the dense unscaled inner QP of
Eq. inner-qp with the diagonal scalings applied as vectors, or the scaled
problem rebuilt from the setup's Ruiz factors), so a dropped term, a
transposed operand, a swapped constant or a wrong comparison in the oracle
fails here:

* kkt_metric / restart test (Sec. 3.3 restart paragraph; PDLP's criteria,
  reading A5) -> test_restart_metric_matches_definition,
  test_restart_decision_follows_pdlp_criteria;
* inner_residuals (Eqs. inner-residuals / inner-scales)
  -> test_inner_residuals_match_definition;
* primal-weight update (Eqs. primal-weight-movement / primal-weight-update)
  -> test_primal_weight_update;
* inner-tolerance factor (Eq. inner-tolerance-factor, floor reading A14)
  -> test_inner_tolerance_factor;
* center update (Eqs. center-update / center-tolerance-update, reading 18)
  -> test_center_update;
* row-penalty growth (Eq. penalty-trigger-eq, readings A12/A13) and the
  multiplier update (Eq. practical-multiplier-update) -> test_penalty_update,
  test_multiplier_update;
* scaled and original outer residuals (Eqs. outer-residuals / outer-scales)
  -> test_outer_residuals_recomputed;
* initial penalty (QPALM's rule, reading A12) -> test_initial_penalty_hand_cases.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2609_19557_gb300 import instances as I

# PDLP's published restart parameters (Applegate et al., "Practical large-scale
# linear programming using primal-dual hybrid gradient", 2021): sufficient
# decay 0.2, necessary decay 0.8, artificial restart after 0.36 of the
# iterations; Table tab:parameters: rho_in in [0.3, 0.95], rho_z = 0.95,
# theta_sigma = 0.25, sigma_init = 20.
BETA_SUFF, BETA_NEC, BETA_ART = 0.2, 0.8, 0.36
RHO_MIN, RHO_MAX, RHO_Z, THETA_SIGMA, SIGMA_INIT = 0.3, 0.95, 0.95, 0.25, 20.0
# Readings of the penalty growth (A12) and of the tolerance floor (A14).
DELTA_SIGMA, SIGMA_MAX, TOL_FLOOR = 2.0, 1e6, 0.1


def _proj(v, lo, hi):
    return np.minimum(np.maximum(v, lo), hi)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def checks(oracle):
    inst = I.small_qp(0)
    ck, info = oracle.debug_checks(inst, 24)
    assert len(ck) == 24
    steps = oracle.inner_steps(inst)
    # Inner QP of outer iteration 0: z = projected x0 = 0 (box [0, 1]), lambda = 0, sigma = sigma0.
    n, m = inst["Q"].shape[0], inst["A"].shape[0]
    qp = oracle.inner_qp_dense(inst, np.zeros(n), np.zeros(m), np.full(m, info["sigma0"]), info["gamma"])
    return ck, steps, qp


def _metric(qp, E, D, w, y, omega):
    """KKT_omega of reading A5 in the scaled inner space (w = E w~, y = D y~),
    written with the unscaled dense inner QP: B~ w~ - h~ = D (B w - h) and
    w~ - P(w~ - g~) = (w - P_[lo,hi](w - E^2 g)) / E with g = H w + q - B'y."""
    H, q, B, h, lo, hi = qp["H"], qp["q"], qp["B"], qp["h"], qp["lo"], qp["hi"]
    p = D * (B @ w - h)
    g = H @ w + q - B.T @ y
    d = (w - _proj(w - E * E * g, lo, hi)) / E
    return np.sqrt(omega * (p @ p) + (d @ d) / omega)


def test_restart_metric_matches_definition(checks):
    ck, st, qp = checks
    for c in ck:
        kc = _metric(qp, st["ew"], st["dy"], c["w"], c["y"], c["omega"])
        ka = _metric(qp, st["ew"], st["dy"], c["wbar"], c["ybar"], c["omega"])
        # relative 1e-9, plus rounding of B w - h and of the projected step (entries O(1))
        assert abs(c["k_cur"] - kc) <= 1e-9 * kc + 1e-12, (c["t_total"], c["k_cur"], kc)
        assert abs(c["k_avg"] - ka) <= 1e-9 * ka + 1e-12, (c["t_total"], c["k_avg"], ka)


def test_inner_residuals_match_definition(checks):
    """Eqs. inner-residuals / inner-scales at every check, for the current point
    and the average, recomputed from the dense unscaled inner QP:
    r_p = ||Bw - h||, r_d = ||w - P_W(w - H w - q + B'y)||, s_p = max(1, ||Bw||,
    ||h||), s_d = max(1, ||Hw||, ||q||, ||B'y||) (all l_inf)."""
    ck, _, qp = checks
    H, q, B, h, lo, hi = qp["H"], qp["q"], qp["B"], qp["h"], qp["lo"], qp["hi"]
    for c in ck:
        for tag, w, y in (("cur", c["w"], c["y"]), ("avg", c["wbar"], c["ybar"])):
            bw, hw, bty = B @ w, H @ w, B.T @ y
            rp = np.abs(bw - h).max()
            rd = np.abs(w - _proj(w - (hw + q - bty), lo, hi)).max()
            sp_ = max(1.0, np.abs(bw).max(), np.abs(h).max())
            sd = max(1.0, np.abs(hw).max(), np.abs(q).max(), np.abs(bty).max())
            for name, want, scale in (("rp", rp, sp_), ("rd", rd, sd), ("sp", sp_, sp_), ("sd", sd, sd)):
                got = c[f"{name}_{tag}"]
                assert abs(got - want) <= 1e-12 * scale, (c["t_total"], name, tag, got, want)


def test_restart_decision_follows_pdlp_criteria(checks):
    ck, _, _ = checks
    kinds = set()
    for c in ck:
        use_avg = c["k_avg"] < c["k_cur"]
        cand = c["k_avg"] if use_avg else c["k_cur"]
        suff = cand <= BETA_SUFF * c["k_restart"]
        nec = cand <= BETA_NEC * c["k_restart"] and cand > c["k_last"]
        art = c["t"] >= BETA_ART * c["t_total"]
        assert bool(c["use_avg"]) == use_avg
        assert bool(c["restart"]) == (suff or nec or art), c
        if c["restart"]:
            kinds.add("suff" if suff else ("nec" if nec else "art"))
            assert c["t_after"] == 0 and c["kappa_after"] == 1.0 and c["k_restart_after"] == cand
        else:
            kinds.add("none")
            assert c["t_after"] == c["t"] and c["kappa_after"] == c["kappa"] and c["omega_after"] == c["omega"]
            assert c["k_restart_after"] == c["k_restart"]
    # both outcomes, and a restart that the artificial criterion alone would not explain
    assert "none" in kinds and ("suff" in kinds or "nec" in kinds), kinds


def test_primal_weight_update(checks):
    ck, st, _ = checks
    E, D = st["ew"], st["dy"]
    seen = 0
    for c in ck:
        if not c["restart"]:
            continue
        w, y = (c["wbar"], c["ybar"]) if c["use_avg"] else (c["w"], c["y"])
        dW = np.linalg.norm((w - c["wst"]) / E)
        dY = np.linalg.norm((y - c["yst"]) / D)
        if dW > 0 and dY > 0:
            want = c["omega"] ** 0.75 * (dY / dW) ** 0.25
            seen += 1
        else:
            want = c["omega"]
        # the trace holds E w~ rather than w~: the movements lose about
        # 1e-16 ||w~|| / dW of relative precision to that rounding
        tol = 1e-10 + 1e-15 * (np.linalg.norm(w / E) / max(dW, 1e-300) + np.linalg.norm(y / D) / max(dY, 1e-300))
        assert _rel(c["omega_after"], want) < tol, (c["t_total"], c["omega_after"], want, tol)
    assert seen >= 3


@pytest.fixture(scope="module")
def outer(oracle):
    # mid-size generator at n = 600: equality rows, free variables, and outer
    # iterations where the center stays put
    inst = I.mid_qp(0, n=600, m=300)
    eps = 1e-4
    x, y, info, tr = oracle.solve_traced(inst, eps_abs=eps, eps_rel=eps, anderson=0)
    assert info["status_name"] == "SOLVED" and len(tr) > 10
    return inst, tr, oracle.setup_info(inst), eps


def test_inner_tolerance_factor(outer):
    _, tr, _, eps = outer
    floor_hit = interior = 0
    for t in tr:
        dx = np.abs(t["x"] - t["z"]).max()
        assert _rel(t["dx_inf"], dx) < 1e-14
        ratio = min(1.0, (dx / t["gamma"]) / t["sc_rd"]) if t["sc_rd"] > 0 else 1.0
        rho = RHO_MAX - (RHO_MAX - RHO_MIN) * ratio
        assert _rel(t["rho"], rho) < 1e-12
        assert t["sd_in"] >= 1.0  # Eq. inner-scales include 1
        assert _rel(t["dta_after"], max(t["dta"] * rho, TOL_FLOOR * eps)) < 1e-12
        assert _rel(t["dtr_after"], max(t["dtr"] * rho, TOL_FLOOR * eps)) < 1e-12
        floor_hit += t["dta"] * rho < TOL_FLOOR * eps
        interior += ratio < 0.999
    assert floor_hit and interior


def test_center_update(outer):
    _, tr, _, eps = outer
    moved = kept = 0
    for t in tr:
        go = t["sc_rp"] <= t["eak"] + t["erk"] * t["sc_sp"]
        assert bool(t["moved"]) == go
        if go:
            moved += 1
            assert np.array_equal(t["z_after"], t["x"])
            assert t["eak_after"] == max(t["eak"] * RHO_Z, eps) and t["erk_after"] == max(t["erk"] * RHO_Z, eps)
        else:
            kept += 1
            assert np.array_equal(t["z_after"], t["z"])
            assert t["eak_after"] == t["eak"] and t["erk_after"] == t["erk"]
    assert moved and kept


def test_penalty_update(outer):
    _, tr, info, _ = outer
    mE = info["mE"]
    grew = 0
    for t in tr:
        r, rp_, lam, sig = t["r"], t["r_prev"], t["lam"], t["sig"]
        assert _rel(t["r_inf"], np.abs(r).max()) < 1e-15
        active = (np.arange(r.size) < mE) | (lam != 0.0)
        trig = active & (not t["primal_ok"]) & (np.abs(r) > THETA_SIGMA * np.abs(rp_)) & (t["r_inf"] > 0)
        want = np.where(trig, np.minimum(SIGMA_MAX, sig * np.maximum(1.0, DELTA_SIGMA * np.abs(r) / t["r_inf"])), sig)
        assert np.allclose(t["sig_after"], want, rtol=1e-15, atol=0), np.abs(t["sig_after"] - want).max()
        grew += int((want > sig).sum())
    assert grew > 0


def _scaled(inst, info):
    """The scaled problem of Sec. 3.1 rebuilt from the setup's Ruiz factors and
    objective scalar: Q~ = c_s Dx Q Dx, c~ = c_s Dx c, A~ = Dc A[perm] Dx."""
    Dx, Dc, cs, perm = info["Dx"], info["Dc"], info["cs"], info["perm"]
    Q = cs * (sp.diags(Dx) @ inst["Q"] @ sp.diags(Dx))
    A = sp.diags(Dc) @ inst["A"][perm] @ sp.diags(Dx)
    return dict(Q=Q.toarray(), A=A.toarray(), c=cs * Dx * inst["c"], lx=inst["l_x"] / Dx, ux=inst["u_x"] / Dx,
                lc=Dc * inst["l_c"][perm], uc=Dc * inst["u_c"][perm])


def test_multiplier_update(outer):
    """Eq. practical-multiplier-update (two-sided rows, reading A1): with lambda^k the
    previous iteration's multipliers (no Anderson step, consecutive iterations),
    s = P_[l_c,u_c](A x + lambda^k / sigma) on inequality rows, s = l_c on equality
    rows, r = A x - s and lambda^{k+1} = lambda^k + sigma r."""
    inst, tr, info, _ = outer
    S = _scaled(inst, info)
    mE = info["mE"]
    checked = 0
    for prev, t in zip(tr, tr[1:]):
        if t["k"] != prev["k"] + 1:
            continue
        lam0, sig = prev["lam"], t["sig"]
        ax = S["A"] @ t["x"]
        s = np.where(np.arange(ax.size) < mE, S["lc"], _proj(ax + lam0 / sig, S["lc"], S["uc"]))
        r = ax - s
        assert np.allclose(t["r"], r, rtol=1e-10, atol=1e-13)
        assert np.allclose(t["lam"], lam0 + sig * r, rtol=1e-10, atol=1e-13)
        checked += 1
    assert checked > 5


def test_outer_residuals_recomputed(outer, oracle):
    """Eqs. outer-residuals / outer-scales in the scaled space from the rebuilt scaled
    problem, and on the original data equal to the external test of Sec. 4.1."""
    inst, tr, info, _ = outer
    S = _scaled(inst, info)
    Dx, Dc, cs, perm = info["Dx"], info["Dc"], info["cs"], info["perm"]
    for t in tr[::5]:
        x, lam = t["x"], t["lam"]
        ax = S["A"] @ x
        rp = np.maximum(np.maximum(S["lc"] - ax, ax - S["uc"]), 0).max()
        sp_ = max(1.0, np.abs(ax).max(), np.abs(S["lc"]).max(), np.abs(S["uc"]).max())
        g = S["Q"] @ x + S["c"] + S["A"].T @ lam
        rd = np.abs(x - _proj(x - g, S["lx"], S["ux"])).max()
        sd = max(1.0, np.abs(S["Q"] @ x).max(), np.abs(S["c"]).max(), np.abs(S["A"].T @ lam).max())
        for got, want in ((t["sc_rp"], rp), (t["sc_sp"], sp_), (t["sc_rd"], rd), (t["sc_sd"], sd)):
            assert _rel(got, want) < 1e-10, (got, want)
        lam_o = np.zeros_like(lam)
        lam_o[perm] = Dc * lam / cs
        ref = oracle.kkt_check(inst, Dx * x, lam_o)
        for got, want in zip((t["un_rp"], t["un_rd"], t["un_sp"], t["un_sd"]), ref):
            assert _rel(got, want) < 1e-10, (got, want)


def _hand(c, lc, x0=None):
    """min 1/2 (x1^2 - x2^2) + c'x  s.t.  x1 + x2 = lc,  0 <= x <= 1 (no scaling)."""
    return dict(Q=sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]])), c=np.asarray(c, float),
                A=sp.csr_matrix(np.array([[1.0, 1.0]])), l_c=np.array([lc]), u_c=np.array([lc]),
                l_x=np.zeros(2), u_x=np.ones(2), x0=x0)


@pytest.mark.parametrize("c, lc, x0, want", [
    # x0 = 0: f = 0, A x0 - P(A x0) = -1.5: 20 * 1 / (2.25 / 2) = 17.77...
    ([1.0, 0.0], 1.5, None, 20.0 / 1.125),
    # x0 = (1, 1): f = 1, distance 0.5: 20 * 1 / max(1, 0.125) = 20
    ([1.0, 0.0], 1.5, [1.0, 1.0], 20.0),
    # x0 = (1, 0): f = 1/2 - 300 = -299.5, distance 0.5: 20 * 299.5 = 5990
    ([-300.0, 0.0], 1.5, [1.0, 0.0], 5990.0),
    # same with c1 = -1000: 20 * 999.5 is clamped to 1e4
    ([-1000.0, 0.0], 1.5, [1.0, 0.0], 1e4),
    # far from feasible: x0 = 0, lc = 1000 (distance 1000): 20 / 5e5 = 4e-5 is clamped to 1e-4
    ([1.0, 0.0], 1000.0, None, 1e-4),
])
def test_initial_penalty_hand_cases(oracle, c, lc, x0, want):
    """QPALM's initial penalty (reading A12 of Sec. 3.2.1's 'as in QPALM'):
    sigma0 = clamp(sigma_init max(1, |f(x0)|) / max(1, ||A x0 - P(A x0)||^2 / 2), 1e-4, 1e4),
    worked by hand on a 2-variable instance without scaling."""
    t = _hand(c, lc)
    info = oracle.setup_info(t, None if x0 is None else np.asarray(x0, float), no_scaling=1)
    assert _rel(info["sigma0"], want) < 1e-14, (info["sigma0"], want)
