"""Brute-force active-set enumeration for tiny QPs (test helper, numpy only).

These routines are independent of both the oracle and the CUDA path: they
enumerate every active set of a tiny problem, solve the corresponding KKT
linear system with numpy, and keep the sign-consistent, feasible solutions.
"""
from __future__ import annotations

import itertools

import numpy as np


def inner_qp_minimizer(H, q, B, h, lo, hi, tol=1e-9):
    """Unique minimiser (w, y) of  min 1/2 w'Hw + q'w  s.t. Bw = h, lo <= w <= hi.

    y is the multiplier of Bw = h in the convention L = 1/2 w'Hw + q'w - y'(Bw - h)
    (Eq. base-inner-saddle).  Requires H positive definite on ker B.
    """
    dw, m = H.shape[0], B.shape[0]
    bounded = [i for i in range(dw) if np.isfinite(lo[i]) or np.isfinite(hi[i])]
    found = []
    for pat in itertools.product("LUF", repeat=len(bounded)):
        fixed = {}
        ok = True
        for i, p in zip(bounded, pat):
            if p == "L":
                if not np.isfinite(lo[i]):
                    ok = False
                    break
                fixed[i] = lo[i]
            elif p == "U":
                if not np.isfinite(hi[i]) or lo[i] == hi[i]:
                    ok = False
                    break
                fixed[i] = hi[i]
        if not ok:
            continue
        fx = sorted(fixed)
        fr = [i for i in range(dw) if i not in fixed]
        wx = np.array([fixed[i] for i in fx])
        Hff = H[np.ix_(fr, fr)]
        Bf = B[:, fr]
        rhs1 = -q[fr] - (H[np.ix_(fr, fx)] @ wx if fx else 0.0)
        rhs2 = h - (B[:, fx] @ wx if fx else 0.0)
        K = np.block([[Hff, -Bf.T], [Bf, np.zeros((m, m))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([rhs1, rhs2]))
        except np.linalg.LinAlgError:
            continue
        if np.linalg.norm(K @ sol - np.concatenate([rhs1, rhs2])) > 1e-8 * (1 + np.linalg.norm(sol)):
            continue
        w = np.zeros(dw)
        w[fr] = sol[:len(fr)]
        w[fx] = wx
        y = sol[len(fr):]
        if np.any(w[fr] < lo[fr] - tol) or np.any(w[fr] > hi[fr] + tol):
            continue
        g = H @ w + q - B.T @ y
        good = True
        for i in fx:
            if fixed[i] == lo[i] and g[i] < -tol:
                good = False
            if fixed[i] == hi[i] and lo[i] != hi[i] and g[i] > tol:
                good = False
        if good:
            found.append((w, y))
    if not found:
        raise RuntimeError("no KKT point found")
    w0 = found[0][0]
    for w, _ in found[1:]:
        assert np.allclose(w, w0, atol=1e-7), "strongly convex QP with two minimisers"
    return found[0]


def qp_kkt_points(Q, c, A, l_c, u_c, l_x, u_x, tol=1e-9):
    """All KKT points (x, lam) of  min c'x + 1/2 x'Qx  s.t. l_c <= Ax <= u_c, l_x <= x <= u_x.

    Stationarity 0 in Qx + c + A'lam + N(x) (Eq. kkt-stationarity); lam_j <= 0 on a row
    active at its lower side, >= 0 at its upper side, free on equality rows.
    """
    Q, A = np.asarray(Q, float), np.asarray(A, float)
    n, m = Q.shape[0], A.shape[0]
    eq = [j for j in range(m) if l_c[j] == u_c[j]]
    ineq = [j for j in range(m) if l_c[j] != u_c[j]]
    pts = []
    for xp in itertools.product("LUF", repeat=n):
        for rp in itertools.product("LUN", repeat=len(ineq)):
            fixed = {}
            ok = True
            for i, p in enumerate(xp):
                if p == "L":
                    if not np.isfinite(l_x[i]):
                        ok = False
                    fixed[i] = l_x[i]
                elif p == "U":
                    if not np.isfinite(u_x[i]):
                        ok = False
                    fixed[i] = u_x[i]
            act = list(eq)
            bval = {j: l_c[j] for j in eq}
            side = {j: "E" for j in eq}
            for j, p in zip(ineq, rp):
                if p == "L":
                    if not np.isfinite(l_c[j]):
                        ok = False
                    act.append(j); bval[j] = l_c[j]; side[j] = "L"
                elif p == "U":
                    if not np.isfinite(u_c[j]):
                        ok = False
                    act.append(j); bval[j] = u_c[j]; side[j] = "U"
            if not ok:
                continue
            fx = sorted(fixed)
            fr = [i for i in range(n) if i not in fixed]
            wx = np.array([fixed[i] for i in fx])
            Aa = A[act, :] if act else np.zeros((0, n))
            na = len(act)
            K = np.block([[Q[np.ix_(fr, fr)], Aa[:, fr].T], [Aa[:, fr], np.zeros((na, na))]])
            r1 = -c[fr] - (Q[np.ix_(fr, fx)] @ wx if fx else 0.0)
            r2 = np.array([bval[j] for j in act]) - (Aa[:, fx] @ wx if fx else 0.0)
            rhs = np.concatenate([r1, r2])
            if K.size == 0:
                sol = np.zeros(0)
            else:
                try:
                    sol = np.linalg.solve(K, rhs)
                except np.linalg.LinAlgError:
                    continue
                if np.linalg.norm(K @ sol - rhs) > 1e-8 * (1 + np.linalg.norm(sol)):
                    continue
            x = np.zeros(n)
            x[fr] = sol[:len(fr)]
            x[fx] = wx
            lam = np.zeros(m)
            lam[act] = sol[len(fr):]
            if np.any(x < l_x - tol) or np.any(x > u_x + tol):
                continue
            ax = A @ x
            if np.any(ax < l_c - tol) or np.any(ax > u_c + tol):
                continue
            good = True
            for j in act:
                if side[j] == "L" and lam[j] > tol:
                    good = False
                if side[j] == "U" and lam[j] < -tol:
                    good = False
            g = Q @ x + c + A.T @ lam
            for i in fx:
                if fixed[i] == l_x[i] and g[i] < -tol:
                    good = False
                if fixed[i] == u_x[i] and g[i] > tol:
                    good = False
            if good:
                pts.append((x, lam))
    return pts
