"""ctypes front end of the PDNQP oracle (pdnqp_oracle.c) -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain sequential FP64 C implementation of the paper's method
(Algorithm 3 driving Algorithm 4, Eqs. practical-multiplier-update ..
adaptive-condition).  Only the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path never
does.  It shares nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdnqp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SNAP_SCALARS = 8
CHK_COLS = 22
OTR_COLS = 25
STATUS = {0: "SOLVED", 1: "PRIMAL_INFEASIBLE", 2: "DUAL_INFEASIBLE", 3: "ITER_LIMIT", 4: "TIME_LIMIT",
          5: "NUMERICAL_ERROR"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int),
                ("q_rp", C.c_void_p), ("q_ci", C.c_void_p), ("q_v", C.c_void_p), ("c", C.c_void_p),
                ("a_rp", C.c_void_p), ("a_ci", C.c_void_p), ("a_v", C.c_void_p),
                ("lc", C.c_void_p), ("uc", C.c_void_p), ("lx", C.c_void_p), ("ux", C.c_void_p),
                ("x0", C.c_void_p), ("lam0", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("eps_abs", C.c_double), ("eps_rel", C.c_double), ("time_limit", C.c_double),
                ("k_out", C.c_longlong), ("k_in", C.c_longlong),
                ("sigma_init", C.c_double), ("theta_sigma", C.c_double), ("delta_gamma", C.c_double),
                ("rho_in_min", C.c_double), ("rho_in_max", C.c_double), ("rho_z", C.c_double),
                ("ruiz_outer", C.c_int), ("ruiz_inner", C.c_int), ("lanczos_steps", C.c_int),
                ("k_chk", C.c_int), ("beta_suff", C.c_double), ("beta_nec", C.c_double),
                ("beta_art", C.c_double), ("rej_limit", C.c_int), ("kappa_shrink", C.c_double),
                ("delta_sigma", C.c_double), ("sigma_max", C.c_double), ("tol_floor", C.c_double),
                ("gamma_override", C.c_double), ("no_scaling", C.c_int), ("verbose", C.c_int),
                ("eps_inf", C.c_double), ("anderson", C.c_int), ("anderson_mem", C.c_int)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_longlong), ("inner_iters", C.c_longlong),
                ("trials", C.c_longlong), ("restarts", C.c_longlong),
                ("r_p", C.c_double), ("r_d", C.c_double), ("s_p", C.c_double), ("s_d", C.c_double),
                ("rel_kkt", C.c_double), ("gamma", C.c_double), ("lambda_min", C.c_double),
                ("obj", C.c_double), ("seconds", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER
            L.or_default_params.argtypes = [dp(_Params)]
            L.or_solve.argtypes = [dp(_Problem), dp(_Params), C.c_void_p, C.c_void_p, dp(_Result)]
            L.or_debug_inner.argtypes = [dp(_Problem), dp(_Params), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_setup_info.argtypes = [dp(_Problem), dp(_Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_inner_qp_dense.argtypes = [dp(_Problem), dp(_Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_double] + [C.c_void_p] * 7
            L.or_inner_steps.argtypes = [dp(_Problem), dp(_Params)] + [C.c_void_p] * 4
            L.or_inner_solve_given.argtypes = [dp(_Problem), dp(_Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_double, C.c_double, C.c_longlong, C.c_void_p, C.c_void_p,
                                               C.c_void_p]
            L.or_kkt_check.argtypes = [dp(_Problem), C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_anderson_step.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_lanczos_min.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_uint64]
            L.or_lanczos_min.restype = C.c_double
            L.or_tridiag_min_eig.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
            L.or_tridiag_min_eig.restype = C.c_double
            L.or_ruiz_outer.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 6 + [C.c_int, C.c_void_p, C.c_void_p]
            L.or_project.argtypes = [C.c_int] + [C.c_void_p] * 4
            L.or_debug_inner_timed.argtypes = [dp(_Problem), dp(_Params), C.c_int] + [C.c_void_p] * 4
            L.or_debug_checks.argtypes = [dp(_Problem), dp(_Params), C.c_int, C.c_void_p, C.c_void_p]
            L.or_solve_traced.argtypes = [dp(_Problem), dp(_Params), C.c_void_p, C.c_void_p, dp(_Result), C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


class Problem:
    """Keeps the contiguous arrays alive while the C struct points at them."""

    def __init__(self, inst: dict, x0=None, lam0=None):
        Q, A = inst["Q"].tocsr(), inst["A"].tocsr()
        self.n, self.m = Q.shape[0], A.shape[0]
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.keep = [i32(Q.indptr), i32(Q.indices), f64(Q.data), f64(inst["c"]),
                     i32(A.indptr), i32(A.indices), f64(A.data),
                     f64(inst["l_c"]), f64(inst["u_c"]), f64(inst["l_x"]), f64(inst["u_x"]),
                     f64(x0) if x0 is not None else None, f64(lam0) if lam0 is not None else None]
        k = self.keep
        self.s = _Problem(self.n, self.m, *[_ptr(a) for a in k])

    def ref(self):
        return C.byref(self.s)


def default_params(**over) -> _Params:
    p = _Params()
    lib().or_default_params(C.byref(p))
    for key, v in over.items():
        if not hasattr(p, key):
            raise KeyError(key)
        setattr(p, key, v)
    return p


def solve(inst: dict, x0=None, lam0=None, **params):
    """Algorithm 3 + 4.  Returns (x, y, info) in the original coordinates."""
    P = Problem(inst, x0, lam0)
    params.setdefault("time_limit", 120.0)  # a test must never hang
    prm = default_params(**params)
    x = np.zeros(P.n)
    y = np.zeros(P.m)
    r = _Result()
    lib().or_solve(P.ref(), C.byref(prm), _ptr(x), _ptr(y), C.byref(r))
    info = {f[0]: getattr(r, f[0]) for f in _Result._fields_}
    info["status_name"] = STATUS.get(info["status"], "?")
    return x, y, info


def snapshot_len(n, m, mI):
    dw = n + mI + m
    return 2 * (dw + m) + SNAP_SCALARS, dw


def split_snapshot(v, dw, m):
    return dict(w=v[:dw], y=v[dw:dw + m], wbar=v[dw + m:2 * dw + m], ybar=v[2 * dw + m:2 * dw + 2 * m],
                omega=v[-8], kappa=v[-7], t=int(v[-6]), t_total=int(v[-5]), trials=int(v[-4]),
                restarts=int(v[-3]), kkt_restart=v[-2], kkt_last=v[-1])


def setup_info(inst: dict, x0=None, **params):
    P = Problem(inst, x0)
    prm = default_params(**params)
    Dc, Dx, perm = np.zeros(P.m), np.zeros(P.n), np.zeros(P.m, dtype=np.int32)
    sc = np.zeros(6)
    lib().or_setup_info(P.ref(), C.byref(prm), _ptr(Dc), _ptr(Dx), _ptr(perm), _ptr(sc))
    return dict(Dc=Dc, Dx=Dx, perm=perm, cs=sc[0], gamma=sc[1], lambda_min=sc[2], sigma0=sc[3],
                mE=int(sc[4]), qnorm=sc[5])


def debug_inner(inst: dict, checkpoints, x0=None, **params):
    """Snapshots of the first inner solve after the given accepted-iteration counts."""
    P = Problem(inst, x0)
    prm = default_params(**params)
    info = setup_info(inst, x0, **params)
    mI = P.m - info["mE"]
    L, dw = snapshot_len(P.n, P.m, mI)
    ck = np.ascontiguousarray(sorted(checkpoints), dtype=np.int64)
    out = np.zeros(L * len(ck))
    g = np.zeros(1)
    got = lib().or_debug_inner(P.ref(), C.byref(prm), len(ck), _ptr(ck), _ptr(out), _ptr(g))
    snaps = [split_snapshot(out[i * L:(i + 1) * L], dw, P.m) for i in range(max(got, 0))]
    return snaps, dict(info, gamma=g[0], dw=dw, mI=mI, status=got)


def inner_qp_dense(inst: dict, z, lam, sig, gamma, **params):
    P = Problem(inst)
    prm = default_params(**params)
    info = setup_info(inst, **params)
    mI = P.m - info["mE"]
    dw = P.n + mI + P.m
    H, B = np.zeros((dw, dw)), np.zeros((P.m, dw))
    q, h, lo, hi = np.zeros(dw), np.zeros(P.m), np.zeros(dw), np.zeros(dw)
    dims = np.zeros(5, dtype=np.int32)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    z, lam, sig = f64(z), f64(lam), f64(sig)
    lib().or_inner_qp_dense(P.ref(), C.byref(prm), _ptr(z), _ptr(lam), _ptr(sig), float(gamma),
                            _ptr(H), _ptr(q), _ptr(B), _ptr(h), _ptr(lo), _ptr(hi), _ptr(dims))
    return dict(H=H, q=q, B=B, h=h, lo=lo, hi=hi, n=int(dims[0]), m=int(dims[1]), mE=int(dims[2]),
                mI=int(dims[3]), dw=int(dims[4]), perm=info["perm"])


def inner_steps(inst: dict, x0=None, **params):
    P = Problem(inst, x0)
    prm = default_params(**params)
    info = setup_info(inst, x0, **params)
    mI = P.m - info["mE"]
    dw = P.n + mI + P.m
    mw, my, ew, dy = np.zeros(dw), np.zeros(P.m), np.zeros(dw), np.zeros(P.m)
    lib().or_inner_steps(P.ref(), C.byref(prm), _ptr(mw), _ptr(my), _ptr(ew), _ptr(dy))
    return dict(mw=mw, my=my, ew=ew, dy=dy, dw=dw, mI=mI, info=info)


def inner_solve_given(inst: dict, z, lam_int, sig_int, gamma, tol=1e-10, kin=400000, x=None, y=None, **params):
    P = Problem(inst)
    prm = default_params(**params)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).copy()
    x = f64(np.zeros(P.n) if x is None else x)
    y = f64(np.zeros(P.m) if y is None else y)
    it = np.zeros(1, dtype=np.int64)
    z, lam_int, sig_int = f64(z), f64(lam_int), f64(sig_int)  # keep alive across the call
    st = lib().or_inner_solve_given(P.ref(), C.byref(prm), _ptr(z), _ptr(lam_int), _ptr(sig_int),
                                    float(gamma), float(tol), int(kin), _ptr(x), _ptr(y), _ptr(it))
    return x, y, int(st), int(it[0])


def kkt_check(inst: dict, x, lam):
    """External KKT test of Sec. 4.1 on the original data: (r_p, r_d, s_p, s_d)."""
    P = Problem(inst)
    out = np.zeros(4)
    x = np.ascontiguousarray(x, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    lib().or_kkt_check(P.ref(), _ptr(x), _ptr(lam), _ptr(out))
    return tuple(out)


def kkt_pass(inst, x, lam, eps_abs, eps_rel):
    rp, rd, sp, sd = kkt_check(inst, x, lam)
    return rp <= eps_abs + eps_rel * sp and rd <= eps_abs + eps_rel * sd


def lanczos_min(Q, steps=64, seed=1):
    Q = Q.tocsr()
    rp = np.ascontiguousarray(Q.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(Q.indices, dtype=np.int32)
    v = np.ascontiguousarray(Q.data, dtype=np.float64)
    return lib().or_lanczos_min(Q.shape[0], _ptr(rp), _ptr(ci), _ptr(v), int(steps), int(seed))


def tridiag_min_eig(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(np.concatenate([b, [0.0]]), dtype=np.float64)
    return lib().or_tridiag_min_eig(_ptr(a), _ptr(b), a.size)


def ruiz_outer(A, sweeps=8, Q=None):
    A = A.tocsr().copy()
    if Q is not None:
        Q = Q.tocsr()
        qk = [np.ascontiguousarray(Q.indptr, dtype=np.int32), np.ascontiguousarray(Q.indices, dtype=np.int32),
              np.ascontiguousarray(Q.data, dtype=np.float64)]
    else:
        qk = [None, None, None]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    v = np.ascontiguousarray(A.data, dtype=np.float64).copy()
    Dc, Dx = np.zeros(A.shape[0]), np.zeros(A.shape[1])
    lib().or_ruiz_outer(A.shape[0], A.shape[1], _ptr(rp), _ptr(ci), _ptr(v), *[_ptr(a) for a in qk], int(sweeps),
                        _ptr(Dc), _ptr(Dx))
    A.data = v
    return A, Dc, Dx


def project(v, lo, hi):
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    v, lo, hi = f64(v), f64(lo), f64(hi)
    out = np.zeros_like(v)
    lib().or_project(v.size, _ptr(v), _ptr(lo), _ptr(hi), _ptr(out))
    return out


def debug_inner_timed(inst: dict, checkpoints, x0=None, **params):
    """Wall-clock seconds (from the first inner iteration) at each checkpoint, and the setup time."""
    P = Problem(inst, x0)
    prm = default_params(**params)
    info = setup_info(inst, x0, **params) if P.n <= 200_000 else None
    mE = info["mE"] if info else None
    ck = np.ascontiguousarray(sorted(checkpoints), dtype=np.int64)
    # snapshot buffer sized for the largest possible layout (dw <= n + 2m)
    L = 2 * (P.n + 3 * P.m) + SNAP_SCALARS
    out = np.zeros(L * len(ck))
    times = np.zeros(len(ck))
    setup = np.zeros(1)
    got = lib().or_debug_inner_timed(P.ref(), C.byref(prm), len(ck), _ptr(ck), _ptr(out), _ptr(times), _ptr(setup))
    del mE
    return times[:max(got, 0)], float(setup[0])


def anderson_step(U, G):
    """One Type-II Anderson step from stored pairs (rows of U, G, oldest first);
    returns the extrapolated point or None."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.zeros(U.shape[1])
    rc = lib().or_anderson_step(int(U.shape[0]), int(U.shape[1]), _ptr(U), _ptr(G), _ptr(out))
    return out if rc == 0 else None


def debug_checks(inst: dict, max_checks: int, x0=None, **params):
    """Trace of the periodic checks of the first inner solve (convergence ignored):
    per check a dict with the scalars of the restart decision and the vectors w, y,
    wbar, ybar, w_start, y_start (inner-unscaled) before it."""
    P = Problem(inst, x0)
    prm = default_params(**params)
    info = setup_info(inst, x0, **params)
    mI = P.m - info["mE"]
    dw = P.n + mI + P.m
    rows = np.zeros((max_checks, CHK_COLS))
    vecs = np.zeros((max_checks, 3 * (dw + P.m)))
    got = lib().or_debug_checks(P.ref(), C.byref(prm), int(max_checks), _ptr(rows), _ptr(vecs))
    names = ["t_total", "t", "k_cur", "k_avg", "k_restart", "k_last", "use_avg", "restart", "omega",
             "omega_after", "kappa", "kappa_after", "t_after", "k_restart_after", "rp_cur", "rd_cur", "sp_cur",
             "sd_cur", "rp_avg", "rd_avg", "sp_avg", "sd_avg"]
    out = []
    for r, v in zip(rows[:max(got, 0)], vecs[:max(got, 0)]):
        d = dict(zip(names, r))
        o = 0
        for key, ln in (("w", dw), ("y", P.m), ("wbar", dw), ("ybar", P.m), ("wst", dw), ("yst", P.m)):
            d[key] = v[o:o + ln]
            o += ln
        out.append(d)
    return out, dict(info, dw=dw, mI=mI, status=got)


def solve_traced(inst: dict, max_rows: int = 10000, x0=None, lam0=None, **params):
    """solve() plus a per-outer-iteration trace of the outer rules (scaled internal
    coordinates): list of dicts with the scalars and vectors of each iteration that
    reached the tolerance update."""
    P = Problem(inst, x0, lam0)
    params.setdefault("time_limit", 120.0)
    prm = default_params(**params)
    n, m = P.n, P.m
    x, y = np.zeros(n), np.zeros(m)
    r = _Result()
    rows = np.zeros((max_rows, OTR_COLS))
    vecs = np.zeros((max_rows, 3 * n + 5 * m))
    nr = C.c_int(0)
    lib().or_solve_traced(P.ref(), C.byref(prm), _ptr(x), _ptr(y), C.byref(r), int(max_rows), _ptr(rows),
                          _ptr(vecs), C.byref(nr))
    info = {f[0]: getattr(r, f[0]) for f in _Result._fields_}
    info["status_name"] = STATUS.get(info["status"], "?")
    names = ["k", "primal_ok", "r_inf", "dx_inf", "sc_rp", "sc_rd", "sc_sp", "sc_sd", "un_rp", "un_rd", "un_sp",
             "un_sd", "gamma", "ratio", "rho", "dta", "dtr", "dta_after", "dtr_after", "eak", "erk", "eak_after",
             "erk_after", "moved", "sd_in"]
    tr = []
    for row, v in zip(rows[:nr.value], vecs[:nr.value]):
        d = dict(zip(names, row))
        o = 0
        for key, ln in (("x", n), ("z", n), ("z_after", n), ("lam", m), ("sig", m), ("sig_after", m), ("r", m),
                        ("r_prev", m)):
            d[key] = v[o:o + ln]
            o += ln
        tr.append(d)
    return x, y, info, tr
