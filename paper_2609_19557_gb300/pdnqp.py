"""Thin ctypes binding of libpdnqp.so (include/pdnqp.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no fallback: if the shared library is missing or no
GPU is usable, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdnqp.so")

PDNQP_SOLVED, PDNQP_PRIMAL_INFEASIBLE, PDNQP_DUAL_INFEASIBLE = 0, 1, 2
PDNQP_ITER_LIMIT, PDNQP_TIME_LIMIT, PDNQP_NUMERICAL_ERROR = 3, 4, 5
PDNQP_FP64, PDNQP_FP32_BULK = 64, 32
STATUS_NAMES = {0: "SOLVED", 1: "PRIMAL_INFEASIBLE", 2: "DUAL_INFEASIBLE", 3: "ITER_LIMIT", 4: "TIME_LIMIT",
                5: "NUMERICAL_ERROR"}
SNAP_SCALARS = 8

# Every function declared in include/pdnqp.h.
EXPORTED = ["pdnqp_create", "pdnqp_create_ex", "pdnqp_destroy", "pdnqp_solve", "pdnqp_get", "pdnqp_set_start",
            "pdnqp_set_param", "pdnqp_get_param", "pdnqp_dims", "pdnqp_last_error", "pdnqp_debug_inner",
            "pdnqp_replay_kernel", "pdnqp_kernel_bytes", "pdnqp_kkt_residuals", "pdnqp_kkt_last_error",
            "pdnqp_kkt_residuals_noalloc", "pdnqp_replay_last_ms", "pdnqp_mlp_param_count", "pdnqp_mlp_forward",
            "pdnqp_mlp_wmse", "pdnqp_mlp_backward", "pdnqp_mlp_adam", "pdnqp_mlp_to_bf16", "pdnqp_mlp_last_error",
            "pdnqp_set_controller", "pdnqp_get_trace", "pdnqp_solve_batch",
            "pdnqp_selftest_wait"]


class pdnqp_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class pdnqp_residuals(C.Structure):
    _fields_ = [("r_p", C.c_double), ("r_d", C.c_double), ("s_p", C.c_double), ("s_d", C.c_double),
                ("rel_kkt", C.c_double), ("outer_iters", C.c_int64), ("inner_iters", C.c_int64),
                ("trials", C.c_int64), ("restarts", C.c_int64), ("kkt_passes", C.c_int64),
                ("solve_seconds", C.c_double), ("gamma", C.c_double), ("lambda_min", C.c_double),
                ("obj", C.c_double), ("kernel_launches", C.c_int64),
                ("inner_seconds", C.c_double), ("setup_seconds", C.c_double),
                ("loop_seconds", C.c_double), ("loop_trials", C.c_int64), ("loop_blocks", C.c_int64),
                ("loop_launches", C.c_int64),
                ("loop_phase_seconds", C.c_double * 6), ("ctrl_used", C.c_int64), ("ctrl_fallbacks", C.c_int64)]


class pdnqp_device_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class pdnqp_device_problem(C.Structure):
    _fields_ = [("Q", pdnqp_device_csr), ("A", pdnqp_device_csr), ("At", pdnqp_device_csr),
                ("c", C.c_void_p), ("l_c", C.c_void_p), ("u_c", C.c_void_p), ("l_x", C.c_void_p),
                ("u_x", C.c_void_p)]


class pdnqp_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p)]


class PdnqpError(RuntimeError):
    pass


_lib = None


def load(path: str | None = None):
    """Load libpdnqp.so (build it first with paper_2609_19557_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise PdnqpError(f"{p} not found: build the CUDA library first (python -m paper_2609_19557_gb300.build)")
    L = C.CDLL(p)
    vp, ip = C.c_void_p, C.c_int
    L.pdnqp_create.argtypes = [C.POINTER(vp), C.POINTER(pdnqp_csr), vp, C.POINTER(pdnqp_csr), vp, vp, vp, vp]
    L.pdnqp_create_ex.argtypes = L.pdnqp_create.argtypes + [C.POINTER(pdnqp_options)]
    L.pdnqp_destroy.argtypes = [vp]
    L.pdnqp_destroy.restype = None
    L.pdnqp_solve.argtypes = [vp, C.c_double, C.c_double]
    L.pdnqp_selftest_wait.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.pdnqp_solve_batch.argtypes = [C.POINTER(vp), C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.pdnqp_get.argtypes = [vp, vp, vp, C.POINTER(pdnqp_residuals)]
    L.pdnqp_set_start.argtypes = [vp, vp, vp]
    L.pdnqp_set_param.argtypes = [vp, C.c_char_p, C.c_double]
    L.pdnqp_get_param.argtypes = [vp, C.c_char_p, C.POINTER(C.c_double)]
    L.pdnqp_dims.argtypes = [vp, vp]
    L.pdnqp_last_error.argtypes = [vp]
    L.pdnqp_last_error.restype = C.c_char_p
    L.pdnqp_debug_inner.argtypes = [vp, ip, vp, vp]
    L.pdnqp_replay_kernel.argtypes = [vp, ip, ip]
    L.pdnqp_replay_last_ms.argtypes = [vp]
    L.pdnqp_replay_last_ms.restype = C.c_double
    L.pdnqp_kernel_bytes.argtypes = [vp, ip, C.POINTER(C.c_double)]
    L.pdnqp_kkt_residuals.argtypes = [C.POINTER(pdnqp_device_problem), vp, vp, vp, vp]
    L.pdnqp_kkt_residuals_noalloc.argtypes = [C.POINTER(pdnqp_device_problem), vp, vp, vp, vp]
    L.pdnqp_kkt_last_error.argtypes = []
    L.pdnqp_kkt_last_error.restype = C.c_char_p
    L.pdnqp_mlp_param_count.argtypes = []
    L.pdnqp_mlp_forward.argtypes = [vp, vp, ip, vp, vp, vp]
    L.pdnqp_mlp_wmse.argtypes = [vp, vp, vp, ip, vp, vp, vp]
    L.pdnqp_mlp_backward.argtypes = [vp, vp, vp, vp, ip, vp, vp, vp]
    fl = C.c_float
    L.pdnqp_mlp_adam.argtypes = [vp, vp, vp, vp, vp, ip, fl, fl, fl, fl, vp]
    L.pdnqp_mlp_to_bf16.argtypes = [vp, vp, ip, vp]
    L.pdnqp_mlp_last_error.argtypes = []
    L.pdnqp_mlp_last_error.restype = C.c_char_p
    L.pdnqp_set_controller.argtypes = [vp, vp, ip]
    L.pdnqp_get_trace.argtypes = [vp, vp, C.c_int64, vp]
    for name in EXPORTED:
        if not hasattr(L, name):
            raise PdnqpError(f"{p} does not export {name}")
    _lib = L
    return L


def _csr(M, keep):
    M = M.tocsr()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    v = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [rp, ci, v]
    return pdnqp_csr(M.shape[0], M.shape[1], int(v.size), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)


def _f64(a, keep):
    a = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data


def _check(h, rc):
    if rc < 0:
        msg = load().pdnqp_last_error(h)
        raise PdnqpError(f"pdnqp error {rc}: {msg.decode() if msg else ''}")
    return rc


class Handle:
    """Owns one pdnqp_t (destroyed on close / garbage collection)."""

    def __init__(self, ptr, n, m):
        self.ptr, self.n, self.m = ptr, n, m

    def close(self):
        if self.ptr:
            load().pdnqp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pdnqp_create(Q, c, A, l_c, u_c, l_x, u_x, precision: int = PDNQP_FP64, device: int = -1, stream=None) -> Handle:
    """Q, A: scipy.sparse matrices (Q symmetric, both triangles); vectors: array-likes."""
    L = load()
    keep = []
    q = _csr(Q, keep)
    a = _csr(A, keep) if A is not None and A.shape[0] > 0 else None
    opt = pdnqp_options(int(precision), int(device), C.c_void_p(int(stream)) if stream else None)
    h = C.c_void_p()
    m = A.shape[0] if A is not None else 0
    rc = L.pdnqp_create_ex(C.byref(h), C.byref(q), _f64(c, keep), C.byref(a) if a is not None else None,
                           _f64(l_c, keep) if m else None, _f64(u_c, keep) if m else None, _f64(l_x, keep),
                           _f64(u_x, keep), C.byref(opt))
    _check(None, rc)
    return Handle(h.value, Q.shape[0], m)


def pdnqp_destroy(h: Handle):
    h.close()


def pdnqp_solve(h: Handle, eps_abs: float, eps_rel: float) -> int:
    return _check(h.ptr, load().pdnqp_solve(h.ptr, float(eps_abs), float(eps_rel)))


def pdnqp_solve_batch(handles, eps_abs: float, eps_rel: float, threads: int = 0) -> list:
    """Solves the problems of `handles` concurrently (pdnqp_solve_batch); returns their statuses."""
    k = len(handles)
    arr = (C.c_void_p * max(k, 1))(*[h.ptr for h in handles])
    st = (C.c_int * max(k, 1))()
    _check(None, load().pdnqp_solve_batch(arr, k, float(eps_abs), float(eps_rel), int(threads), st))
    return list(st)[:k]


def pdnqp_selftest_wait(kind: int):
    """Runs one bounded device wait out on purpose (see include/pdnqp.h); returns (gave_up, seconds)."""
    g = C.c_int(-1)
    t = C.c_double(0.0)
    _check(None, load().pdnqp_selftest_wait(int(kind), C.byref(g), C.byref(t)))
    return g.value == 1, t.value


def pdnqp_get(h: Handle):
    """Returns (x, y, residuals-dict)."""
    x = np.zeros(h.n)
    y = np.zeros(h.m)
    r = pdnqp_residuals()
    _check(h.ptr, load().pdnqp_get(h.ptr, x.ctypes.data, y.ctypes.data if h.m else None, C.byref(r)))
    out = {f[0]: getattr(r, f[0]) for f in pdnqp_residuals._fields_}
    out["loop_phase_seconds"] = list(out["loop_phase_seconds"])
    return x, y, out


def pdnqp_set_start(h: Handle, x0=None, y0=None):
    keep = []
    _check(h.ptr, load().pdnqp_set_start(h.ptr, _f64(x0, keep) if x0 is not None else None,
                                         _f64(y0, keep) if y0 is not None else None))


def pdnqp_set_param(h: Handle, name: str, value: float):
    _check(h.ptr, load().pdnqp_set_param(h.ptr, name.encode(), float(value)))


def pdnqp_get_param(h: Handle, name: str) -> float:
    v = C.c_double()
    _check(h.ptr, load().pdnqp_get_param(h.ptr, name.encode(), C.byref(v)))
    return v.value


def pdnqp_dims(h: Handle):
    out = np.zeros(5, dtype=np.int64)
    _check(h.ptr, load().pdnqp_dims(h.ptr, out.ctypes.data))
    return dict(n=int(out[0]), m=int(out[1]), mE=int(out[2]), mI=int(out[3]), nnz_q=int(out[4]))


def pdnqp_last_error(h: Handle | None = None) -> str:
    s = load().pdnqp_last_error(h.ptr if h else None)
    return s.decode() if s else ""


def pdnqp_debug_inner(h: Handle, checkpoints):
    """Snapshots of the first inner solve (see include/pdnqp.h) as dicts."""
    d = pdnqp_dims(h)
    n, m, mI = d["n"], d["m"], d["mI"]
    dw = n + mI + m
    L = 2 * (dw + m) + SNAP_SCALARS
    ck = np.ascontiguousarray(checkpoints, dtype=np.int64)
    out = np.zeros(L * ck.size)
    got = _check(h.ptr, load().pdnqp_debug_inner(h.ptr, int(ck.size), ck.ctypes.data, out.ctypes.data))
    snaps = []
    for i in range(got):
        v = out[i * L:(i + 1) * L]
        snaps.append(dict(w=v[:dw], y=v[dw:dw + m], wbar=v[dw + m:2 * dw + m], ybar=v[2 * dw + m:2 * dw + 2 * m],
                          omega=v[-8], kappa=v[-7], t=int(v[-6]), t_total=int(v[-5]), trials=int(v[-4]),
                          restarts=int(v[-3]), kkt_restart=v[-2], kkt_last=v[-1]))
    return snaps


def pdnqp_replay_kernel(h: Handle, which: int, reps: int):
    _check(h.ptr, load().pdnqp_replay_kernel(h.ptr, int(which), int(reps)))


def pdnqp_replay_last_ms(h: Handle) -> float:
    return load().pdnqp_replay_last_ms(h.ptr)


def pdnqp_kernel_bytes(h: Handle, which: int) -> float:
    v = C.c_double()
    _check(h.ptr, load().pdnqp_kernel_bytes(h.ptr, int(which), C.byref(v)))
    return v.value


def create_from_instance(inst: dict, precision: int = PDNQP_FP64, stream=None) -> Handle:
    """Convenience: handle for an instance dict as produced by instances.py."""
    return pdnqp_create(inst["Q"], inst["c"], inst["A"], inst["l_c"], inst["u_c"], inst["l_x"], inst["u_x"],
                        precision=precision, stream=stream)


class DeviceProblem:
    """Eq. qp copied to the current CUDA device with torch (device memory only);
    keeps the tensors alive while the C struct points at them."""

    def __init__(self, inst: dict):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        Q, A = inst["Q"].tocsr(), inst["A"].tocsr()
        At = A.T.tocsr()
        i32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device=dev)
        f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
        self.t = {}

        def csr(M, name):
            rp, ci, v = i32(M.indptr), i32(M.indices), f64(M.data)
            self.t[name] = (rp, ci, v)
            return pdnqp_device_csr(M.shape[0], M.shape[1], int(M.nnz), rp.data_ptr(), ci.data_ptr(), v.data_ptr())

        vec = {k: f64(inst[k]) for k in ("c", "l_c", "u_c", "l_x", "u_x")}
        self.t.update(vec)
        self.s = pdnqp_device_problem(csr(Q, "Q"), csr(A, "A"), csr(At, "At"), vec["c"].data_ptr(),
                                      vec["l_c"].data_ptr(), vec["u_c"].data_ptr(), vec["l_x"].data_ptr(),
                                      vec["u_x"].data_ptr())
        self.n, self.m = Q.shape[0], A.shape[0]


def pdnqp_kkt_residuals(prob: DeviceProblem, x, y, out, stream=None):
    """x, y, out: torch float64 CUDA tensors (out has 4 entries)."""
    rc = load().pdnqp_kkt_residuals(C.byref(prob.s), x.data_ptr(), y.data_ptr() if prob.m else None, out.data_ptr(),
                                    C.c_void_p(int(stream)) if stream else None)
    if rc < 0:
        raise PdnqpError(f"pdnqp_kkt_residuals error {rc}: {load().pdnqp_kkt_last_error().decode()}")


def pdnqp_kkt_residuals_noalloc(prob: DeviceProblem, x, y, out, stream=None):
    """Allocation-free variant (static device scratch); asynchronous on `stream`."""
    rc = load().pdnqp_kkt_residuals_noalloc(C.byref(prob.s), x.data_ptr(), y.data_ptr() if prob.m else None,
                                            out.data_ptr(), C.c_void_p(int(stream)) if stream else None)
    if rc < 0:
        raise PdnqpError(f"pdnqp_kkt_residuals_noalloc error {rc}: {load().pdnqp_kkt_last_error().decode()}")


# ---------------------------------------------------------------- controller MLP
# Thin wrappers over the pdnqp_mlp_* entry points; arguments are torch CUDA
# tensors (contiguous), the work goes on the current torch stream.
def _mlp_check(rc):
    if rc != 0:
        raise PdnqpError(f"pdnqp_mlp error {rc}: {load().pdnqp_mlp_last_error().decode()}")


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def mlp_param_count() -> int:
    return int(load().pdnqp_mlp_param_count())


def mlp_forward(w_bf16, x, y, cache=None):
    _mlp_check(load().pdnqp_mlp_forward(_dptr(w_bf16), _dptr(x), int(x.shape[0]), _dptr(y), _dptr(cache), _stream()))


def mlp_wmse(y, target, weight, dy, loss=None):
    _mlp_check(load().pdnqp_mlp_wmse(_dptr(y), _dptr(target), _dptr(weight), int(y.shape[0]), _dptr(dy),
                                     _dptr(loss), _stream()))


def mlp_backward(w_bf16, x, cache, dy, grad, scratch):
    _mlp_check(load().pdnqp_mlp_backward(_dptr(w_bf16), _dptr(x), _dptr(cache), _dptr(dy), int(x.shape[0]),
                                         _dptr(grad), _dptr(scratch), _stream()))


def mlp_adam(w, w_bf16, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _mlp_check(load().pdnqp_mlp_adam(_dptr(w), _dptr(w_bf16), _dptr(grad), _dptr(m), _dptr(v), int(step),
                                     float(lr), float(beta1), float(beta2), float(eps), _stream()))


def mlp_to_bf16(w, w_bf16):
    _mlp_check(load().pdnqp_mlp_to_bf16(_dptr(w), _dptr(w_bf16), int(w.numel()), _stream()))


TRACE_COLS = 24


def pdnqp_set_controller(h: Handle, weights=None):
    """Installs (FP32 host array of mlp_param_count() values) or removes (None)
    the learned controller's weights."""
    if weights is None:
        _check(h.ptr, load().pdnqp_set_controller(h.ptr, None, 0))
        return
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(h.ptr, load().pdnqp_set_controller(h.ptr, w.ctypes.data, int(w.size)))


def pdnqp_get_trace(h: Handle) -> np.ndarray:
    """Per-outer-iteration trace of the last solve, shape (rows, TRACE_COLS)."""
    n = C.c_int64(0)
    _check(h.ptr, load().pdnqp_get_trace(h.ptr, None, 0, C.byref(n)))
    out = np.zeros((n.value, TRACE_COLS))
    if n.value:
        _check(h.ptr, load().pdnqp_get_trace(h.ptr, out.ctypes.data, n.value, C.byref(n)))
    return out
