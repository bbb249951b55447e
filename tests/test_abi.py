"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/pdnqp.h declares (no GPU needed, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pdnqp.h")).read()
    return sorted(set(re.findall(r"PDNQP_API\s+[\w\s\*]*?\b(pdnqp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2609_19557_gb300 import build as B
    return B.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("pdnqp_create", "pdnqp_solve", "pdnqp_get", "pdnqp_destroy", "pdnqp_set_param", "pdnqp_last_error",
                 "pdnqp_debug_inner"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header(lib_path):
    from paper_2609_19557_gb300 import pdnqp as P
    assert sorted(P.EXPORTED) == _declared()
    P.load(lib_path)


def test_library_has_no_cpu_fallback_symbols(lib_path):
    # The library carries no solver path other than its CUDA kernels: it links
    # nothing from the oracle.
    lib = ctypes.CDLL(lib_path)
    for name in ("or_solve", "or_debug_inner", "or_kkt_check"):
        assert not hasattr(lib, name)


def test_last_error_without_handle(lib_path):
    from paper_2609_19557_gb300 import pdnqp as P
    P.load(lib_path)
    assert isinstance(P.pdnqp_last_error(None), str)


def test_host_side_argument_checks(lib_path):
    """Calls rejected before any device work (no GPU needed): an empty batch,
    a batch with a NULL or repeated handle, an unknown self-test kind."""
    from paper_2609_19557_gb300 import pdnqp as P
    P.load(lib_path)
    L = P.load()
    st = (ctypes.c_int * 2)()
    assert L.pdnqp_solve_batch(None, 0, 1e-4, 1e-4, 0, None) == 0
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.pdnqp_solve_batch(arr, 2, 1e-4, 1e-4, 0, st) == -1
    assert L.pdnqp_solve_batch(arr, 2, -1.0, 1e-4, 0, st) == -1
    g, t = ctypes.c_int(0), ctypes.c_double(0.0)
    assert L.pdnqp_selftest_wait(7, ctypes.byref(g), ctypes.byref(t)) == -1
    assert L.pdnqp_selftest_wait(0, None, None) == -1
