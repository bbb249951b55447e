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
