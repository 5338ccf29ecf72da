"""The C-ABI library builds, loads and exports every entry point that
include/casim.h declares.  CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

from paper_2203_02054_gb300 import build as casim_build
from paper_2203_02054_gb300 import casim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "casim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(casim_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(casim.LIB_PATH):
        casim_build.build()
    return ctypes.CDLL(casim.LIB_PATH)


def test_header_declares_the_binding_names():
    assert _declared() == sorted(casim.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_create_errors(lib):
    casim.load_library()
    p = casim.casim_default_params()
    assert p.precision == casim.CASIM_MIXED and p.max_pairs_per_vertex == 8
    p.precision = 7   # invalid: rejected on the host before any CUDA call
    with pytest.raises(casim.CasimError) as ei:
        casim.casim_create(p)
    assert ei.value.code == casim.CASIM_E_INVALID
    assert "precision" in casim.casim_last_error(None)


def test_checked_build_reports_itself_and_exports_the_same_symbols(lib):
    if not os.path.exists(casim.LIB_CHECKED_PATH):
        casim_build.build()
    chk = ctypes.CDLL(casim.LIB_CHECKED_PATH)
    for name in _declared():
        assert hasattr(chk, name), name
    chk.casim_build_checked.restype = ctypes.c_int
    lib.casim_build_checked.restype = ctypes.c_int
    assert chk.casim_build_checked() == 1
    assert lib.casim_build_checked() == 0


def test_plain_build_refuses_the_checked_builds_fault_injection(lib):
    casim.load_library()
    p = casim.casim_default_params()
    p.debug_flags = casim.CASIM_DEBUG_CORRUPT_INCIDENCE  # rejected on the host before any CUDA call
    with pytest.raises(casim.CasimError) as ei:
        casim.casim_create(p)
    assert ei.value.code == casim.CASIM_E_INVALID
    assert "debug_flags" in casim.casim_last_error(None)
