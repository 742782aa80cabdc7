"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/wcns.h declares.  No GPU is needed (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "wcns.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(wcns_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2102_05287_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wcns_create", "wcns_rhs", "wcns_rk3_step", "wcns_advance_to", "wcns_max_wavespeed"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2102_05287_gb300 import wcns
    assert sorted(wcns.EXPORTS) == declared_functions()


def test_host_side_validation_needs_no_gpu(lib):
    """Argument checks run before any CUDA call."""
    from paper_2102_05287_gb300 import wcns
    L = wcns.load()
    g = wcns.wcns_grid()
    g.ndim = 1
    g.n[0] = 10
    g.lo[0], g.hi[0] = 0.0, 1.0
    b = wcns.wcns_bcs()
    h = ctypes.c_void_p()
    # gamma_g > gamma_l breaks Lemma 1 (convexity of the admissible set)
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 4.4, 1.4, 6e8, ctypes.byref(h)) == wcns.WCNS_E_INVALID_ARG
    # one periodic face only
    b.kind[0][0] = wcns.WCNS_BC_PERIODIC
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(h)) == wcns.WCNS_E_INVALID_ARG
    b.kind[0][0] = wcns.WCNS_BC_SYMMETRY
    g.n[0] = 2
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(h)) == wcns.WCNS_E_INVALID_ARG
    g.n[0] = 10
    g.ndim = 4
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(h)) == wcns.WCNS_E_INVALID_ARG
    assert L.wcns_rhs(None, None, None, 1.0) == wcns.WCNS_E_INVALID_ARG
    assert L.wcns_strerror(wcns.WCNS_E_INVALID_ARG).decode() == "invalid argument"
