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


def test_empty_and_oversized_inputs_are_rejected_without_a_gpu(lib):
    """Empty grids and batches, a batch with an empty problem, and a step
    beyond the allocation-free scratch are refused by the host checks,
    before any CUDA call and before the state pointer is used."""
    from paper_2102_05287_gb300 import wcns
    L = wcns.load()
    E = wcns.WCNS_E_INVALID_ARG
    g = wcns.wcns_grid()
    g.ndim = 2
    g.n[0], g.n[1] = 16, 0  # no cells along y
    g.lo[0], g.lo[1], g.hi[0], g.hi[1] = 0.0, 0.0, 1.0, 1.0
    b = wcns.wcns_bcs()
    h = ctypes.c_void_p()
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(h)) == E
    g.n[1] = 8
    g.hi[1] = 0.0  # empty extent
    assert L.wcns_create(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(h)) == E
    assert not h.value

    bh = ctypes.c_void_p()
    IA = ctypes.c_int * 3
    DA = ctypes.c_double * 3
    lo, hi = DA(0.0, 0.0, 0.0), DA(1.0, 1.0, 1.0)
    T, Pd = wcns.WCNS_BC_TRANSMISSIVE, wcns.WCNS_BC_PERIODIC
    assert L.wcns_batch_create(0, IA(4, 5, 6), lo, hi, T, T, 1.4, 4.4, 6e8, ctypes.byref(bh)) == E
    assert L.wcns_batch_create(3, IA(4, 0, 6), lo, hi, T, T, 1.4, 4.4, 6e8, ctypes.byref(bh)) == E
    assert L.wcns_batch_create(3, IA(4, 5, 6), lo, DA(1.0, 0.0, 1.0), T, T, 1.4, 4.4, 6e8,
                               ctypes.byref(bh)) == E
    assert L.wcns_batch_create(3, IA(4, 5, 6), lo, hi, Pd, T, 1.4, 4.4, 6e8, ctypes.byref(bh)) == E
    assert not bh.value

    # the allocation-free step: no scratch for a 2048 x 1024 grid
    # ((3 * 6 + 3) doubles a cell > 8M doubles), nor for a non-positive dt;
    # the state pointer is a placeholder the checks never dereference
    g.n[0], g.n[1] = 2048, 1024
    g.hi[1] = 1.0
    W = ctypes.c_void_p(256)
    assert L.wcns_rk3_step_noalloc(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, None, W,
                                   1e-7) == wcns.WCNS_E_TOO_LARGE
    g.n[0], g.n[1] = 16, 8
    assert L.wcns_rk3_step_noalloc(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, None, W, 0.0) == E
    assert L.wcns_rk3_step_noalloc(ctypes.byref(g), ctypes.byref(b), 1.4, 4.4, 6e8, None, None, 1e-7) == E


def test_grid_batch_and_division_check_host_rejections(lib):
    """wcns_batch_create_grids refuses empty or inconsistent problem tables,
    Dirichlet faces (not provided in batches), symmetry on a problem with
    fewer than 3 cells, and three dimensions (unsupported);
    wcns_check_division refuses a negative length or missing arrays;
    wcns_check_limiter_cert refuses bad dimensions, kinds, lengths, arrays,
    tolerances and EOS parameters.  All before any CUDA call."""
    from paper_2102_05287_gb300 import wcns
    L = wcns.load()
    E = wcns.WCNS_E_INVALID_ARG
    b = wcns.wcns_bcs()
    bh = ctypes.c_void_p()
    n = (ctypes.c_int * 4)(8, 6, 10, 12)
    lo = (ctypes.c_double * 4)(0.0, 0.0, 0.0, 0.0)
    hi = (ctypes.c_double * 4)(1.0, 1.0, 1.0, 1.0)

    def create(ndim, nprob, nn=n, lo_=lo, hi_=hi):
        return L.wcns_batch_create_grids(ndim, nprob, nn, lo_, hi_, ctypes.byref(b), 1.4, 4.4, 6e8, ctypes.byref(bh))
    assert create(2, 0) == E
    assert create(2, 2, nn=(ctypes.c_int * 4)(8, 0, 10, 12)) == E
    assert create(2, 2, hi_=(ctypes.c_double * 4)(1.0, 0.0, 1.0, 1.0)) == E
    assert create(3, 1, nn=(ctypes.c_int * 3)(4, 4, 4)) == wcns.WCNS_E_UNSUPPORTED
    b.kind[1][0] = wcns.WCNS_BC_DIRICHLET
    assert create(2, 2) == E
    b.kind[1][0] = wcns.WCNS_BC_PERIODIC  # periodic on one face only
    assert create(2, 2) == E
    b.kind[1][0] = b.kind[1][1] = wcns.WCNS_BC_SYMMETRY
    assert create(2, 2, nn=(ctypes.c_int * 4)(8, 2, 10, 12)) == E
    assert L.wcns_batch_create_grids(2, 2, n, lo, hi, None, 1.4, 4.4, 6e8, ctypes.byref(bh)) == E
    assert L.wcns_batch_create_grids(2, 2, n, lo, hi, ctypes.byref(b), 5.0, 4.4, 6e8, ctypes.byref(bh)) == E
    assert not bh.value
    assert L.wcns_check_division(None, None, None, -1, None) == E
    assert L.wcns_check_division(None, None, None, 4, None) == E
    assert L.wcns_check_division(None, None, None, 0, None) == wcns.WCNS_OK
    # wcns_check_limiter_cert: dimension, kind, length, arrays, tolerances, EOS
    cert = (ctypes.c_int * 1)()
    ok = (1e-10, 1e-10, 1e-8, 1.4, 4.4, 6e8)
    assert L.wcns_check_limiter_cert(0, 0, None, 0, *ok, None, None, None) == E
    assert L.wcns_check_limiter_cert(4, 0, None, 0, *ok, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 3, None, 0, *ok, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, -1, None, 0, *ok, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 2, None, 0, *ok, None, None, None) == wcns.WCNS_OK
    assert L.wcns_check_limiter_cert(2, 0, None, -1, *ok, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 1, None, 3, *ok, cert, cert, None) == E
    assert L.wcns_check_limiter_cert(2, 0, None, 0, -1e-10, *ok[1:], None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 0, None, 0, 1e-10, 1e-10, float("nan"), *ok[3:], None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 0, None, 0, *ok[:3], 5.0, 4.4, 6e8, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 0, None, 0, *ok[:3], 1.4, 4.4, -1.0, None, None, None) == E
    assert L.wcns_check_limiter_cert(2, 1, None, 0, *ok, None, None, None) == wcns.WCNS_OK


def test_plain_c_program_uses_the_boundary(lib, tmp_path):
    """The header is self-contained C99, and a C program linked against the
    library gets the documented answers from its host-side checks."""
    import subprocess
    from paper_2102_05287_gb300 import build
    from tests.conftest import build_abi_consumer
    exe = build_abi_consumer(build.LIB, tmp_path)
    r = subprocess.run([exe, "--checks"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr


def test_launch_grid_limits_are_refused_on_the_host(lib):
    """The documented launch-grid limits of wcns_create (gridDim.y and
    gridDim.z <= 65535: in 2D/3D n[0] <= 524,280 and n[1] <= 131,070, in 3D
    also n[1], n[2] <= 65,535) and the cell-count cap are refused before any
    allocation; sizes just inside pass the checks (and then fail only for
    want of a GPU here)."""
    from paper_2102_05287_gb300 import wcns
    L = wcns.load()
    E = wcns.WCNS_E_INVALID_ARG

    def create(*n):
        g = wcns.wcns_grid()
        g.ndim = len(n)
        for d, k in enumerate(n):
            g.n[d] = k
            g.lo[d], g.hi[d] = 0.0, 1.0
        h = ctypes.c_void_p()
        st = L.wcns_create(ctypes.byref(g), ctypes.byref(wcns.wcns_bcs()), 1.4, 4.4, 6e8, ctypes.byref(h))
        if h.value:  # created (a machine with a GPU)
            L.wcns_destroy(h)
        return st

    assert create(524281, 1) == E
    assert create(16, 131071) == E
    assert create(16, 65536, 2) == E
    assert create(16, 2, 65536) == E
    assert create(1 << 30 | 1) == E
    assert create(65535, 65535, 300) == E  # beyond 2^40 cells
    for ok in ((524280, 1), (16, 131070), (16, 65535, 65535)):
        assert create(*ok) != E, ok
