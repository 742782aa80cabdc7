"""The allocation-free SSPRK3 entry point, wcns_rk3_step_noalloc.

It exists for callers that must not call cudaMalloc: real-time loops in
which an allocation can synchronise the device and miss a deadline, host
applications that give a plugin a fixed device-memory budget, and code that
keeps no per-solver state.  Its scratch is a fixed device array inside the
library, shared by every call.  These tests call it through the C ABI twice
in a row and check each result against the ordinary handle-based
wcns_rk3_step, within the 1e-12 per-field relative tolerance of the FP64
parity tests, in 1D, 2D and 3D, with transmissive, symmetry and uniform
Dirichlet faces; the file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2102_05287_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300 import wcns  # noqa: E402

TOL = 1e-12


def relerr(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


def c_grid_bcs(pr):
    g = wcns.wcns_grid()
    g.ndim = pr.ndim
    for d in range(3):
        g.n[d] = pr.n[d] if d < pr.ndim else 1
        g.lo[d] = pr.lo[d] if d < pr.ndim else 0.0
        g.hi[d] = pr.hi[d] if d < pr.ndim else 1.0
    b = wcns.wcns_bcs()
    for d in range(pr.ndim):
        for s in range(2):
            b.kind[d][s] = wcns._BC[pr.bcs[d][s]]
            st = pr.extra.get("dirichlet_states", {}).get((d, s))
            if st is not None:
                for q, v in enumerate(st):
                    b.dirichlet[d][s][q] = float(v)
    return g, b


def shock_tube_dirichlet():
    """The 1D water-air shock tube (200 cells) with its right face a uniform
    Dirichlet state: the pre-shock air moving left into the tube at 50 m/s
    (its wave speed then enters dt, Sec. 3.3)."""
    pr = P.water_air_shock_tube(200)
    right = pr.W[:, -1].copy()
    rho = right[0] + right[1]
    right[2] = -50.0 * rho
    right[3] += 0.5 * rho * 50.0 ** 2
    pr.bcs = (("transmissive", "dirichlet"),)
    pr.extra["dirichlet_states"] = {(0, 1): right}
    return pr


def shock_bubble_dirichlet():
    """The 2D shock/bubble problem (96 x 48) with uniform Dirichlet states on
    the left face (its own post-shock state) and the top face (the ambient
    water)."""
    pr = P.shock_bubble_2d(96, 48, seed=5)
    pr.bcs = (("dirichlet", "transmissive"), ("symmetry", "dirichlet"))
    pr.extra["dirichlet_states"] = {(0, 0): pr.W[:, 0, 0].copy(), (1, 1): pr.W[:, -1, -1].copy()}
    return pr


PROBLEMS = {"shock_bubble_2d_96x48": lambda: P.shock_bubble_2d(96, 48, seed=5),
            "bubble_collapse_3d_24": lambda: P.bubble_collapse_3d(n=24),
            "shock_tube_1d_200": lambda: P.water_air_shock_tube(200),
            "shock_tube_1d_200_dirichlet": shock_tube_dirichlet,
            "shock_bubble_2d_96x48_dirichlet": shock_bubble_dirichlet}


def dirichlet_arg(pr):
    """The Solver's `dirichlet` argument for the problem's uniform states."""
    st = pr.extra.get("dirichlet_states")
    if not st:
        return None
    return [[st.get((d, s)) for s in range(2)] for d in range(pr.ndim)]


@pytest.mark.parametrize("problem", sorted(PROBLEMS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_step_matches_handle_step_twice(precision, problem):
    lib = wcns.load()
    pr = PROBLEMS[problem]()
    stream = torch.cuda.current_stream()
    ref = wcns.Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, stream=stream, dirichlet=dirichlet_arg(pr),
                      **pr.eos)
    g, b = c_grid_bcs(pr)
    o = wcns.wcns_default_options()
    o.precision = wcns._PREC[precision]
    o.stream = C.c_void_p(stream.cuda_stream)
    W_ref = torch.from_numpy(pr.W).cuda()
    W_na = torch.from_numpy(pr.W).cuda()
    sm = ref.max_wavespeed(W_ref)
    dt = 0.4 / sum(sm[d] * pr.n[d] / (pr.hi[d] - pr.lo[d]) for d in range(pr.ndim))
    for call in range(2):
        ref.rk3_step(W_ref, dt)
        st = lib.wcns_rk3_step_noalloc(C.byref(g), C.byref(b), pr.eos["gamma_g"], pr.eos["gamma_l"],
                                       pr.eos["pinf_l"], C.byref(o), C.c_void_p(W_na.data_ptr()), dt)
        assert st == wcns.WCNS_OK, lib.wcns_strerror(st)
        torch.cuda.synchronize()
        err = relerr(W_na.cpu().numpy(), W_ref.cpu().numpy())
        assert np.all(err < TOL), (call, err)
    ref.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = wcns.load()
    g = wcns.wcns_grid()
    g.ndim = 2
    g.n[0], g.n[1] = 2048, 1024  # (3 * 6 + 3) * 2M doubles > 8M
    g.lo[0], g.lo[1], g.hi[0], g.hi[1] = 0.0, 0.0, 2.0, 1.0
    b = wcns.wcns_bcs()
    W = torch.zeros(6, 1024, 2048, dtype=torch.float64, device="cuda")
    st = lib.wcns_rk3_step_noalloc(C.byref(g), C.byref(b), 1.4, 4.4, 6e8, None, C.c_void_p(W.data_ptr()), 1e-7)
    assert st == wcns.WCNS_E_TOO_LARGE
    assert "too large" in lib.wcns_strerror(st).decode()
    # just above the 2D limit of 399,457 cells (21 doubles a cell)
    g.n[0], g.n[1] = 800, 500
    st = lib.wcns_rk3_step_noalloc(C.byref(g), C.byref(b), 1.4, 4.4, 6e8, None, C.c_void_p(W.data_ptr()), 1e-7)
    assert st == wcns.WCNS_E_TOO_LARGE
