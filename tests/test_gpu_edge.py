"""Edge cases of the CUDA path against the FP64 oracle.

- the smallest grids each boundary kind allows: one cell (transmissive,
  where every ghost copies it), the three cells a symmetry wall mirrors, the
  six cells of a periodic axis, and axes of one cell in 2D and 3D (the
  sweep along such an axis must add exactly nothing);
- uniform states (free-stream preservation): every midpoint flux is the
  same, so the flux differences and the alpha1 div(u) term vanish exactly
  (Sec. 4 semi-discrete form);
- zero steps leave the state and the time untouched;
- a batch of one- to fifteen-cell Riemann problems;
- a plain C99 program (tests/abi_consumer.c) driving the C ABI directly.

FP64 bar: 1e-12 relative per field (with the oracle's 1-ulp spread as the
fallback where a limiter theta solve amplifies round-off); mixed bar: the
forward-Euler stage W + dt L within 1e-5 (L1) of the oracle's.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import Batch, Solver  # noqa: E402
from tests.test_gpu_mixed import dirichlet_states, stage_errors  # noqa: E402
from tests.test_gpu_parity import assert_parity, relerr  # noqa: E402

EOS = P.WORKLOAD_EOS
T, S, PD, D = "transmissive", "symmetry", "periodic", "dirichlet"

TINY = [
    ((1,), ((T, T),)),
    ((2,), ((T, T),)),
    ((3,), ((S, T),)),
    ((4,), ((D, T),)),
    ((6,), ((PD, PD),)),
    ((1, 9), ((T, T), (S, T))),
    ((9, 1), ((PD, PD), (T, T))),
    ((3, 6), ((S, S), (PD, PD))),
    ((1, 1, 5), ((T, T), (T, T), (T, D))),
    ((2, 3, 4), ((T, T), (S, S), (T, D))),
]


def unit_box(n):
    return (0.0,) * len(n), (1.0,) * len(n)


def cfl_dt(o, W, n, cfl=0.4):
    sm = o.max_wavespeed(W)
    return cfl / sum(sm[d] * n[d] for d in range(len(n)))


def tiny_pair(n, bcs, W, precision):
    lo, hi = unit_box(n)
    dl = dirichlet_states(W, bcs)
    o = Oracle(n, lo, hi, bcs, dirichlet=dl, **EOS)
    s = Solver(n, lo, hi, bcs, precision=precision, dirichlet=dl, **EOS)
    return o, s


@pytest.mark.parametrize("k", range(len(TINY)), ids=[str(c[0]) for c in TINY])
def test_tiny_grids_fp64(k):
    n, bcs = TINY[k]
    W = P.random_admissible(n, seed=50 + k)
    o, s = tiny_pair(n, bcs, W, "fp64")
    dt = cfl_dt(o, W, n)
    ref = o.rhs(W, dt)
    got = s.rhs(torch.from_numpy(W).cuda(), dt).cpu().numpy()
    assert_parity(got, ref, lambda X: o.rhs(X, dt), W)
    ref = o.rk3_step(W, dt)
    Wg = torch.from_numpy(W).cuda()
    s.rk3_step(Wg, dt)
    assert_parity(Wg.cpu().numpy(), ref, lambda X: o.rk3_step(X, dt), W)
    st = s.stats()
    assert st["inadmissible"] == 0 and st["nonfinite"] == 0, st
    s.close()


@pytest.mark.parametrize("k", range(len(TINY)), ids=[str(c[0]) for c in TINY])
def test_tiny_grids_mixed(k):
    n, bcs = TINY[k]
    W = P.random_admissible(n, seed=50 + k, jumps=False)
    o, s = tiny_pair(n, bcs, W, "mixed")
    dt = cfl_dt(o, W, n)
    ref = o.rhs(W, dt)
    got = s.rhs(torch.from_numpy(W).cuda(), dt).cpu().numpy()
    assert np.isfinite(got).all()
    l1, linf = stage_errors(W, dt, got, ref)
    assert l1.max() < 1e-5 and linf.max() < 1e-4, (l1, linf)
    st = s.stats()
    assert st["inadmissible"] == 0 and st["nonfinite"] == 0, st
    s.close()


def uniform_state(n, vel):
    shape = tuple(reversed(n))
    a1 = np.full(shape, 0.3)
    v = [np.full(shape, x) for x in vel[:len(n)]]
    return P.conservative(EOS, a1 * 1000.0, (1.0 - a1) * 1.2, v, np.full(shape, 2e6), a1)


UNIFORM = [
    ((300,), ((PD, PD),)),
    ((257,), ((T, D),)),
    ((70, 45), ((PD, PD), (T, T))),
    ((40, 36), ((D, T), (PD, PD))),
    ((14, 13, 15), ((T, T), (PD, PD), (D, T))),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", range(len(UNIFORM)), ids=[str(c[0]) for c in UNIFORM])
def test_uniform_state_rhs_vanishes(k, precision):
    """Free-stream preservation: on a uniform state (moving in every
    direction, Dirichlet faces holding the same state) every midpoint computes
    the same flux, so the oracle's RHS and the FP64 kernels' are exactly
    zero; the mixed kernels' deviations about node i are exactly zero too,
    checked here at 1e-14 of the state."""
    n, bcs = UNIFORM[k]
    W = uniform_state(n, (120.0, -35.0, 7.0))
    o, s = tiny_pair(n, bcs, W, precision)
    dt = cfl_dt(o, W, n)
    ref = o.rhs(W, dt)
    assert np.all(ref == 0.0)
    got = s.rhs(torch.from_numpy(W).cuda(), dt).cpu().numpy()
    if precision == "fp64":
        assert np.all(got == 0.0), np.abs(got).max(axis=tuple(range(1, len(n) + 1)))
    else:
        l1, linf = stage_errors(W, dt, got, ref)
        assert linf.max() <= 1e-14, linf
    # one fused step: the SSPRK3 combine alone rounds (3/4 W + 1/4 W)
    Wg = torch.from_numpy(W).cuda()
    s.rk3_step(Wg, dt)
    assert relerr(Wg.cpu().numpy(), W).max() <= 1e-14
    st = s.stats()
    assert st["interp_limited"] == 0 and st["flux_limited"] == 0 and st["inadmissible"] == 0, st
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_steps_leave_the_state_untouched(precision):
    n = (40, 36)
    bcs = ((T, T), (PD, PD))
    W = P.random_admissible(n, seed=61)
    lo, hi = unit_box(n)
    s = Solver(n, lo, hi, bcs, precision=precision, **EOS)
    Wg = torch.from_numpy(W).cuda()
    t = s.advance_steps(Wg, 0, cfl=0.5, t=0.25)
    assert t == 0.25
    assert np.array_equal(Wg.cpu().numpy(), W)
    s.close()
    rb = P.riemann_batch(nprob=5, seed=62, nmin=10, nmax=40)
    b = Batch(rb.sizes, np.zeros(5), np.ones(5), T, T, precision=precision, **rb.eos)
    Wb = torch.from_numpy(rb.W).cuda()
    tt = torch.full((5,), 0.5, dtype=torch.float64, device="cuda")
    b.advance(Wb, 0, cfl=0.5, t=tt)
    assert np.array_equal(Wb.cpu().numpy(), rb.W) and torch.all(tt == 0.5)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_tiny_problems(precision):
    """Problems of 1 to 15 cells in one batch: each evolves exactly as it
    does alone through the single-grid path, and (FP64) its first step is
    the oracle's SSPRK3 step with its own CFL dt.

    Both runs take their 8 steps in one call: a call starts from the wave
    speeds of its input state, while later steps reuse the maxima reduced
    in the previous step's combine (FP32 with a safety margin in the mixed
    path), so splitting the run changes dt at the ulp level, and where a
    limiter sits at its tolerance that can flip a theta branch (the
    discontinuity of Algorithms 1 and 4)."""
    rb = P.riemann_batch(nprob=20, seed=9, nmin=1, nmax=16)
    assert rb.sizes.min() == 1 and rb.sizes.max() <= 15
    nprob = len(rb.sizes)
    b = Batch(rb.sizes, np.zeros(nprob), np.ones(nprob), T, T, precision=precision, **rb.eos)
    W1 = torch.from_numpy(rb.W).cuda()
    b.advance(W1, 1, cfl=0.5, t=torch.zeros(nprob, dtype=torch.float64, device="cuda"))
    first = W1.cpu().numpy()
    Wb = torch.from_numpy(rb.W).cuda()
    t = torch.zeros(nprob, dtype=torch.float64, device="cuda")
    b.advance(Wb, 8, cfl=0.5, t=t)
    got, tt = Wb.cpu().numpy(), t.cpu().numpy()
    st = b.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    for k in range(nprob):
        sl = slice(int(rb.offsets[k]), int(rb.offsets[k + 1]))
        n = int(rb.sizes[k])
        W0 = np.ascontiguousarray(rb.W[:, sl])
        if precision == "fp64":
            o = Oracle((n,), (0.0,), (1.0,), ((T, T),), **rb.eos)
            dt = 0.5 / (o.max_wavespeed(W0)[0] * n)
            ref = o.rk3_step(W0, dt)
            assert_parity(first[:, sl], ref, lambda X: o.rk3_step(X, dt), W0)
        s = Solver((n,), (0.0,), (1.0,), ((T, T),), precision=precision, **rb.eos)
        W = torch.from_numpy(W0.copy()).cuda()
        t_single = s.advance_steps(W, 8, cfl=0.5)
        assert relerr(got[:, sl], W.cpu().numpy()).max() <= 1e-14, (k, n)
        assert abs(tt[k] - t_single) <= 1e-14 * t_single
        s.close()
    b.close()


def test_plain_c_program_advances_the_shock_tube(tmp_path):
    """tests/abi_consumer.c, a C99 program that sees only include/wcns.h,
    advances the Sec. 6 water-air shock tube (200 cells) 20 steps through
    wcns_advance_steps_host; its result is the Python binding's, bit for bit,
    and its first step is the oracle's."""
    import subprocess
    from paper_2102_05287_gb300 import build
    from tests.conftest import build_abi_consumer
    exe = build_abi_consumer(build.LIB, tmp_path)
    pr = P.water_air_shock_tube(200)
    assert pr.eos == {"gamma_g": 1.4, "gamma_l": 4.4, "pinf_l": 6e8}  # the program's fluids
    W0 = np.ascontiguousarray(pr.W)
    src, dst = tmp_path / "w0.bin", tmp_path / "w1.bin"
    W0.tofile(src)
    for nsteps in (1, 20):
        r = subprocess.run([exe, str(src), str(dst), str(nsteps), "0.5"], capture_output=True, text=True,
                           timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        words = r.stdout.split()
        t_c = float(words[1])
        assert int(words[5]) == 0 and int(words[7]) == 0, r.stdout  # nonfinite, inadmissible
        got = np.fromfile(dst).reshape(W0.shape)
        s = Solver((200,), (0.0,), (1.0,), ((T, T),), **pr.eos)
        Wh = torch.from_numpy(W0.copy())
        t_py = s.advance_steps_host(Wh, nsteps, cfl=0.5)
        s.close()
        assert np.array_equal(got, Wh.numpy()) and t_c == t_py
        if nsteps == 1:
            o = Oracle((200,), (0.0,), (1.0,), ((T, T),), **pr.eos)
            dt = 0.5 / (o.max_wavespeed(W0)[0] * 200)
            assert abs(t_c - dt) <= 1e-14 * dt
            assert_parity(got, o.rk3_step(W0, dt), lambda X: o.rk3_step(X, dt), W0)
