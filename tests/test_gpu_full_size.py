"""Parity at the workloads' full sizes, through the calls the benchmark times.

- 2D shock / air bubble, 1024x512: one SSPRK3 step through
  wcns_advance_steps (the captured step graph, CFL 0.5, device-side dt)
  against the oracle's step on the whole grid, FP64 and mixed.
- 2D shock / air bubble, 2048x1024: whole-grid RHS, FP64 and mixed.
- 3D bubble collapse, 384^3: whole-grid RHS on the GPU; sampled 12^3 boxes
  (the interface, a domain corner) recomputed by the oracle on the box plus
  a three-cell halo, with sigma_d set from the whole grid's maxima of
  |u_d| + c (Section 3.3), since each cell's RHS reads three nodes either
  side along each direction.

An RHS L is compared through the forward-Euler stage W + dt L it feeds (the
first SSPRK3 stage), in the units of the state: on these initial states some
components of the exact RHS vanish (the transverse momentum of a planar
shock, the volume fraction of a bubble at rest), so both sides carry only
round-off there and a scale taken from the RHS itself would be meaningless.
- 4096 Riemann problems: one batched step; sampled problems (the smallest,
  the largest and a seeded few) against the oracle's step with each
  problem's own CFL dt.

FP64 bar: 1e-12 relative per field (or 4x the oracle's own 1-ulp spread).
Mixed bar: relative L1 error per field below 1e-5.  Momentum components are
measured against the momentum vector's magnitude.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import Batch, Solver  # noqa: E402
from tests.test_gpu_parity import assert_parity, relerr, scales  # noqa: E402

MIXED_L1 = 1e-5


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.abs(a - b).sum(axis=1) / scales(b, l1=True)


@pytest.fixture(scope="module")
def bubble_1024():
    return P.shock_bubble_2d(1024, 512)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shock_bubble_1024x512_step(bubble_1024, precision):
    pr = bubble_1024
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, **pr.eos)
    Wg = torch.from_numpy(pr.W).cuda()
    dt = s.advance_steps(Wg, 1, cfl=0.5)
    got = Wg.cpu().numpy()
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    sm = o.max_wavespeed(pr.W)
    dt_ref = 0.5 / (sm[0] / (2.0 / pr.n[0]) + sm[1] / (1.0 / pr.n[1]))
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref
    ref = o.rk3_step(pr.W, dt)
    st = s.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0
    if precision == "fp64":
        assert_parity(got, ref, lambda X: o.rk3_step(X, dt), pr.W)
    else:
        assert np.all(rel_l1(got, ref) < MIXED_L1), rel_l1(got, ref)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shock_bubble_2048x1024_rhs(precision):
    pr = P.shock_bubble_2d(2048, 1024, seed=2)
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    sm = o.max_wavespeed(pr.W)
    dt = 0.5 / (sm[0] / (2.0 / pr.n[0]) + sm[1] / (1.0 / pr.n[1]))
    ref = pr.W + dt * o.rhs(pr.W, dt)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, **pr.eos)
    got = pr.W + dt * s.rhs(torch.from_numpy(pr.W).cuda(), dt).cpu().numpy()
    if precision == "fp64":
        assert_parity(got, ref, lambda X: X + dt * o.rhs(X, dt), pr.W)
    else:
        assert np.all(rel_l1(got, ref) < MIXED_L1), rel_l1(got, ref)
    s.close()


def _box(n, lo_idx, m, halo=3):
    """Index ranges of a box of m cells starting at lo_idx (per axis, x first)
    widened by the halo where it stays inside the grid; returns the slices
    into the full grid, the slices of the box's own cells inside the widened
    box, and for each axis whether each side is a domain face."""
    full, inner, faces = [], [], []
    for a in range(3):
        a0 = max(lo_idx[a] - halo, 0)
        a1 = min(lo_idx[a] + m + halo, n)
        full.append(slice(a0, a1))
        inner.append(slice(lo_idx[a] - a0, lo_idx[a] - a0 + m))
        faces.append((a0 == 0, a1 == n))
    return full, inner, faces


@pytest.fixture(scope="module")
def bubble_384():
    return P.bubble_collapse_3d(384)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bubble_collapse_384_sampled_rhs(bubble_384, precision):
    pr = bubble_384
    n = 384
    dx = 1.0 / n
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, **pr.eos)
    Wg = torch.from_numpy(pr.W).cuda()
    smax = np.array(s.max_wavespeed(Wg))
    dt = 0.5 / (smax.sum() / dx)
    L = s.rhs(Wg, dt)
    del Wg
    m = 12
    boxes = [(282, 186, 186),   # the interface on the +x axis
             (241, 241, 241),   # the interface on the diagonal
             (0, 0, 0),         # a domain corner (transmissive faces)
             (372, 186, 0)]     # far-field faces
    for b in boxes:
        full, inner, faces = _box(n, b, m)
        zs, ys, xs = full[2], full[1], full[0]
        Wb = np.ascontiguousarray(pr.W[:, zs, ys, xs])
        nb = (xs.stop - xs.start, ys.stop - ys.start, zs.stop - zs.start)
        lo = (xs.start * dx, ys.start * dx, zs.start * dx)
        hi = (xs.stop * dx, ys.stop * dx, zs.stop * dx)
        bcs = tuple(("transmissive", "transmissive") for _ in range(3))
        o = Oracle(nb, lo, hi, bcs, **pr.eos)
        sl = (slice(None), inner[2], inner[1], inner[0])
        ref = (Wb + dt * o.rhs_smax(Wb, dt, smax))[sl]
        got = Wb[sl] + dt * L[:, zs, ys, xs][sl].cpu().numpy()
        if precision == "fp64":
            fn = lambda X: (X + dt * o.rhs_smax(X, dt, smax))[sl]  # noqa: E731
            assert_parity(got, ref, fn, Wb)
        else:
            assert np.all(rel_l1(got, ref) < MIXED_L1), (b, rel_l1(got, ref))
    s.close()
    del L
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_riemann_batch_4096_sampled_step(precision):
    rb = P.riemann_batch()
    nprob = len(rb.sizes)
    b = Batch(rb.sizes, np.zeros(nprob), np.ones(nprob), "transmissive", "transmissive",
              precision=precision, **rb.eos)
    Wb = torch.from_numpy(rb.W).cuda()
    t = torch.zeros(nprob, dtype=torch.float64, device="cuda")
    b.advance(Wb, 1, cfl=0.5, t=t)
    got, tt = Wb.cpu().numpy(), t.cpu().numpy()
    st = b.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0
    rng = np.random.default_rng(0)
    picks = {int(np.argmin(rb.sizes)), int(np.argmax(rb.sizes))} | set(rng.choice(nprob, 6, replace=False).tolist())
    for k in sorted(picks):
        sl = slice(int(rb.offsets[k]), int(rb.offsets[k + 1]))
        n = int(rb.sizes[k])
        o = Oracle((n,), (0.0,), (1.0,), (("transmissive", "transmissive"),), **rb.eos)
        W0 = np.ascontiguousarray(rb.W[:, sl])
        dt = 0.5 / (o.max_wavespeed(W0)[0] * n)
        assert abs(tt[k] - dt) <= 1e-14 * dt
        ref = o.rk3_step(W0, dt)
        if precision == "fp64":
            assert relerr(got[:, sl], ref).max() < 1e-12, (k, relerr(got[:, sl], ref))
        else:
            assert np.all(rel_l1(got[:, sl], ref) < MIXED_L1), (k, rel_l1(got[:, sl], ref))
    b.close()
