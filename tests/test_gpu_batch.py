"""Batched mode: many independent 1D two-phase Riemann problems in one
persistent launch per stage, CUDA-graph replayed, autotuned.

Each problem must evolve exactly as it does alone through the single-grid
path (same kernels, same per-problem CFL dt), and a few small problems are
checked against the FP64 oracle.
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


def relerr(a, b):
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_single_problem_runs(precision):
    rb = P.riemann_batch(nprob=24, seed=7, nmin=5, nmax=700)
    b = Batch(rb.sizes, np.zeros(24), np.ones(24), "transmissive", "transmissive", precision=precision, **rb.eos)
    Wb = torch.from_numpy(rb.W).cuda()
    t = torch.zeros(24, dtype=torch.float64, device="cuda")
    steps = 12
    b.advance(Wb, steps, cfl=0.5, t=t)
    got = Wb.cpu().numpy()
    tt = t.cpu().numpy()
    tune = b.tuning()
    tiles = (63, 127, 255) if precision == "fp64" else (58, 122, 250)
    assert tune is not None and tune["tile_cells"] in tiles and tune["grid"] >= 1
    st = b.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0
    for k in range(24):
        sl = slice(int(rb.offsets[k]), int(rb.offsets[k + 1]))
        n = int(rb.sizes[k])
        s = Solver((n,), (0.0,), (1.0,), (("transmissive", "transmissive"),), precision=precision, **rb.eos)
        W = torch.from_numpy(np.ascontiguousarray(rb.W[:, sl])).cuda()
        t_single = s.advance_steps(W, steps, cfl=0.5)
        ref = W.cpu().numpy()
        assert relerr(got[:, sl], ref).max() <= 1e-14, (k, n, relerr(got[:, sl], ref))
        assert abs(tt[k] - t_single) <= 1e-14 * t_single
        s.close()
    b.close()


def test_batch_first_step_against_oracle():
    """One batched step from the initial states: every problem matches the
    oracle's SSPRK3 step with its own CFL dt (per-problem dt, Sec. 3.3)."""
    rb = P.riemann_batch(nprob=6, seed=8, nmin=40, nmax=300)
    b = Batch(rb.sizes, np.zeros(6), np.ones(6), "transmissive", "transmissive", **rb.eos)
    Wb = torch.from_numpy(rb.W).cuda()
    t = torch.zeros(6, dtype=torch.float64, device="cuda")
    b.advance(Wb, 1, cfl=0.5, t=t)
    got, tt = Wb.cpu().numpy(), t.cpu().numpy()
    for k in range(6):
        sl = slice(int(rb.offsets[k]), int(rb.offsets[k + 1]))
        n = int(rb.sizes[k])
        o = Oracle((n,), (0.0,), (1.0,), (("transmissive", "transmissive"),), **rb.eos)
        W0 = np.ascontiguousarray(rb.W[:, sl])
        dt = 0.5 / (o.max_wavespeed(W0)[0] * n)
        ref = o.rk3_step(W0, dt)
        assert abs(tt[k] - dt) <= 1e-14 * dt
        err = relerr(got[:, sl], ref)
        assert err.max() < 1e-12, (k, err)
    b.close()


def test_batch_rejects_bad_arguments():
    with pytest.raises(Exception):
        Batch([10, 0], [0, 0], [1, 1], "transmissive", "transmissive", 1.4, 4.4, 6e8)
    with pytest.raises(Exception):
        Batch([10], [0], [1], "periodic", "transmissive", 1.4, 4.4, 6e8)
