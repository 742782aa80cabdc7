"""Batched mode for 2D problems of uneven sizes (wcns_batch_create_grids).

Seeded 2D shock / air-bubble problems, 8 to 48 cells an axis drawn
separately (so most tiles are ragged), advanced together in one persistent
launch per direction and stage: every problem must equal the same problem
advanced alone through the single-grid solver, step for step (its own CFL
dt and directional split of Sec. 3.3 included), in FP64 and in mixed
precision; the batch's first FP64 step of a few problems must equal the
oracle's SSPRK3 step at the parity bar of the single-grid tests.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import Batch, Solver, WcnsError  # noqa: E402
from tests.test_gpu_parity import assert_parity, relerr  # noqa: E402

NPROB = 72


@pytest.fixture(scope="module")
def gb():
    # at least 3 cells an axis (symmetry faces need them)
    return P.bubble_batch_2d(nprob=NPROB, seed=7, nmin=8, nmax=48)


BCS = {"transmissive": (("transmissive", "transmissive"), ("transmissive", "transmissive")),
       "periodic_x_symmetry_y": (("periodic", "periodic"), ("symmetry", "transmissive"))}


@pytest.mark.parametrize("bcs", sorted(BCS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch2d_equals_single_grid_runs(gb, precision, bcs):
    bcs = BCS[bcs]
    b = Batch.grids(gb.sizes, gb.lo, gb.hi, bcs, precision=precision, **gb.eos)
    W = torch.from_numpy(gb.W).cuda()
    t = torch.zeros(NPROB, dtype=torch.float64, device="cuda")
    steps = 6
    b.advance(W, steps, cfl=0.5, t=t)
    st = b.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    assert st["midpoints"] > 0
    tune = b.tuning()
    assert tune is not None and tune["grid"] >= 1
    got, tt = W.cpu().numpy(), t.cpu().numpy()
    worst = 0.0
    for k in range(NPROB):
        nx, ny = (int(v) for v in gb.sizes[k])
        s = Solver((nx, ny), tuple(gb.lo[k]), tuple(gb.hi[k]), bcs, precision=precision, **gb.eos)
        Wk = torch.from_numpy(np.ascontiguousarray(gb.problem(k))).cuda()
        tk = s.advance_steps(Wk, steps, cfl=0.5)
        ref = Wk.cpu().numpy()
        mine = got[:, int(gb.offsets[k]):int(gb.offsets[k + 1])].reshape(ref.shape)
        e = relerr(mine, ref).max()
        worst = max(worst, e)
        assert e <= 1e-14, (k, nx, ny, relerr(mine, ref))
        assert abs(tt[k] - tk) <= 1e-14 * tk, (k, tt[k], tk)
        s.close()
    b.close()
    print("2D batch of %d problems vs single grids (%s, %s): worst relative difference %.1e" %
          (NPROB, precision, bcs, worst))


def test_batch2d_first_step_against_oracle(gb):
    """One batched FP64 step from the initial states of six problems: each
    equals the oracle's SSPRK3 step at its own CFL dt (Sec. 3.3)."""
    picks = [0, 5, 17, 33, 50, 71]
    sub = P.GridBatch(gb.sizes[picks], None, None, gb.lo[picks], gb.hi[picks], gb.bcs, gb.eos, {})
    parts = [np.ascontiguousarray(gb.problem(k)).reshape(6, -1) for k in picks]
    sub.offsets = np.concatenate([[0], np.cumsum([p.shape[1] for p in parts])])
    sub.W = np.ascontiguousarray(np.concatenate(parts, axis=1))
    b = Batch.grids(sub.sizes, sub.lo, sub.hi, sub.bcs, **gb.eos)
    W = torch.from_numpy(sub.W).cuda()
    t = torch.zeros(len(picks), dtype=torch.float64, device="cuda")
    b.advance(W, 1, cfl=0.5, t=t)
    got, tt = W.cpu().numpy(), t.cpu().numpy()
    for j, k in enumerate(picks):
        nx, ny = (int(v) for v in gb.sizes[k])
        W0 = np.ascontiguousarray(gb.problem(k))
        o = Oracle((nx, ny), tuple(gb.lo[k]), tuple(gb.hi[k]), gb.bcs, **gb.eos)
        sm = o.max_wavespeed(W0)
        dt = 0.5 / (sm[0] * nx + sm[1] * ny)
        assert abs(tt[j] - dt) <= 1e-13 * dt, (k, tt[j], dt)
        ref = o.rk3_step(W0, tt[j])
        mine = got[:, int(sub.offsets[j]):int(sub.offsets[j + 1])].reshape(W0.shape)
        assert_parity(mine, ref, lambda X: o.rk3_step(X, tt[j]), W0)
    b.close()


def test_batch2d_rejects_dirichlet_and_3d(gb):
    with pytest.raises(WcnsError):
        Batch.grids(gb.sizes[:2], gb.lo[:2], gb.hi[:2], (("dirichlet", "transmissive"), ("transmissive",) * 2),
                    **gb.eos)
    with pytest.raises(WcnsError):
        Batch.grids(np.full((2, 3), 8), np.zeros((2, 3)), np.ones((2, 3)), (("transmissive",) * 2,) * 3, **gb.eos)
