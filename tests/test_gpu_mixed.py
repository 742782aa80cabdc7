"""GPU parity of the mixed FP32/FP64 path against the FP64 oracle, at the RHS
level, in 2D and 3D with every boundary kind.

These cases cover the parts of the mixed sweeps that the workload tests
reach only indirectly:
- the node cache that the sweeps of one RHS share (p, 1/rho, sound speed and
  certification bits stored by the first sweep and read by the others for
  cells and for periodic, symmetry and transmissive ghosts; Dirichlet ghosts
  are computed);
- the raw flux-difference scaling of the L array inside a step;
- the deferred pass that recomputes, with the FP64 limiter fallbacks, the
  midpoints whose FP32 certification fails.

An RHS L is compared through the forward-Euler stage W + dt L it feeds
(Sec. 5.3), in the units of the state.  The error is taken per field,
relative to that field's L1 (or max) norm of W, and the momentum components
share the momentum vector's scale.  The mixed bar is L1 <= 1e-5 relative
(the stated accuracy of the mixed solver).  On smooth data the L-infinity
error must also stay far below O(1): a cache entry read for the wrong cell
puts O(1) errors into whole midpoint fluxes.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import Solver  # noqa: E402

EOS = P.WORKLOAD_EOS


def scales(W, l1):
    nd = W.shape[0] - 4
    m = slice(2, 2 + nd)
    X = W.reshape(W.shape[0], -1)
    if l1:
        s = np.abs(X).sum(axis=1)
        s[m] = np.sqrt((X[m] ** 2).sum(axis=0)).sum()
    else:
        s = np.abs(X).max(axis=1)
        s[m] = np.sqrt((X[m] ** 2).sum(axis=0)).max()
    return np.maximum(s, 1e-300)


def stage_errors(W, dt, L_got, L_ref):
    """L1 and L-infinity errors of W + dt L_got against W + dt L_ref,
    relative to the state's per-field norms."""
    d = (dt * (L_got - L_ref)).reshape(W.shape[0], -1)
    return np.abs(d).sum(axis=1) / scales(W, True), np.abs(d).max(axis=1) / scales(W, False)


def cfl_dt(o, W, n, cfl=0.4):
    sm = o.max_wavespeed(W)
    return cfl / sum(sm[d] * n[d] for d in range(len(n)))


def dirichlet_states(W, bcs):
    """Uniform Dirichlet states: a boundary cell's state on each Dirichlet face."""
    nd = len(bcs)
    out = []
    for d in range(nd):
        pair_ = []
        for s in range(2):
            if bcs[d][s] != "dirichlet":
                pair_.append(None)
                continue
            sl = [slice(None)] + [0] * nd
            sl[nd - d] = 0 if s == 0 else -1
            pair_.append(W[tuple(sl)].copy())
        out.append(tuple(pair_))
    return tuple(out)


def admissible(W, eos):
    """The admissible set G of Sec. 2, written out here: positive partial
    densities, 0 <= alpha1 <= 1 and rho ctilde^2 = rho e - pbar > 0."""
    nd = W.shape[0] - 4
    a1 = W[3 + nd]
    rho = W[0] + W[1]
    ke = sum(W[2 + j] ** 2 for j in range(nd)) / (2.0 * rho)
    G = a1 / (eos["gamma_l"] - 1) + (1 - a1) / (eos["gamma_g"] - 1)
    Pi = a1 * eos["gamma_l"] * eos["pinf_l"] / (eos["gamma_l"] - 1)
    rct = (W[2 + nd] - ke) - Pi / (G + 1.0)
    return bool((W[0] >= 0).all() and (W[1] >= 0).all() and (a1 >= 0).all() and (a1 <= 1).all()
                and (rct > 0).all())


CASES = [
    ((48, 40), (("periodic", "periodic"), ("symmetry", "transmissive"))),
    ((45, 38), (("symmetry", "dirichlet"), ("periodic", "periodic"))),
    ((40, 36), (("dirichlet", "transmissive"), ("dirichlet", "symmetry"))),
    # several y tiles of 58 cells and a ragged tail
    ((30, 130), (("transmissive", "symmetry"), ("symmetry", "transmissive"))),
    ((16, 14, 12), (("periodic", "periodic"), ("symmetry", "dirichlet"), ("transmissive", "symmetry"))),
    ((14, 13, 15), (("dirichlet", "symmetry"), ("transmissive", "transmissive"), ("periodic", "periodic"))),
    # rows of 100 cells: two x tiles of 58 cells (58 + 42), while the small
    # grids above fit one
    ((100, 4, 6), (("transmissive", "symmetry"), ("periodic", "periodic"), ("transmissive", "transmissive"))),
]


@pytest.mark.parametrize("n,bcs", CASES)
def test_mixed_rhs_smooth_every_boundary_kind(n, bcs):
    W = P.random_admissible(n, seed=31 + len(n), jumps=False)
    dirichlet = dirichlet_states(W, bcs)
    o = Oracle(n, (0.0,) * len(n), (1.0,) * len(n), bcs, dirichlet=dirichlet, **EOS)
    s = Solver(n, (0.0,) * len(n), (1.0,) * len(n), bcs, precision="mixed", dirichlet=dirichlet, **EOS)
    dt = cfl_dt(o, W, n)
    ref = o.rhs(W, dt)
    got = s.rhs(torch.from_numpy(W).cuda(), dt).cpu().numpy()
    l1, linf = stage_errors(W, dt, got, ref)
    assert l1.max() < 1e-5 and linf.max() < 1e-4, (l1, linf)
    s.close()


@pytest.mark.parametrize("n,bcs", CASES[:1] + CASES[3:4])
def test_mixed_step_smooth_matches_oracle(n, bcs):
    """One SSPRK3 step (raw L scaling and the node cache in every stage)."""
    W = P.random_admissible(n, seed=41 + len(n), jumps=False)
    dirichlet = dirichlet_states(W, bcs)
    o = Oracle(n, (0.0,) * len(n), (1.0,) * len(n), bcs, dirichlet=dirichlet, **EOS)
    s = Solver(n, (0.0,) * len(n), (1.0,) * len(n), bcs, precision="mixed", dirichlet=dirichlet, **EOS)
    dt = cfl_dt(o, W, n)
    ref = o.rk3_step(W, dt)
    Wg = torch.from_numpy(W).cuda()
    s.rk3_step(Wg, dt)
    got = Wg.cpu().numpy()
    d = (got - ref).reshape(W.shape[0], -1)
    l1 = np.abs(d).sum(axis=1) / scales(ref, True)
    linf = np.abs(d).max(axis=1) / scales(ref, False)
    assert l1.max() < 1e-5 and linf.max() < 1e-4, (l1, linf)
    s.close()


def thin_phase_state(n, seed):
    """Smooth random fields with a band 0.4 < x < 0.6 in which the gas is
    nearly absent (alpha2 = 1e-9, so alpha2 rho2 sits about ten times above
    the 1e-10 limiter tolerance) around a pressure jump at x = 0.5: the flux
    limiter acts there, so the mixed path cannot certify those midpoints in
    FP32 and takes its FP64 fallback pass."""
    rng = np.random.default_rng(seed)
    grid = tuple(reversed(n))
    coords = np.meshgrid(*[(np.arange(k) + 0.5) / k for k in grid], indexing="ij")
    x = coords[-1]
    a1 = 0.5 + 0.3 * np.sin(2 * np.pi * (coords[0] + x))
    a1 = np.where((x > 0.4) & (x < 0.6), 1.0 - 1e-9, a1)
    rho_l = 1000.0 + 20.0 * rng.uniform(-1, 1) * np.cos(2 * np.pi * x)
    rho_g = 1.0 + 0.5 * np.sin(2 * np.pi * coords[0])
    p = np.where(x < 0.5, 2e6, 1e5) * (1.0 + 0.01 * np.sin(2 * np.pi * coords[0]))
    vel = [50.0 * np.sin(2 * np.pi * c) for c in reversed(coords)]
    return P.conservative(EOS, a1 * rho_l, (1.0 - a1) * rho_g, vel, p, a1), x


@pytest.mark.parametrize("n", [(64, 48), (20, 18, 16)])
def test_mixed_rhs_fallback_pass(n):
    """Where FP32 cannot resolve the flux of a nearly absent phase (deviations
    of O(1) next to partial densities of 1e-9), the mixed result legitimately
    departs from the oracle's: the limiter blends differently, as the design
    notes state for such flows.  What must hold exactly is checked instead:
    the deferred FP64 pass ran, every stage state is admissible (Sec. 5),
    the conserved components telescope to round-off on a periodic grid (each
    midpoint flux is stored once and used by both cells), and the cells
    whose stencils stay clear of the band match the oracle at the mixed bar."""
    W, x = thin_phase_state(n, seed=7)
    bcs = tuple(("periodic", "periodic") for _ in n)
    assert admissible(W, EOS)
    o = Oracle(n, (0.0,) * len(n), (1.0,) * len(n), bcs, **EOS)
    s = Solver(n, (0.0,) * len(n), (1.0,) * len(n), bcs, precision="mixed", **EOS)
    dt = cfl_dt(o, W, n, cfl=0.5)
    ref = o.rhs(W, dt)
    got = s.rhs(torch.from_numpy(W).cuda(), dt).cpu().numpy()
    st = s.stats()
    assert st["fp64_fallbacks"] > 0, st  # the deferred FP64 pass ran
    assert st["inadmissible"] == 0 and st["nonfinite"] == 0, st
    assert np.isfinite(got).all()
    # the positivity property of Sec. 5: the forward-Euler stage stays in G
    assert admissible(W + dt * ref, EOS)
    assert admissible(W + dt * got, EOS)
    # conservation of every component but alpha1 (periodic: the sums telescope)
    nf = W.shape[0]
    G = got.reshape(nf, -1)
    for f in range(nf - 1):
        assert abs(G[f].sum()) <= 1e-11 * np.abs(G[f]).sum(), (f, G[f].sum(), np.abs(G[f]).sum())
    # away from the band: 4 cells of stencil margin, and clear of the
    # periodic seam at x = 0 (where the pressure jumps back)
    h = 1.0 / n[0]
    far = ((x > 0.15) & (x < 0.4 - 4 * h)) | ((x > 0.6 + 4 * h) & (x < 0.85))
    d = (dt * (got - ref))[:, far]
    Wf = W[:, far]
    l1 = np.abs(d).sum(axis=1) / scales(Wf, True)
    linf = np.abs(d).max(axis=1) / scales(Wf, False)
    assert l1.max() < 1e-5 and linf.max() < 1e-3, (l1, linf)
    s.close()
