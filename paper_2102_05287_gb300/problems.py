"""Seeded synthetic initial states for the five-equation gas-liquid solver.

This module only builds inputs.  It holds none of the scheme's arithmetic:
each problem is given by primitive fields (partial densities, velocity,
pressure, liquid volume fraction) and converted to the conservative vector
W = (a1r1, a2r2, rho u_1..rho u_ndim, E, alpha1) through the mixture
equation of state that defines E (Wong et al., Section 2):

    rho e = p * sum_k a_k/(g_k-1) + sum_k a_k g_k pinf_k/(g_k-1),
    E = rho e + rho |u|^2 / 2.

Phase 1 is the liquid (stiffened gas), phase 2 the gas (ideal).  Arrays are
float64 SoA of shape (nf, [n_z,] [n_y,] n_x), x fastest.

Problems follow the paper's tests (Section 6) and the solver's benchmark
workloads; every random draw comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Fluid table of the paper (Section 6): water (phase 1) and air (phase 2).
PAPER_EOS = dict(gamma_g=1.4, gamma_l=6.12, pinf_l=3.43e8)
# Water/air parameters of the shock-tube and bubble workloads.
WORKLOAD_EOS = dict(gamma_g=1.4, gamma_l=4.4, pinf_l=6e8)


@dataclass
class Problem:
    name: str
    W: np.ndarray
    n: tuple
    lo: tuple
    hi: tuple
    bcs: tuple
    eos: dict
    t_end: float = 0.0
    dt_fixed: float = 0.0
    cfl: float = 0.5
    steps: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.n)

    @property
    def ncells(self):
        return int(np.prod(self.n))


def conservative(eos, a1r1, a2r2, vel, p, alpha1):
    """Conservative SoA array from primitive fields (broadcast together)."""
    g1, p1 = eos["gamma_l"], eos["pinf_l"]
    g2 = eos["gamma_g"]
    a1 = np.asarray(alpha1, dtype=np.float64)
    a2 = 1.0 - a1
    rho = a1r1 + a2r2
    rhoe = p * (a1 / (g1 - 1.0) + a2 / (g2 - 1.0)) + a1 * (g1 * p1 / (g1 - 1.0))
    ke = sum(v * v for v in vel)
    fields = [a1r1, a2r2] + [rho * v for v in vel] + [rhoe + 0.5 * rho * ke, a1]
    shape = np.broadcast(*fields).shape
    return np.ascontiguousarray(np.stack([np.broadcast_to(f, shape) for f in fields]).astype(np.float64))


def _centers(n, lo, hi):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx


def stiffened_shock(rho0, p0, p1, gamma, pinf):
    """Post-shock density and velocity, and shock speed, for a right-moving
    shock into a stiffened gas at rest (Rankine-Hugoniot with p + pinf)."""
    a, b = p1 + pinf, p0 + pinf
    rho1 = rho0 * ((gamma + 1) * a + (gamma - 1) * b) / ((gamma - 1) * a + (gamma + 1) * b)
    m = math.sqrt((p1 - p0) / (1.0 / rho0 - 1.0 / rho1))
    return rho1, m * (1.0 / rho0 - 1.0 / rho1), m / rho0


def mixture_params(eos, alpha1):
    """(gamma_bar, pinf_bar) of a fixed-alpha mixture (Section 2)."""
    g1, p1, g2 = eos["gamma_l"], eos["pinf_l"], eos["gamma_g"]
    G = alpha1 / (g1 - 1) + (1 - alpha1) / (g2 - 1)
    Pi = alpha1 * g1 * p1 / (g1 - 1)
    gb = 1 + 1 / G
    return gb, Pi * (gb - 1) / gb


# ---------------------------------------------------------------------------
# Paper tests (Section 6)
# ---------------------------------------------------------------------------
def advection_2d(N, eos=PAPER_EOS):
    """Convergence study of Section 6.1: periodic [-1,1)^2, alpha1 =
    0.5 + 0.25 sin(pi(x+y)), rho1 = 1000, rho2 = 1, u = v = 10, p = 101325,
    dt/dx = 4e-5 s/m, t_end = 0.1 ms."""
    x = _centers(N, -1.0, 1.0)
    X, Y = np.meshgrid(x, x, indexing="xy")  # shape (ny, nx)
    a1 = 0.5 + 0.25 * np.sin(np.pi * (X + Y))
    W = conservative(eos, 1000.0 * a1, 1.0 * (1 - a1), [10.0, 10.0], 101325.0, a1)
    dx = 2.0 / N
    return Problem("advection_2d", W, (N, N), (-1.0, -1.0), (1.0, 1.0),
                   (("periodic", "periodic"), ("periodic", "periodic")), dict(eos),
                   t_end=1e-4, dt_fixed=4e-5 * dx,
                   extra=dict(exact=lambda t: 0.5 + 0.25 * np.sin(np.pi * (X + Y - 20.0 * t))))


def advection_1d_smooth(N, eos=WORKLOAD_EOS, t_end=1e-3):
    """Smooth-interface advection: periodic [0,1), alpha1 = 0.5 + 0.25 sin 2 pi x,
    rho1 = 1000, rho2 = 1, u = 1, p = 1e5; dt = 4e-5 dx."""
    x = _centers(N, 0.0, 1.0)
    a1 = 0.5 + 0.25 * np.sin(2 * np.pi * x)
    W = conservative(eos, 1000.0 * a1, 1.0 * (1 - a1), [1.0], 1e5, a1)
    return Problem("advection_1d_smooth", W, (N,), (0.0,), (1.0,), (("periodic", "periodic"),),
                   dict(eos), t_end=t_end, dt_fixed=4e-5 / N,
                   extra=dict(exact=lambda t: 0.5 + 0.25 * np.sin(2 * np.pi * (x - t))))


def interface_advection_1d(N=200, eos=PAPER_EOS):
    """Section 6.2: two material interfaces advected once around [0,1)."""
    x = _centers(N, 0.0, 1.0)
    inside = (x >= 0.25) & (x < 0.75)
    eps = 1e-8
    a1 = np.where(inside, 1 - eps, eps)
    a1r1 = np.where(inside, 1000.0, 1e-8)
    a2r2 = np.where(inside, 1e-8, 1.204)
    W = conservative(eos, a1r1, a2r2, [100.0], 101325.0, a1)
    return Problem("interface_advection_1d", W, (N,), (0.0,), (1.0,), (("periodic", "periodic"),),
                   dict(eos), t_end=0.01, dt_fixed=1.25e-6)


def sod_gas_liquid(N=200, eos=PAPER_EOS):
    """Section 6.3: gas/liquid Sod tube on [0, 1.5], split at 0.8."""
    x = _centers(N, 0.0, 1.5)
    left = x < 0.8
    eps = 1e-8
    a1 = np.where(left, 1 - eps, eps)
    a1r1 = np.where(left, 1000.0, 1e-8)
    a2r2 = np.where(left, 1e-8, 20.0)
    p = np.where(left, 1e9, 1e5)
    W = conservative(eos, a1r1, a2r2, [0.0], p, a1)
    return Problem("sod_gas_liquid", W, (N,), (0.0,), (1.5,),
                   (("transmissive", "transmissive"),), dict(eos), t_end=3e-4, dt_fixed=1.25e-6)


def sedov_multimaterial(N=401, eos=PAPER_EOS):
    """Section 6.4: planar multi-material Sedov blast in [0, 4]; the centre
    cell holds air at p = 1.28e6/dx, the rest water at p = -3e7."""
    dx = 4.0 / N
    x = _centers(N, 0.0, 4.0)
    core = np.abs(x - 2.0) <= 0.5 * dx
    eps = 1e-8
    a1 = np.where(core, eps, 1 - eps)
    a1r1 = np.where(core, 1e-8, 1000.0)
    a2r2 = np.where(core, 1.0, 1e-8)
    p = np.where(core, 1.28e6 / dx, -3e7)
    W = conservative(eos, a1r1, a2r2, [0.0], p, a1)
    return Problem("sedov_multimaterial", W, (N,), (0.0,), (4.0,),
                   (("transmissive", "transmissive"),), dict(eos), t_end=1e-3, dt_fixed=2.5e-7)


def mach10_water_cylinder(nx=1152, ny=768, eos=PAPER_EOS, x_shock=8e-3):
    """Section 6 Mach 10 shock / water cylinder: [0, 30L] x [-10L, 10L],
    L = 1 mm, constant extrapolation on every face; water cylinder of
    diameter 8L at (13L, 0) in air, cells whose centre lies inside it are
    water (sharp interface); the incident shock stands at x = x_shock
    (8L, one L upstream of the cylinder: the paper gives the position only
    in a schematic).  States from the paper's initial-condition table."""
    L = 1e-3
    x = _centers(nx, 0.0, 30 * L)
    y = _centers(ny, -10 * L, 10 * L)
    X, Y = np.meshgrid(x, y, indexing="xy")
    water = np.hypot(X - 13 * L, Y) < 4 * L
    post = X < x_shock
    eps = 1e-8
    a1 = np.where(water, 1 - eps, eps)
    a1r1 = np.where(water, 1000.0, 1e-8)
    a2r2 = np.where(water, 1e-8, np.where(post, 6.8571, 1.2))
    u = np.where(post & ~water, 2.8179e3, 0.0)
    p = np.where(post & ~water, 1.165e7, 1e5)
    W = conservative(eos, a1r1, a2r2, [u, np.zeros_like(u)], p, a1)
    tr = ("transmissive", "transmissive")
    return Problem("mach10_water_cylinder", W, (nx, ny), (0.0, -10 * L), (30 * L, 10 * L), (tr, tr), dict(eos),
                   cfl=0.5)


def mach100_water_jet(nx=1024, ny=512, eos=PAPER_EOS):
    """Section 6 Mach 100 water jet: [0, 1] x [-0.25, 0.25] filled with
    ambient air (p 1e5); the left face is a Dirichlet face whose state is a
    water jet (rho 1000, u 1.5e5, p 1e5) for |y| <= 0.05 and the ambient air
    elsewhere; constant extrapolation on the other faces.  The face states
    are in extra["dirichlet_face"][(0, 0)] as a (6, ny) array."""
    x = _centers(nx, 0.0, 1.0)
    y = _centers(ny, -0.25, 0.25)
    eps = 1e-8
    ones = np.ones((ny, nx))
    W = conservative(eos, 1e-8 * ones, ones, [0.0 * ones, 0.0 * ones], 1e5 * ones, eps * ones)
    jet = np.abs(y) <= 0.05
    face = conservative(eos, np.where(jet, 1000.0, 1e-8), np.where(jet, 1e-8, 1.0),
                        [np.where(jet, 1.5e5, 0.0), np.zeros(ny)], np.full(ny, 1e5),
                        np.where(jet, 1 - eps, eps))
    ambient = conservative(eos, 1e-8, 1.0, [0.0, 0.0], 1e5, eps)
    bcs = (("dirichlet", "transmissive"), ("transmissive", "transmissive"))
    return Problem("mach100_water_jet", W, (nx, ny), (0.0, -0.25), (1.0, 0.25), bcs, dict(eos), cfl=0.5,
                   extra=dict(dirichlet=((ambient, None), (None, None)), dirichlet_face={(0, 0): face}))


# ---------------------------------------------------------------------------
# Benchmark workloads
# ---------------------------------------------------------------------------
def water_air_shock_tube(N=200, eos=WORKLOAD_EOS, floor=1e-6):
    """1D water-air shock tube: [0,1], transmissive; water rho 1000, p 1e9 for
    x < 0.7, air rho 50, p 1e5 beyond; volume-fraction floor 1e-6; RK3 at
    CFL 0.5 to t = 2.4e-4 s."""
    x = _centers(N, 0.0, 1.0)
    left = x < 0.7
    a1 = np.where(left, 1 - floor, floor)
    a1r1 = a1 * 1000.0
    a2r2 = (1 - a1) * 50.0
    p = np.where(left, 1e9, 1e5)
    W = conservative(eos, a1r1, a2r2, [0.0], p, a1)
    return Problem("water_air_shock_tube", W, (N,), (0.0,), (1.0,),
                   (("transmissive", "transmissive"),), dict(eos), t_end=2.4e-4, cfl=0.5,
                   extra=dict(x0=0.7, left=(1000.0, 0.0, 1e9, 1 - floor), right=(50.0, 0.0, 1e5, floor),
                              rho_l=(1000.0, 50.0)))


def _fourier_radius(rng, R0, amp, mmax=16):
    a = rng.uniform(-1.0, 1.0, size=mmax - 1)
    phi = rng.uniform(0.0, 2 * np.pi, size=mmax - 1)
    m = np.arange(2, mmax + 1)
    th = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
    pert = (a[:, None] * np.cos(m[:, None] * th[None, :] + phi[:, None])).sum(0)
    scale = amp / np.abs(pert).max()
    return lambda theta: R0 + scale * (a[:, None] * np.cos(m[:, None] * theta[None, ...] + phi[:, None])
                                       ).sum(0)


def shock_bubble_2d(nx=1024, ny=512, eos=WORKLOAD_EOS, seed=1, floor=1e-6, steps=2000):
    """2D shock / air-bubble interaction in water on [0,2]x[0,1]: symmetry at
    y = 0, transmissive elsewhere.  Air bubble (rho 1, p 1e5) of radius 0.2 at
    (1, 0) with a tanh interface about two cells wide and a seeded Fourier
    radius perturbation (modes 2..16, max amplitude 1e-3); water (rho 1000,
    p 1e5) with a planar shock at x = 0.6 whose post-shock pressure is 1.9e9
    (Rankine-Hugoniot of the fixed-alpha mixture)."""
    rng = np.random.default_rng(seed)
    dx = 2.0 / nx
    x = _centers(nx, 0.0, 2.0)
    y = _centers(ny, 0.0, 1.0)
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.hypot(X - 1.0, Y)
    theta = np.arctan2(Y, X - 1.0)
    Rfun = _fourier_radius(rng, 0.2, 1e-3)
    Rth = Rfun(theta.ravel()).reshape(theta.shape)
    a_gas = floor + (1 - 2 * floor) * 0.5 * (1 - np.tanh((r - Rth) / dx))
    a1 = 1.0 - a_gas
    gb, pb = mixture_params(eos, 1 - floor)
    rho_pre = (1 - floor) * 1000.0 + floor * 1.0
    rho_post, u_post, _ = stiffened_shock(rho_pre, 1e5, 1.9e9, gb, pb)
    comp = rho_post / rho_pre
    post = X < 0.6
    rho_w = np.where(post, 1000.0 * comp, 1000.0)
    rho_a = np.where(post, 1.0 * comp, 1.0)
    u = np.where(post, u_post, 0.0)
    p = np.where(post, 1.9e9, 1e5)
    W = conservative(eos, a1 * rho_w, (1 - a1) * rho_a, [u, np.zeros_like(u)], p, a1)
    return Problem("shock_bubble_2d", W, (nx, ny), (0.0, 0.0), (2.0, 1.0),
                   (("transmissive", "transmissive"), ("symmetry", "transmissive")), dict(eos),
                   cfl=0.5, steps=steps)


def bubble_collapse_3d(n=384, eos=WORKLOAD_EOS, seed=4, floor=1e-6, steps=500):
    """3D air-bubble collapse in water on [0,1]^3, transmissive: bubble of
    radius 0.25 at the centre (air rho 1, p 1e5) in water (rho 1000, p 1e8),
    radius perturbed by seeded zonal spherical harmonics of degree 2..16
    about random axes, max amplitude 1e-3; tanh interface about two cells.

    Built one z-slab at a time.  The perturbation is evaluated only within
    25 cells of the unperturbed sphere: farther out (r - R)/dx exceeds 19,
    where tanh is +-1 in double precision, so it cannot change the state;
    its amplitude is normalised over those cells."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    x = _centers(n, 0.0, 1.0)
    modes = []
    for l in range(2, 17):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        coef = np.zeros(l + 1)
        coef[l] = rng.uniform(-1, 1)
        modes.append((k, coef))
    Y, X = np.meshgrid(x, x, indexing="ij")
    dX, dY = X - 0.5, Y - 0.5
    shell = 25 * dx

    def slab_pert(zc):
        dZ = zc - 0.5
        r = np.sqrt(dX * dX + dY * dY + dZ * dZ)
        near = np.abs(r - 0.25) < shell
        rs = r[near]
        cx, cy, cz = dX[near] / rs, dY[near] / rs, dZ / rs
        pert = np.zeros(rs.shape)
        for k, coef in modes:
            pert += np.polynomial.legendre.legval(cx * k[0] + cy * k[1] + cz * k[2], coef)
        return r, near, pert

    slabs = [slab_pert(zc) for zc in x]
    amp = max((np.abs(pv).max() for _, _, pv in slabs if pv.size), default=0.0)
    scale = 1e-3 / max(amp, 1e-300)
    nf = 7
    W = np.empty((nf, n, n, n))
    zero = np.zeros((n, n))
    for iz, (r, near, pert) in enumerate(slabs):
        R = np.full(r.shape, 0.25)
        R[near] += pert * scale
        a_gas = floor + (1 - 2 * floor) * 0.5 * (1 - np.tanh((r - R) / dx))
        a1 = 1.0 - a_gas
        p = np.where(r < R, 1e5, 1e8)
        W[:, iz] = conservative(eos, a1 * 1000.0, (1 - a1) * 1.0, [zero, zero, zero], p, a1)
    tr = ("transmissive", "transmissive")
    return Problem("bubble_collapse_3d", W, (n, n, n), (0.0,) * 3, (1.0,) * 3, (tr, tr, tr), dict(eos),
                   cfl=0.5, steps=steps)


@dataclass
class RiemannBatch:
    sizes: np.ndarray       # cells per problem
    offsets: np.ndarray     # first cell of each problem in the packed array
    W: np.ndarray           # packed SoA (5, total_cells)
    eos: dict
    params: dict


def riemann_batch(nprob=4096, seed=3, eos=WORKLOAD_EOS, nmin=128, nmax=8192, floor=1e-6):
    """Independent 1D two-phase Riemann problems on [0,1] with transmissive
    ends: sizes log-uniform in [nmin, nmax]; pressure ratio log-uniform in
    [10, 1e4] with gas at p = 1e5 on the right and liquid at 1e5*ratio on the
    left; liquid density U[900,1100], gas density U[1,100], interface
    position U[0.3, 0.7]."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=nprob)).astype(np.int64)
    ratio = np.exp(rng.uniform(np.log(10.0), np.log(1e4), size=nprob))
    rho_l = rng.uniform(900.0, 1100.0, size=nprob)
    rho_g = rng.uniform(1.0, 100.0, size=nprob)
    x0 = rng.uniform(0.3, 0.7, size=nprob)
    offsets = np.zeros(nprob + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    a1 = np.empty(total)
    a1r1 = np.empty(total)
    a2r2 = np.empty(total)
    p = np.empty(total)
    for k in range(nprob):
        n = int(sizes[k])
        x = _centers(n, 0.0, 1.0)
        left = x < x0[k]
        sl = slice(int(offsets[k]), int(offsets[k + 1]))
        a = np.where(left, 1 - floor, floor)
        a1[sl] = a
        a1r1[sl] = a * rho_l[k]
        a2r2[sl] = (1 - a) * rho_g[k]
        p[sl] = np.where(left, 1e5 * ratio[k], 1e5)
    W = conservative(eos, a1r1, a2r2, [np.zeros(total)], p, a1)
    return RiemannBatch(sizes, offsets, W, dict(eos),
                        dict(ratio=ratio, rho_l=rho_l, rho_g=rho_g, x0=x0))


@dataclass
class GridBatch:
    sizes: np.ndarray       # (nprob, ndim) cells per axis, x first
    offsets: np.ndarray     # first cell of each problem in the packed array
    W: np.ndarray           # packed SoA (nf, total_cells), each problem x fastest
    lo: np.ndarray          # (nprob, ndim)
    hi: np.ndarray          # (nprob, ndim)
    bcs: tuple
    eos: dict
    params: dict

    def problem(self, k):
        """Problem k's state as a (nf, ny, nx) array."""
        nx, ny = (int(v) for v in self.sizes[k])
        return self.W[:, int(self.offsets[k]):int(self.offsets[k + 1])].reshape(self.W.shape[0], ny, nx)


def bubble_batch_2d(nprob=1024, seed=5, eos=WORKLOAD_EOS, nmin=32, nmax=256, floor=1e-6):
    """Independent 2D shock / air-bubble problems of uneven sizes on [0,1]^2,
    transmissive on every face (the 2D shock/bubble workload's physics in
    problems of tens to hundreds of cells an axis): nx and ny log-uniform in
    [nmin, nmax] (drawn separately); an air bubble (density U[1,100], p 1e5)
    of radius U[0.1, 0.25] centred at U[0.4, 0.6]^2 with a tanh interface
    about one cell wide, in water (density U[900,1100], p 1e5); a planar
    shock at x = U[0.05, 0.12] with post-shock pressure 1e5 times a ratio
    log-uniform in [10, 1e4] (Rankine-Hugoniot of the fixed-alpha mixture)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=(nprob, 2))).astype(np.int64)
    ratio = np.exp(rng.uniform(np.log(10.0), np.log(1e4), size=nprob))
    rho_l = rng.uniform(900.0, 1100.0, size=nprob)
    rho_g = rng.uniform(1.0, 100.0, size=nprob)
    R = rng.uniform(0.1, 0.25, size=nprob)
    ctr = rng.uniform(0.4, 0.6, size=(nprob, 2))
    xs = rng.uniform(0.05, 0.12, size=nprob)
    ncell = sizes[:, 0] * sizes[:, 1]
    offsets = np.zeros(nprob + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ncell)
    total = int(offsets[-1])
    a1 = np.empty(total)
    a1r1 = np.empty(total)
    a2r2 = np.empty(total)
    u = np.empty(total)
    p = np.empty(total)
    gb, pb = mixture_params(eos, 1 - floor)
    for k in range(nprob):
        nx, ny = int(sizes[k, 0]), int(sizes[k, 1])
        X, Y = np.meshgrid(_centers(nx, 0.0, 1.0), _centers(ny, 0.0, 1.0), indexing="xy")
        r = np.hypot(X - ctr[k, 0], Y - ctr[k, 1])
        h = min(1.0 / nx, 1.0 / ny)
        a_gas = floor + (1 - 2 * floor) * 0.5 * (1 - np.tanh((r - R[k]) / h))
        a = 1.0 - a_gas
        rho_pre = (1 - floor) * rho_l[k] + floor * rho_g[k]
        rho_post, u_post, _ = stiffened_shock(rho_pre, 1e5, 1e5 * ratio[k], gb, pb)
        comp = rho_post / rho_pre
        post = X < xs[k]
        sl = slice(int(offsets[k]), int(offsets[k + 1]))
        a1[sl] = a.ravel()
        a1r1[sl] = (a * np.where(post, rho_l[k] * comp, rho_l[k])).ravel()
        a2r2[sl] = ((1 - a) * np.where(post, rho_g[k] * comp, rho_g[k])).ravel()
        u[sl] = np.where(post, u_post, 0.0).ravel()
        p[sl] = np.where(post, 1e5 * ratio[k], 1e5).ravel()
    W = conservative(eos, a1r1, a2r2, [u, np.zeros(total)], p, a1)
    lo = np.zeros((nprob, 2))
    hi = np.ones((nprob, 2))
    return GridBatch(sizes, offsets, W, lo, hi, (("transmissive", "transmissive"),) * 2, dict(eos),
                     dict(ratio=ratio, rho_l=rho_l, rho_g=rho_g, R=R, centre=ctr, x_shock=xs))


def random_admissible(shape_n, eos=WORKLOAD_EOS, seed=0, jumps=True):
    """Random admissible states on a grid of shape n (x first): smooth random
    fields plus, if ``jumps``, a few material/pressure discontinuities.
    Values span the workloads' ranges (liquid/gas densities, pressures up to
    ~1e9, velocities up to a few hundred m/s, alpha in [1e-6, 1-1e-6])."""
    rng = np.random.default_rng(seed)
    ndim = len(shape_n)
    grid_shape = tuple(reversed(shape_n))

    def smooth(lo, hi):
        f = np.zeros(grid_shape)
        coords = np.meshgrid(*[np.linspace(0, 1, s) for s in grid_shape], indexing="ij")
        for _ in range(3):
            k = rng.uniform(0.5, 3.0, size=ndim)
            ph = rng.uniform(0, 2 * np.pi)
            f += np.sin(2 * np.pi * sum(k[i] * coords[i] for i in range(ndim)) + ph)
        f = (f - f.min()) / max(f.max() - f.min(), 1e-30)
        return lo + (hi - lo) * f

    a1 = smooth(0.05, 0.95)
    rho_w = smooth(950.0, 1050.0)
    rho_a = smooth(1.0, 5.0)
    p = smooth(1e5, 5e6)
    vel = [smooth(-200.0, 200.0) for _ in range(ndim)]
    if jumps:
        coords = np.meshgrid(*[np.linspace(0, 1, s) for s in grid_shape], indexing="ij")
        for _ in range(2):
            ax = rng.integers(0, ndim)
            pos = rng.uniform(0.2, 0.8)
            mask = coords[ax] > pos
            a1 = np.where(mask, rng.choice([1e-6, 1 - 1e-6]), a1)
            p = np.where(mask, p * rng.uniform(1.0, 50.0), p)
    W = conservative(eos, a1 * rho_w, (1 - a1) * rho_a, vel, p, a1)
    return W
