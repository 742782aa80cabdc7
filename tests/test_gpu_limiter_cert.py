"""The FP64 sweeps' FP32 certification of the limiter threshold tests.

The FP64 sweeps skip the interpolation limiter (Sec. 5.1, Algorithms 1-3)
and the flux limiter (Sec. 5.2, Algorithms 4-6) at a midpoint when an FP32
test, formed from operands truncated to 20 mantissa bits with a rigorous
error margin, shows that every threshold test passes.  That is only correct
if the FP64 limiter would leave the states and fluxes unchanged too.  Through
the C ABI (wcns_check_limiter_cert) both run on the same inputs on the
device:

* soundness: every certified case is one the FP64 limiter leaves unchanged;
  the cases crowd every threshold (alpha1 rho1, alpha2 rho2, alpha1,
  1 - alpha1, rho ctilde^2) from both sides, at relative distances from a
  few ulps to 1e3, with zero, subnormal, huge and non-finite components;
* liveness: clearly admissible states and half states are certified, so
  the fast path is the one the sweeps take away from the limiters' work.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300 import problems as P  # noqa: E402
from paper_2102_05287_gb300 import wcns  # noqa: E402

EPS = dict(eps_ar=1e-10, eps_a=1e-10, eps_rc=1e-8)
EOS = P.WORKLOAD_EOS
DELTAS = np.array([-1.0, -1e-3, -1e-6, -1e-9, -1e-12, -1e-15, 0.0, 1e-15, 1e-12, 1e-9, 1e-7, 4e-6, 1e-5,
                   1e-4, 1e-2, 1.0, 1e3])


def check(ndim, kind, rows):
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    n = rows.shape[0]
    t = torch.from_numpy(rows).cuda()
    cert = torch.zeros(n, dtype=torch.int32, device="cuda")
    exact = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = wcns.load().wcns_check_limiter_cert(ndim, kind, C.c_void_p(t.data_ptr()), n, EPS["eps_ar"], EPS["eps_a"],
                                             EPS["eps_rc"], EOS["gamma_g"], EOS["gamma_l"], EOS["pinf_l"],
                                             C.c_void_p(cert.data_ptr()), C.c_void_p(exact.data_ptr()), None)
    assert st == wcns.WCNS_OK
    torch.cuda.synchronize()
    return cert.cpu().numpy().astype(bool), exact.cpu().numpy().astype(bool)


def eos_terms(W, ndim):
    """Kinetic energy and pbar = Pi / (Gamma + 1) of conservative states
    (Sec. 2); used only to place test states at a chosen rho ctilde^2."""
    g1, p1, g2 = EOS["gamma_l"], EOS["pinf_l"], EOS["gamma_g"]
    r1, r2 = 1.0 / (g1 - 1.0), 1.0 / (g2 - 1.0)
    q1 = g1 * p1 / (g1 - 1.0)
    rho = W[0] + W[1]
    ke = 0.5 * sum(W[2 + j] ** 2 for j in range(ndim)) / rho
    a = W[3 + ndim]
    return ke, q1 * a / (r2 + (r1 - r2) * a + 1.0)


def random_primitives(rng, n, ndim, extreme=False, pmin=1.0):
    """Primitive states over the workloads' range: water and air, pmin to
    1 GPa, speeds up to 1 km/s (up to 30 km/s with extreme)."""
    a1 = np.where(rng.random(n) < 0.5, rng.uniform(1e-6, 1e-3, n), 1.0 - rng.uniform(1e-6, 1e-3, n))
    a1 = np.where(rng.random(n) < 0.3, rng.uniform(0.0, 1.0, n), a1)
    p = 10.0 ** rng.uniform(np.log10(pmin), 9.0, n)
    vmax = 3e4 if extreme else 1e3
    vel = [rng.uniform(-vmax, vmax, n) * (rng.random(n) < 0.8) for _ in range(ndim)]
    return [a1 * 1000.0 * rng.uniform(0.5, 1.5, n), (1 - a1) * rng.uniform(0.5, 2.0, n), vel, p, a1]


def random_states(rng, n, ndim, extreme=False, pmin=1.0):
    """Admissible conservative states (columns)."""
    return P.conservative(EOS, *random_primitives(rng, n, ndim, extreme, pmin))


def nearby_states(rng, prim):
    """Admissible states within 10 % of given primitives (alpha1 within 10 %
    of its distance to 0 and 1), as a half step of smooth flow leaves them."""
    a1r1, a2r2, vel, p, a1 = prim
    n = p.size

    def f():
        return rng.uniform(0.9, 1.1, n)

    vs = [v * f() + rng.uniform(-10.0, 10.0, n) for v in vel]
    a1n = a1 + rng.uniform(-0.1, 0.1, n) * np.minimum(a1, 1.0 - a1)
    return P.conservative(EOS, a1r1 * f(), a2r2 * f(), vs, p * f(), a1n)


def place(W, ndim, which, delta):
    """Move quantity `which` of states W (columns) to its tolerance times
    (1 + delta): 0 alpha1 rho1, 1 alpha2 rho2, 2 alpha1, 3 1 - alpha1,
    4 rho ctilde^2 (through E)."""
    W = W.copy()
    A, E = 3 + ndim, 2 + ndim
    if which == 0:
        W[0] = EPS["eps_ar"] * (1 + delta)
    elif which == 1:
        W[1] = EPS["eps_ar"] * (1 + delta)
    elif which == 2:
        W[A] = EPS["eps_a"] * (1 + delta)
    elif which == 3:
        W[A] = 1.0 - EPS["eps_a"] * (1 + delta)
    else:
        ke, pb = eos_terms(W, ndim)
        W[E] = ke + pb + EPS["eps_rc"] * (1 + delta)
    return W


def special(rng, W, ndim):
    """Put zeros, subnormals, huge values and non-finite values into random
    components of some states."""
    W = W.copy()
    nf, n = W.shape
    vals = np.array([0.0, -0.0, 5e-324, -2e-310, 1e-40, 3e38, 1e39, 1e200, np.inf, -np.inf, np.nan])
    k = rng.integers(0, n, n // 4)
    W[rng.integers(0, nf, k.size), k] = vals[rng.integers(0, vals.size, k.size)]
    return W


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_interp_certification_is_sound_and_live(ndim):
    rng = np.random.default_rng(100 + ndim)
    nf = ndim + 4
    n = 4000
    node = random_states(rng, n, ndim, pmin=1e3)
    interp = random_states(rng, n, ndim, pmin=1e3)
    # liveness on clearly admissible pairs
    cert, exact = check(ndim, 0, np.concatenate([node, interp]).T)
    assert np.all(exact[cert]), "certified a pair the FP64 limiter changes"
    assert cert.mean() > 0.99, cert.mean()
    # soundness next to every threshold, for the interpolated and the node state
    rows = []
    for which in range(5):
        for d in DELTAS:
            m = 300
            a, b = random_states(rng, m, ndim, extreme=True), random_states(rng, m, ndim, extreme=True)
            rows.append(np.concatenate([a, place(b, ndim, which, d)]).T)
            rows.append(np.concatenate([place(a, ndim, which, d), b]).T)
    rows.append(np.concatenate([special(rng, random_states(rng, n, ndim), ndim),
                                special(rng, random_states(rng, n, ndim), ndim)]).T)
    rows = np.concatenate(rows)
    assert rows.shape[1] == 2 * nf
    cert, exact = check(ndim, 0, rows)
    bad = np.flatnonzero(cert & ~exact)
    assert bad.size == 0, rows[bad[:3]]
    assert (~exact).sum() > 1000  # the placed states do straddle the thresholds
    assert cert.sum() > 1000


def flux_rows(rng, n, ndim, extreme=False, pmin=1.0):
    """Midpoint inputs of the flux limiter whose four half states are
    chosen admissible states near their nodes: W_i - 2 lam (G^- - F_i) = X_i
    and W_{i+1} + 2 lam (G^- - F_{i+1}) = X_{i+1} fix the node fluxes F for
    a random high-order flux G^-, and the first-order flux is G^- to within
    1e-7 (as in smooth flow), so its half states are X to within that."""
    nf, A = ndim + 4, 3 + ndim
    pi, pi1 = random_primitives(rng, n, ndim, extreme, pmin), random_primitives(rng, n, ndim, extreme, pmin)
    Wi, Wi1 = P.conservative(EOS, *pi), P.conservative(EOS, *pi1)
    Xi, Xi1 = nearby_states(rng, pi), nearby_states(rng, pi1)
    lam = 10.0 ** rng.uniform(-6.0, -2.0, n)
    l2 = 2 * lam
    Gm = rng.uniform(-0.5, 0.5, (nf, n)) * np.maximum(np.abs(Wi), np.abs(Wi1)) / l2
    Fi = Gm + (Xi - Wi) / l2
    Fi1 = Gm - (Xi1 - Wi1) / l2
    Gm[A] = (Wi[A] - Xi[A]) / l2
    Gp = Gm.copy()
    Gp[A] = (Xi1[A] - Wi1[A]) / l2
    GHm = Gm * (1 + rng.uniform(-1e-7, 1e-7, (nf, n)))
    GHp = GHm.copy()
    GHp[A] = Gp[A] * (1 + rng.uniform(-1e-7, 1e-7, n))
    return [Wi, Wi1, Fi, Fi1, GHm, GHp, Gm, Gp], lam


def pack(parts, lam):
    return np.concatenate(parts + [lam[None, :]]).T


def place_half(parts, lam, ndim, st, which, delta):
    """Set half state st (0 W_i - 2 lam (G^{HLLC,-} - F_i), 1 W_{i+1} +
    2 lam (G^{HLLC,+} - F_{i+1}), 2 and 3 the same with G^-, G^+) so that
    its quantity `which` sits at its tolerance times (1 + delta), through
    the flux (shared components of G^{HLLC} / G^- move both half states of
    that flux; the alpha flux is per side)."""
    Wi, Wi1, Fi, Fi1, GHm, GHp, Gm, Gp = [x.copy() for x in parts]
    A, E = 3 + ndim, 2 + ndim
    right = st & 1
    W, F = (Wi1, Fi1) if right else (Wi, Fi)
    G = (GHp if right else GHm) if st < 2 else (Gp if right else Gm)
    Gshared = GHm if st < 2 else Gm
    s = 1.0 if right else -1.0
    l2 = 2 * lam
    Fa = np.zeros_like(W[0])

    def half(f):
        g = G[f] if f == A else Gshared[f]
        return W[f] + s * l2 * (g - (Fa if f == A else F[f]))

    X = np.stack([half(f) for f in range(ndim + 4)])
    target = place(X, ndim, which, delta)
    f = {0: 0, 1: 1, 2: A, 3: A, 4: E}[which]
    if f == A:
        G[A] = (target[A] - W[A]) / (s * l2)
    else:
        Gshared[f] = F[f] + (target[f] - W[f]) / (s * l2)
    if st < 2:
        GHp[:A] = GHm[:A]
    else:
        Gp[:A] = Gm[:A]
    return [Wi, Wi1, Fi, Fi1, GHm, GHp, Gm, Gp]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_flux_certification_is_sound_and_live(ndim):
    rng = np.random.default_rng(200 + ndim)
    nf = ndim + 4
    parts, lam = flux_rows(rng, 4000, ndim, pmin=1e3)
    cert, exact = check(ndim, 1, pack(parts, lam))
    assert np.all(exact[cert]), "certified a midpoint the FP64 limiter changes"
    assert cert.mean() > 0.99, cert.mean()
    rows = []
    for st in range(4):
        for which in range(5):
            for d in DELTAS:
                parts, lam = flux_rows(rng, 120, ndim, extreme=True)
                rows.append(pack(place_half(parts, lam, ndim, st, which, d), lam))
    parts, lam = flux_rows(rng, 4000, ndim)
    rows.append(pack([special(rng, x, ndim) for x in parts], lam))
    rows = np.concatenate(rows)
    assert rows.shape[1] == 8 * nf + 1
    cert, exact = check(ndim, 1, rows)
    bad = np.flatnonzero(cert & ~exact)
    assert bad.size == 0, rows[bad[:2]]
    assert (~exact).sum() > 1000
    assert cert.sum() > 1000


def node_data(W, ndim):
    """Velocity, pressure and sound speed of conservative states (Sec. 2:
    p = (rho e - Pi) / Gamma, rho c^2 = ((Gamma + 1) rho e - Pi) / Gamma^2)
    and their physical flux along the last axis (alpha component unused)."""
    g1, p1, g2 = EOS["gamma_l"], EOS["pinf_l"], EOS["gamma_g"]
    r1, r2 = 1.0 / (g1 - 1.0), 1.0 / (g2 - 1.0)
    q1 = g1 * p1 / (g1 - 1.0)
    A, E = 3 + ndim, 2 + ndim
    rho = W[0] + W[1]
    v = np.stack([W[2 + j] / rho for j in range(ndim)])
    rhoe = W[E] - 0.5 * sum(W[2 + j] * v[j] for j in range(ndim))
    Gam = r2 + (r1 - r2) * W[A]
    Pi = q1 * W[A]
    p = (rhoe - Pi) / Gam
    c = np.sqrt(np.maximum((Gam + 1.0) * rhoe - Pi, 0.0) / (Gam * Gam * rho))
    u = v[ndim - 1]
    F = W * u
    F[2 + ndim - 1] += p
    F[E] += p * u
    F[A] = 0.0
    return v, p, c, F


def node_rows(rng, Wi, Wi1, ndim, cfl):
    """Kind-2 rows: nodes i and i+1, their fluxes, a high-order flux near
    the central one, and lambda from a CFL number per row."""
    A = 3 + ndim
    vi, pi, ci, Fi = node_data(Wi, ndim)
    vr, pr, cr, Fr = node_data(Wi1, ndim)
    n = pi.size
    smax = np.maximum(np.abs(vi[ndim - 1]) + ci, np.abs(vr[ndim - 1]) + cr)
    lam = cfl / np.maximum(smax, 1e-300)
    G = 0.5 * (Fi + Fr) * (1 + rng.uniform(-1e-3, 1e-3, Fi.shape))
    u = 0.5 * (vi[ndim - 1] + vr[ndim - 1])
    GmA = 0.5 * (Wi1[A] - Wi[A]) * u
    GpA = 0.5 * (Wi[A] - Wi1[A]) * u
    parts = [Wi, vi, pi[None], ci[None], Wi1, vr, pr[None], cr[None], Fi, Fr, G, GmA[None], GpA[None], lam[None]]
    return np.concatenate(parts).T


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_first_order_flux_certification_is_sound_and_live(ndim):
    """The sweeps' route through the flux limiter from node states: the
    first-order HLLC flux in FP32 with running error bounds (star state
    decided only where |s*| exceeds its bound) against the FP64 flux and
    limiter."""
    rng = np.random.default_rng(300 + ndim)
    nf = ndim + 4
    # liveness: smooth neighbours at CFL numbers up to 0.45
    pi = random_primitives(rng, 4000, ndim, pmin=1e3)
    Wi, Wi1 = P.conservative(EOS, *pi), nearby_states(rng, pi)
    cert, exact = check(ndim, 2, node_rows(rng, Wi, Wi1, ndim, rng.uniform(0.02, 0.45, 4000)))
    assert np.all(exact[cert]), "certified a midpoint the FP64 limiter changes"
    assert cert.mean() > 0.98, cert.mean()
    rows = []
    m = 3000
    # unrelated neighbours (water next to air, pressure jumps of nine decades,
    # 30 km/s) at CFL numbers up to 3: many first-order states leave G
    for _ in range(4):
        a, b = random_states(rng, m, ndim, extreme=True), random_states(rng, m, ndim, extreme=True)
        rows.append(node_rows(rng, a, b, ndim, 10.0 ** rng.uniform(-2.0, 0.5, m)))
    # mirrored neighbours: s* = 0, and within 1e-12 .. 1e-3 of it
    for eps in (0.0, 1e-12, 1e-9, 1e-6, 1e-3):
        pa = random_primitives(rng, m, ndim)
        a1r1, a2r2, vel, p, a1 = pa
        vb = [v.copy() for v in vel]
        vb[ndim - 1] = -vel[ndim - 1] * (1 + eps * rng.uniform(-1, 1, m))
        a = P.conservative(EOS, a1r1, a2r2, vel, p, a1)
        b = P.conservative(EOS, a1r1, a2r2, vb, p, a1)
        rows.append(node_rows(rng, a, b, ndim, 10.0 ** rng.uniform(-2.0, 0.5, m)))
    # neighbours next to every threshold
    for which in range(5):
        for d in DELTAS:
            a = random_states(rng, 200, ndim)
            b = place(random_states(rng, 200, ndim), ndim, which, d)
            rows.append(node_rows(rng, a, b, ndim, rng.uniform(0.02, 0.9, 200)))
            rows.append(node_rows(rng, b, a, ndim, rng.uniform(0.02, 0.9, 200)))
    spec = node_rows(rng, random_states(rng, m, ndim), random_states(rng, m, ndim), ndim, rng.uniform(0.02, 1.0, m))
    k = rng.integers(0, m, m // 3)
    vals = np.array([0.0, -0.0, 5e-324, 1e-40, 3e38, 1e200, np.inf, -np.inf, np.nan])
    spec[k, rng.integers(0, spec.shape[1] - 1, k.size)] = vals[rng.integers(0, vals.size, k.size)]
    rows.append(spec)
    rows = np.concatenate(rows)
    assert rows.shape[1] == 2 * (nf + ndim + 2) + 3 * nf + 3
    with np.errstate(all="ignore"):
        cert, exact = check(ndim, 2, rows)
    bad = np.flatnonzero(cert & ~exact)
    assert bad.size == 0, rows[bad[:2]]
    assert (~exact).sum() > 1000
    assert cert.sum() > 1000


@pytest.mark.parametrize("name,make,steps", [
    ("shock_bubble_2d", lambda: P.shock_bubble_2d(256, 128, seed=2), 20),
    ("bubble_collapse_3d", lambda: P.bubble_collapse_3d(32), 5),
])
def test_fp64_sweeps_certify_smooth_and_still_flow(name, make, steps):
    """In the sweeps themselves: on the bubble workloads (still liquid at
    alpha1 = 1 - 1e-6, decayed velocities, smooth flow) no limiter needs its
    FP64 path (`fp64_fallbacks` counts the limiters that ran in FP64), so
    the certification is what the FP64 sweeps run there."""
    pr = make()
    s = wcns.Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", **pr.eos)
    W = torch.from_numpy(pr.W).cuda()
    s.advance_steps(W, steps, cfl=0.5)
    st = s.stats()
    assert st["midpoints"] > 0 and st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    assert st["fp64_fallbacks"] == 0, st
    s.close()


def test_fp64_fallbacks_stay_rare_where_limiters_fire():
    """On the Mach 10 water cylinder the limiters fire, and the FP64 path
    runs only near them: well under 1 % of the midpoints."""
    pr = P.mach10_water_cylinder(288, 192)
    s = wcns.Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision="fp64", **pr.eos)
    W = torch.from_numpy(pr.W).cuda()
    s.advance_steps(W, 100, cfl=0.5)
    st = s.stats()
    assert st["flux_limited"] > 0, st
    assert 0 < st["fp64_fallbacks"] < 0.01 * st["midpoints"], st
    s.close()
