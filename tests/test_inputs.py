"""The seeded workload generators (paper_2102_05287_gb300/problems.py) against
the input recipe they state, on CPU.

Primitive fields are recovered from the conservative states with the
mixture equation of state of Sec. 2 written out here (pressure from rho e,
Gamma = sum alpha_k / (gamma_k - 1), Pi = sum alpha_k gamma_k pinf_k /
(gamma_k - 1)).  The shock of the 2D shock/bubble workload is checked
against the Rankine-Hugoniot jump conditions of the fixed-alpha mixture,
which is how its post-shock state is defined.
"""
import numpy as np
import pytest

from paper_2102_05287_gb300 import problems as P


def primitives(W, eos):
    nd = W.shape[0] - 4
    a1 = W[3 + nd]
    rho = W[0] + W[1]
    vel = [W[2 + j] / rho for j in range(nd)]
    ke = 0.5 * rho * sum(v * v for v in vel)
    G = a1 / (eos["gamma_l"] - 1) + (1 - a1) / (eos["gamma_g"] - 1)
    Pi = a1 * eos["gamma_l"] * eos["pinf_l"] / (eos["gamma_l"] - 1)
    p = (W[2 + nd] - ke - Pi) / G
    return rho, vel, p, a1


def test_water_air_shock_tube_states():
    pr = P.water_air_shock_tube(200)
    rho, (u,), p, a1 = primitives(pr.W, pr.eos)
    x = (np.arange(200) + 0.5) / 200
    left = x < 0.7
    assert pr.eos == {"gamma_g": 1.4, "gamma_l": 4.4, "pinf_l": 6e8}
    assert np.allclose(a1[left], 1 - 1e-6, rtol=0, atol=1e-15) and np.allclose(a1[~left], 1e-6, rtol=1e-12)
    assert np.allclose(pr.W[0][left], (1 - 1e-6) * 1000.0, rtol=1e-14)  # water partial density
    assert np.allclose(pr.W[1][~left], (1 - 1e-6) * 50.0, rtol=1e-14)  # air partial density
    assert np.allclose(p[left], 1e9, rtol=1e-9) and np.allclose(p[~left], 1e5, rtol=1e-9)
    assert np.all(u == 0.0)
    assert pr.bcs == (("transmissive", "transmissive"),) and pr.t_end == 2.4e-4 and pr.cfl == 0.5


def test_shock_bubble_rankine_hugoniot_and_bubble():
    nx, ny = 256, 128
    pr = P.shock_bubble_2d(nx, ny, seed=1)
    eos = pr.eos
    rho, (u, v), p, a1 = primitives(pr.W, eos)
    x = (np.arange(nx) + 0.5) * 2.0 / nx
    assert pr.lo == (0.0, 0.0) and pr.hi == (2.0, 1.0)
    assert pr.bcs == (("transmissive", "transmissive"), ("symmetry", "transmissive"))
    # a row far from the bubble: post-shock for x < 0.6, pre-shock beyond
    j = ny - 1
    post, pre = x < 0.6, (x > 0.6) & (x < 0.7)
    r1, u1, p1 = rho[j, post][0], u[j, post][0], p[j, post][0]
    r0, u0, p0 = rho[j, pre][0], u[j, pre][0], p[j, pre][0]
    assert p1 == pytest.approx(1.9e9, rel=1e-9) and p0 == pytest.approx(1e5, rel=1e-6) and u0 == 0.0
    assert r0 == pytest.approx((1 - 1e-6) * 1000.0 + 1e-6 * 1.0, rel=1e-12)
    # Rankine-Hugoniot for the fixed-alpha mixture (stiffened gas with
    # gbar, pbar of alpha1 = 1 - 1e-6): mass, momentum and energy
    a = 1 - 1e-6
    G = a / (eos["gamma_l"] - 1) + (1 - a) / (eos["gamma_g"] - 1)
    gb = 1 + 1 / G
    pb = a * eos["gamma_l"] * eos["pinf_l"] / (eos["gamma_l"] - 1) * (gb - 1) / gb
    S = r1 * u1 / (r1 - r0)  # shock speed from the mass condition
    assert S > u1 > 0
    assert r1 * (u1 - S) ** 2 + p1 == pytest.approx(r0 * S ** 2 + p0, rel=1e-10)
    e = lambda pp, rr: (pp + gb * pb) / ((gb - 1) * rr)
    assert e(p1, r1) - e(p0, r0) == pytest.approx(0.5 * (p1 + p0) * (1 / r0 - 1 / r1), rel=1e-10)
    assert np.all(v == 0.0)
    # the air bubble: radius 0.2 at (1, 0), perturbed by at most 1e-3; floors 1e-6
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.hypot(X - 1.0, Y)
    # floors 1e-6 (up to the FP64 rounding of 1 - (1 - 1e-6), ~1e-10 relative)
    assert a1.min() >= 1e-6 * (1 - 1e-9) and 1 - a1.max() >= 1e-6 * (1 - 1e-9)
    assert a1[r < 0.15].max() < 1e-5 and a1[(r > 0.25) & (X > 0.6)].min() > 1 - 1e-5
    gas = (1 - a1) > 0.5
    dx = 2.0 / nx
    assert r[gas].max() < 0.2 + 1e-3 + dx and r[~gas & (X > 0.6)].min() > 0.2 - 1e-3 - dx
    assert np.all(p[r < 0.15] == pytest.approx(1e5, rel=1e-6))


def test_bubble_collapse_3d_layout():
    n = 48
    pr = P.bubble_collapse_3d(n=n)
    rho, vel, p, a1 = primitives(pr.W, pr.eos)
    assert pr.W.shape == (7, n, n, n) and pr.lo == (0.0,) * 3 and pr.hi == (1.0,) * 3
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    # seven cells or more from the tanh interface (dx = 1/48) the floors hold
    assert a1[r < 0.1].max() < 1e-5 and a1[r > 0.4].min() > 1 - 1e-5
    assert np.allclose(p[r < 0.2], 1e5, rtol=1e-6) and np.allclose(p[r > 0.3], 1e8, rtol=1e-9)
    gas = (1 - a1) > 0.5
    assert r[gas].max() < 0.25 + 1e-3 + 1.0 / n and r[~gas].min() > 0.25 - 1e-3 - 1.0 / n
    assert all(np.all(vj == 0.0) for vj in vel)


def test_riemann_batch_distributions():
    rb = P.riemann_batch()
    s, prm = rb.sizes, rb.params
    assert len(s) == 4096 and rb.offsets[-1] == s.sum() and rb.W.shape == (5, int(s.sum()))
    assert s.min() >= 128 and s.max() <= 8192
    # log-uniform sizes: the median sits near the geometric mean 1024
    assert 800 < np.median(s) < 1300
    assert prm["ratio"].min() >= 10 and prm["ratio"].max() <= 1e4
    assert 900 <= prm["rho_l"].min() and prm["rho_l"].max() <= 1100
    assert 1 <= prm["rho_g"].min() and prm["rho_g"].max() <= 100
    assert 0.3 <= prm["x0"].min() and prm["x0"].max() <= 0.7
    rho, (u,), p, a1 = primitives(rb.W, rb.eos)
    for k in (0, 1, 2047, 4095):
        sl = slice(int(rb.offsets[k]), int(rb.offsets[k + 1]))
        n = int(s[k])
        x = (np.arange(n) + 0.5) / n
        left = x < prm["x0"][k]
        assert np.allclose(p[sl][left], 1e5 * prm["ratio"][k], rtol=1e-9)
        assert np.allclose(p[sl][~left], 1e5, rtol=1e-9)
        assert np.allclose(rb.W[0][sl][left], (1 - 1e-6) * prm["rho_l"][k], rtol=1e-14)
        assert np.allclose(rb.W[1][sl][~left], (1 - 1e-6) * prm["rho_g"][k], rtol=1e-14)
        assert np.all(u[sl] == 0.0)


def test_smooth_advection_fields():
    pr = P.advection_1d_smooth(64)
    rho, (u,), p, a1 = primitives(pr.W, pr.eos)
    x = (np.arange(64) + 0.5) / 64
    assert np.allclose(a1, 0.5 + 0.25 * np.sin(2 * np.pi * x), rtol=1e-14)
    assert np.allclose(u, 1.0, rtol=1e-14) and np.allclose(p, 1e5, rtol=1e-9)
    assert pr.dt_fixed == pytest.approx(4e-5 / 64, rel=1e-14)
    pr2 = P.advection_2d(16)
    rho, (u, v), p, a1 = primitives(pr2.W, pr2.eos)
    c = -1.0 + (np.arange(16) + 0.5) * 2.0 / 16
    X, Y = np.meshgrid(c, c, indexing="xy")
    assert np.allclose(a1, 0.5 + 0.25 * np.sin(np.pi * (X + Y)), rtol=1e-14)
    assert np.allclose(u, 10.0) and np.allclose(v, 10.0) and np.allclose(p, 101325.0, rtol=1e-9)
