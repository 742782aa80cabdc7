"""Exact Riemann solver for two stiffened gases (test asset).

TEST INFRASTRUCTURE.  Written from textbook gas-dynamics theory, not from the
paper: inside each constant state of a five-equation Riemann problem the
volume fraction is fixed, so the mixture is itself a stiffened gas with
parameters (gamma_bar(alpha1), pinf_bar(alpha1)) (Wong et al., Section 2),
and alpha1 and the mass fractions only jump at the contact.  The solution is
the classical exact solver with p replaced by p + pinf in the shock
(Rankine-Hugoniot) and rarefaction (isentrope) relations, a Newton/bisection
solve for the star pressure, and sampling in x/t.
"""
from __future__ import annotations

import math

import numpy as np


class Side:
    def __init__(self, rho, u, p, gamma, pinf):
        self.rho, self.u, self.p, self.g, self.pi = float(rho), float(u), float(p), float(gamma), float(pinf)
        self.c = math.sqrt(self.g * (self.p + self.pi) / self.rho)

    def f(self, p):
        """Velocity change across the left/right wave as a function of the
        star pressure, and its derivative."""
        g, pi = self.g, self.pi
        if p > self.p:  # shock
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * (self.p + pi)
            q = math.sqrt(A / (p + pi + B))
            return (p - self.p) * q, q * (1.0 - 0.5 * (p - self.p) / (p + pi + B))
        r = (p + pi) / (self.p + pi)
        e = (g - 1.0) / (2.0 * g)
        return (2.0 * self.c / (g - 1.0)) * (r ** e - 1.0), (1.0 / (self.rho * self.c)) * r ** (-(g + 1.0) / (2.0 * g))


def star_state(L: Side, R: Side, tol=1e-14, maxit=200):
    """Star pressure and velocity."""
    du = R.u - L.u
    pmin = -min(L.pi, R.pi) * (1.0 - 1e-15) + 1e-300
    lo = pmin + 1e-12 * max(1.0, abs(pmin))
    hi = max(L.p, R.p, 1.0) * 10.0
    def F(p):
        fl, dl = L.f(p)
        fr, dr = R.f(p)
        return fl + fr + du, dl + dr
    while F(hi)[0] < 0:
        hi *= 10.0
    if F(lo)[0] > 0:
        raise ValueError("vacuum generated: no positive star pressure")
    p = 0.5 * (L.p + R.p)
    if not (lo < p < hi):
        p = 0.5 * (lo + hi)
    for _ in range(maxit):
        val, der = F(p)
        if val > 0:
            hi = p
        else:
            lo = p
        pn = p - val / der
        if not (lo < pn < hi):
            pn = 0.5 * (lo + hi)
        if abs(pn - p) <= tol * max(abs(p), 1.0):
            p = pn
            break
        p = pn
    fl, _ = L.f(p)
    fr, _ = R.f(p)
    u = 0.5 * (L.u + R.u) + 0.5 * (fr - fl)
    return p, u


def sample(L: Side, R: Side, pstar, ustar, xi):
    """(rho, u, p, side) at similarity coordinate xi = (x - x0)/t; side = 0
    (left material) or 1 (right material)."""
    if xi <= ustar:
        s, sgn, side = L, 1.0, 0
    else:
        s, sgn, side = R, -1.0, 1
    g, pi = s.g, s.pi
    # Work in the frame where the wave is on the "left": mirror the right side.
    u, xr, us = sgn * s.u, sgn * xi, sgn * ustar
    ratio = (pstar + pi) / (s.p + pi)
    if pstar > s.p:  # shock
        S = u - s.c * math.sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))
        if xr < S:
            return s.rho, s.u, s.p, side
        gm = (g - 1.0) / (g + 1.0)
        rho = s.rho * (ratio + gm) / (gm * ratio + 1.0)
        return rho, ustar, pstar, side
    # rarefaction
    cst = s.c * ratio ** ((g - 1.0) / (2.0 * g))
    head, tail = u - s.c, us - cst
    if xr < head:
        return s.rho, s.u, s.p, side
    if xr > tail:
        return s.rho * ratio ** (1.0 / g), ustar, pstar, side
    c = 2.0 / (g + 1.0) * (s.c + 0.5 * (g - 1.0) * (u - xr))
    uu = 2.0 / (g + 1.0) * (s.c + 0.5 * (g - 1.0) * u + xr)
    rho = s.rho * (c / s.c) ** (2.0 / (g - 1.0))
    p = (s.p + pi) * (c / s.c) ** (2.0 * g / (g - 1.0)) - pi
    return rho, sgn * uu, p, side


def mixture(eos, alpha1):
    g1, p1, g2 = eos["gamma_l"], eos["pinf_l"], eos["gamma_g"]
    G = alpha1 / (g1 - 1.0) + (1.0 - alpha1) / (g2 - 1.0)
    Pi = alpha1 * g1 * p1 / (g1 - 1.0)
    gb = 1.0 + 1.0 / G
    return gb, Pi * (gb - 1.0) / gb


def solve_five_equation(eos, left, right, x0, t, x):
    """Exact solution of a 1D five-equation Riemann problem.

    left/right = (a1r1, a2r2, u, p, alpha1).  Returns the conservative SoA
    array (5, len(x)) at time t on the points x."""
    out = np.zeros((5, len(x)))
    sides = []
    for st in (left, right):
        a1r1, a2r2, u, p, a1 = st
        gb, pb = mixture(eos, a1)
        rho = a1r1 + a2r2
        sides.append((Side(rho, u, p, gb, pb), a1r1 / rho, a1))
    L, R = sides[0][0], sides[1][0]
    ps, us = star_state(L, R)
    g1, p1, g2 = eos["gamma_l"], eos["pinf_l"], eos["gamma_g"]
    for i, xx in enumerate(x):
        rho, u, p, side = sample(L, R, ps, us, (xx - x0) / t) if t > 0 else (
            (L.rho, L.u, L.p, 0) if xx < x0 else (R.rho, R.u, R.p, 1))
        _, Y1, a1 = sides[side]
        rhoe = p * (a1 / (g1 - 1.0) + (1 - a1) / (g2 - 1.0)) + a1 * g1 * p1 / (g1 - 1.0)
        out[:, i] = (Y1 * rho, (1 - Y1) * rho, rho * u, rhoe + 0.5 * rho * u * u, a1)
    return out, (ps, us)
