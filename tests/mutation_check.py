"""Mutation check of the oracle pins (test infrastructure, run by hand).

Each mutant is one plausible mistake in oracle/wcns_oracle.cpp (or in the
exact Riemann solver oracle/exact_riemann.py): a dropped
term, a wrong sign, constant, index or operand order.  For every mutant the
repository is copied to a scratch directory, the mistake is planted in the
copy's oracle (the first occurrence of the pattern: the scheme's own code,
not a helper that restates a formula for a unit test), and
tests/test_oracle_pins.py runs there on the CPU.  A mutant that no pin
fails survives; the check exits non-zero if any mutant survives except
those marked harmless (a reading of the paper under which both forms give
the same result).

    python -m tests.mutation_check [--jobs N]
"""
import argparse
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join("oracle", "wcns_oracle.cpp")
RIEMANN_SRC = os.path.join("oracle", "exact_riemann.py")
SKIP = {".git", "_work", "gpurun_out", "_build", "__pycache__", "profiles", "baseline", ".pytest_cache"}

# (what the mistake is, pattern, replacement, harmless)
MUTANTS = [
    ("mixture Gamma with the liquid constant for the gas", "return a1 * e.r1 + a2 * e.r2;",
     "return a1 * e.r1 + a2 * e.r1;", False),
    ("rho c^2 = gbar (p - pbar)", "t.rho_c2 = gb * (t.p + pb);", "t.rho_c2 = gb * (t.p - pb);", False),
    ("kinetic energy without the 1/2", "t.rhoe = W[E] - 0.5 * ke / t.rho;", "t.rhoe = W[E] - ke / t.rho;", False),
    ("energy flux without the pressure work", "F[E] = (W[E] + t.p) * u;", "F[E] = W[E] * u;", False),
    ("V -> W energy with -Pi", "real rhoe = p * mix_Gamma(e, a1) + mix_Pi(e, a1);",
     "real rhoe = p * mix_Gamma(e, a1) - mix_Pi(e, a1);", False),
    ("HLLC left speed with u_L + c_L", "real sL = o_min(ubar - cbar, uL - tL.c);",
     "real sL = o_min(ubar - cbar, uL + tL.c);", False),
    ("contact speed with the pressure difference reversed", "real num = tR.p - tL.p +", "real num = tL.p - tR.p +",
     False),
    ("left star energy divided by s_L - s*", "tL.p / (sL - uL)));", "tL.p / (sL - ss)));", False),
    ("alpha flux upwinded the wrong way", "G[A] = wl * (WL[A] * ss) + wr * (WR[A] * ss);",
     "G[A] = wl * (WR[A] * ss) + wr * (WL[A] * ss);", False),
    ("R^-1 partial-density row with a2r2", "Rinv[1 * nf + P] = -ar1 / (rho * c * c);",
     "Rinv[1 * nf + P] = -ar2 / (rho * c * c);", False),
    ("midpoint sound speed from the left node only", "real c = 0.5 * (ta.c + tb.c);", "real c = ta.c;", False),
    ("R pressure row with the wrong sign", "R[P * nf + 0] = -rho * c / 2.0;", "R[P * nf + 0] = rho * c / 2.0;", False),
    ("S2 with +u_{i+2}", "s[2] = 0.125 * (3.0 * u0 + 6.0 * up1 - up2);",
     "s[2] = 0.125 * (3.0 * u0 + 6.0 * up1 + up2);", False),
    ("beta01 with 13/3", "real b01 = (13.0 / 12.0)", "real b01 = (13.0 / 3.0)", False),
    ("linear weights d0, d1 swapped", "{15.0 / 32.0, 5.0 / 32.0, 5.0 / 16.0, 1.0 / 16.0}",
     "{5.0 / 32.0, 15.0 / 32.0, 5.0 / 16.0, 1.0 / 16.0}", False),
    ("eta0, eta1 without the tau5/beta01 factor", "eta[k] = d[k] * (1.0 + rk * r01);",
     "eta[k] = d[k] * (1.0 + rk);", False),
    ("tau5 with -3 u_{i+1}", "real t5a = up2 - 4.0 * up1 + 6.0 * u0", "real t5a = up2 - 3.0 * up1 + 6.0 * u0",
     False),
    ("right-biased stencil mirrored about node i", "real sr[5] = {U[5][q], U[4][q], U[3][q], U[2][q], U[1][q]};",
     "real sr[5] = {U[4][q], U[3][q], U[2][q], U[1][q], U[0][q]};", False),
    ("HCS outer coefficient with the wrong sign", "- c3 * (g[0] + g[5]);", "+ c3 * (g[0] + g[5]);", False),
    ("HCS psi = 256/176", "HCS_PSI = 256.0 / 175.0;", "HCS_PSI = 256.0 / 176.0;", False),
    ("u-hat not reconstructed (midpoint value used)", "real uh = hcs_recon(ut, un);", "real uh = ut;", False),
    ("theta without the tolerance", "if (fB < eps) return (fA - eps) / (fA - fB);",
     "if (fB < eps) return fA / (fA - fB);", False),
    ("interpolation limiter with node and interpolant swapped",
     "real th = limiter_theta(Wn[k - 1], Wt[k - 1], cfg.eps_ar);",
     "real th = limiter_theta(Wt[k - 1], Wn[k - 1], cfg.eps_ar);", False),
    ("alpha_2 taken as alpha_1", "return k == 1 ? W[3 + ndim] : 1.0 - W[3 + ndim];", "return W[3 + ndim];", False),
    ("half states without the factor 2", "out[q] = Wi[q] - 2.0 * lam * (Gm[q] - Fi[q]);",
     "out[q] = Wi[q] - lam * (Gm[q] - Fi[q]);", False),
    ("flux-limiter blend skips the alpha component",
     "      for (int q = 0; q < nf; ++q) {\n        Gp[q] = (1.0 - th) * GHp[q] + th * Gp[q];",
     "      for (int q = 0; q < nf - 1; ++q) {\n        Gp[q] = (1.0 - th) * GHp[q] + th * Gp[q];", False),
    ("flux hard switch inspects W_i^+ only", "for (int s = 0; s < 2; ++s) {\n    const real *X = B[s];",
     "for (int s = 0; s < 1; ++s) {\n    const real *X = B[s];", False),
    ("first-order split with the other cell's alpha", "GHm[A] = GH[A] - ni.W[A] * uH;",
     "GHm[A] = GH[A] - ni1.W[A] * uH;", False),
    ("high-order split with the other cell's alpha", "Gm[A] = Gh[A] - ni.W[A] * uh;",
     "Gm[A] = Gh[A] - ni1.W[A] * uh;", False),
    ("node flux G without alpha1 u", "nd.G[3 + ndim] = W[3 + ndim] * nd.un;", "nd.G[3 + ndim] = 0.0;", False),
    ("lambda without sigma_d", "const double sigma = c.ndim == 1 ? 1.0 : tau[d] / tsum;",
     "const double sigma = 1.0;", False),
    ("flux difference with the wrong sign",
     "dWdt[(size_t)q * N + idx] = o_val(dWdt[(size_t)q * N + idx] - upd);",
     "dWdt[(size_t)q * N + idx] = o_val(dWdt[(size_t)q * N + idx] + upd);", False),
    ("SSPRK3 last stage 1/2, 1/2", "W[q] = (1.0 / 3.0) * W0[q] + (2.0 / 3.0) * (W2[q] + dt * L[q]);",
     "W[q] = 0.5 * W0[q] + 0.5 * (W2[q] + dt * L[q]);", False),
    ("wave speed without c", "double s = o_val(o_abs(t.vel[d]) + t.c);", "double s = o_val(o_abs(t.vel[d]));",
     False),
    ("symmetry ghost without the momentum flip", "if (flip) dst[2 + d] = -dst[2 + d];",
     "if (flip) dst[2 + d] = dst[2 + d];", False),
    ("symmetry ghost mirrored about the wrong cell", "src = i < 0 ? -1 - i : 2 * n - 1 - i;",
     "src = i < 0 ? -i : 2 * n - 2 - i;", False),
    ("pressure added to the x momentum flux in every direction", "F[2 + d] = F[2 + d] + t.p;",
     "F[2] = F[2] + t.p;", False),
    ("node normal velocity always u_x", "nd.un = nd.t.vel[d];", "nd.un = nd.t.vel[0];", False),
    ("left star normal momentum always in x", "WsL[2 + d] = chi * (tL.rho * ss);",
     "WsL[2] = chi * (tL.rho * ss);", False),
    ("R^-1 tangential rows pick the normal velocity", "Rinv[row * nf + 2 + j] = 1.0;",
     "Rinv[row * nf + 2 + d] = 1.0;", False),
    ("tau_d from the x wave speed", "tau[d] = smax[d] / spacing(c, d);", "tau[d] = smax[0] / spacing(c, d);",
     False),
    ("cell index with the x extent as every stride", "idx = idx * c.n[d] + ijk[d];",
     "idx = idx * c.n[0] + ijk[d];", False),
    ("R tangential rows write the normal velocity", "R[(2 + j) * nf + row] = 1.0;",
     "R[(2 + d) * nf + row] = 1.0;", False),
    ("momentum fluxes all carry the normal momentum", "for (int j = 0; j < ndim; ++j) F[2 + j] = W[2 + j] * u;",
     "for (int j = 0; j < ndim; ++j) F[2 + j] = W[2 + d] * u;", False),
    ("sign(0) = +1 in the HLLC flux (at s* = 0 both sides give the same flux)", "  if (x > 0.0) return 1.0;",
     "  if (x >= 0.0) return 1.0;", True),
]

# mistakes in the exact two-stiffened-gas Riemann solver (the reference of
# the shock-tube convergence pins)
RIEMANN_MUTANTS = [
    ("shock relation B without pinf", "B = (g - 1.0) / (g + 1.0) * (self.p + pi)",
     "B = (g - 1.0) / (g + 1.0) * self.p", False),
    ("rarefaction exponent (g-1)/g", "e = (g - 1.0) / (2.0 * g)", "e = (g - 1.0) / g", False),
    ("star velocity with the wave functions swapped", "u = 0.5 * (L.u + R.u) + 0.5 * (fr - fl)",
     "u = 0.5 * (L.u + R.u) + 0.5 * (fl - fr)", False),
    ("shock speed with the minus term", "(g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))",
     "(g + 1.0) / (2.0 * g) * ratio - (g - 1.0) / (2.0 * g))", False),
    ("post-shock density ratio with -gm", "rho = s.rho * (ratio + gm) / (gm * ratio + 1.0)",
     "rho = s.rho * (ratio - gm) / (gm * ratio + 1.0)", False),
    ("fan pressure without the -pinf", "p = (s.p + pi) * (c / s.c) ** (2.0 * g / (g - 1.0)) - pi",
     "p = (s.p + pi) * (c / s.c) ** (2.0 * g / (g - 1.0))", False),
    ("mixture pinf = Pi / gbar", "return gb, Pi * (gb - 1.0) / gb", "return gb, Pi / gb", False),
]

ALL = [(SRC,) + m for m in MUTANTS] + [(RIEMANN_SRC,) + m for m in RIEMANN_MUTANTS]


def _copy_repo(dst):
    def ignore(_dir, names):
        return [n for n in names if n in SKIP or n.endswith((".so", ".o"))]
    shutil.copytree(ROOT, dst, ignore=ignore, dirs_exist_ok=True)


def run_mutant(k):
    src_file, what, pattern, replacement, harmless = ALL[k]
    work = tempfile.mkdtemp(prefix="oracle_mutant%02d_" % k)
    try:
        _copy_repo(work)
        path = os.path.join(work, src_file)
        with open(path) as f:
            src = f.read()
        if pattern not in src:
            return k, None, "pattern not found"
        with open(path, "w") as f:
            f.write(src.replace(pattern, replacement, 1))
        try:
            r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"), "-q",
                                "-m", "not gpu", "--tb=no", "-p", "no:cacheprovider"],
                               cwd=work, capture_output=True, text=True, timeout=1200)
        except subprocess.TimeoutExpired:
            return k, None, "timed out"
        failed = sorted(set(re.findall(r"FAILED \S*test_oracle_pins.py::(\w+)", r.stdout)))
        if r.returncode != 0 and not failed:  # the oracle crashed the test process
            failed = ["(pytest exited with status %d)" % r.returncode]
        lines = r.stdout.strip().splitlines()
        return k, failed, lines[-1] if lines else r.stderr[-200:]
    finally:
        shutil.rmtree(work, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, min(6, os.cpu_count() or 1)))
    args = ap.parse_args()
    survivors = []
    with cf.ProcessPoolExecutor(max_workers=args.jobs) as ex:
        for k, failed, summary in ex.map(run_mutant, range(len(ALL))):
            _, what, _, _, harmless = ALL[k]
            caught = bool(failed)
            tag = "killed" if caught else ("harmless" if harmless else "SURVIVED")
            if failed is None:
                tag = "ERROR"
            print("%-8s %-62s %s" % (tag, what, ", ".join(failed or []) or summary), flush=True)
            if not caught and not harmless:
                survivors.append(what)
    print("%d mutants, %d survived" % (len(ALL), len(survivors)))
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
