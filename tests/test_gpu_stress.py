"""The robustness set of Section 6 on the GPU, and the unlimited ablation.

PP-WCNS-IS must keep every state in the admissible set G of Section 2
(device counters and a host check of every cell), in FP64 and in the mixed
path; WCNS-IS with the limiters switched off must leave G on the same
problems, which the device counters report without any fault.  First steps
are compared with the oracle; whole runs are not compared point by point
(hard switches flip on 1-ulp differences), but their density fields must
stay close in L1.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P
from tests.test_oracle_pins import in_G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import (Solver, WcnsError, WCNS_E_INADMISSIBLE,  # noqa: E402
                                         WCNS_E_NONFINITE)
from tests.test_gpu_parity import assert_parity  # noqa: E402

STRESS_1D = ["sedov_multimaterial", "sod_gas_liquid", "interface_advection_1d"]


def _bc_kw(pr):
    if "dirichlet" not in pr.extra:
        return {}
    return dict(dirichlet=pr.extra["dirichlet"], dirichlet_face=pr.extra.get("dirichlet_face"))


def solver(pr, precision="fp64", scheme="pp-wcns-is"):
    return Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, scheme=scheme, **pr.eos, **_bc_kw(pr))


def oracle(pr, scheme="pp-wcns-is"):
    return Oracle(pr.n, pr.lo, pr.hi, pr.bcs, scheme=scheme, **pr.eos, **_bc_kw(pr))


def cfl_dt(o, pr, W, cfl=0.5):
    sm = o.max_wavespeed(W)
    return cfl / sum(sm[d] * pr.n[d] / (pr.hi[d] - pr.lo[d]) for d in range(len(pr.n)))


def rho_l1(a, b):
    ra, rb = a[0] + a[1], b[0] + b[1]
    return float(np.abs(ra - rb).sum() / np.abs(rb).sum())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", STRESS_1D)
def test_pp_full_run_1d_stays_admissible(name, precision):
    pr = getattr(P, name)()
    s = solver(pr, precision)
    W = torch.from_numpy(pr.W).cuda()
    steps = int(round(pr.t_end / pr.dt_fixed))
    s.advance_steps(W, steps, dt_fixed=pr.dt_fixed)
    got = W.cpu().numpy()
    st = s.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    assert in_G(pr.eos, got, 1)
    ref, _, _ = oracle(pr).advance_to(pr.W, 0.0, pr.t_end, dt_fixed=pr.dt_fixed)
    assert rho_l1(got, ref) < 1e-3, rho_l1(got, ref)
    s.close()


@pytest.mark.parametrize("name", STRESS_1D)
def test_unlimited_wcns_is_fails_1d(name):
    pr = getattr(P, name)()
    s = solver(pr, scheme="wcns-is")
    W = torch.from_numpy(pr.W).cuda()
    with pytest.raises(WcnsError) as ei:  # the call reports the state that left G
        s.advance_steps(W, 2, dt_fixed=pr.dt_fixed)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    st = s.stats()
    assert not in_G(pr.eos, W.cpu().numpy(), 1)
    assert st["inadmissible"] > 0 or st["nonfinite"] > 0, st
    s.close()


@pytest.fixture(scope="module")
def mach10():
    return P.mach10_water_cylinder(288, 192)


def test_mach10_first_step_matches_oracle(mach10):
    pr = mach10
    o = oracle(pr)
    s = solver(pr)
    W = torch.from_numpy(pr.W).cuda()
    dt = s.advance_steps(W, 1, cfl=0.5)
    assert abs(dt - cfl_dt(o, pr, pr.W)) <= 1e-14 * dt
    assert_parity(W.cpu().numpy(), o.rk3_step(pr.W, dt), lambda X: o.rk3_step(X, dt), pr.W)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mach10_pp_stays_admissible(mach10, precision):
    pr = mach10
    s = solver(pr, precision)
    W = torch.from_numpy(pr.W).cuda()
    s.advance_steps(W, 300, cfl=0.5)
    st = s.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    assert st["flux_limited"] > 0
    assert in_G(pr.eos, W.cpu().numpy(), 2)
    s.close()


def test_mach10_unlimited_fails():
    """At 144 x 96 the unlimited scheme leaves G in its first step (the
    oracle does the same); at 288 x 192 it survives the first steps."""
    pr = P.mach10_water_cylinder(144, 96)
    s = solver(pr, scheme="wcns-is")
    W = torch.from_numpy(pr.W).cuda()
    with pytest.raises(WcnsError) as ei:
        s.advance_steps(W, 2, cfl=0.5)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    st = s.stats()
    assert not in_G(pr.eos, W.cpu().numpy(), 2)
    assert st["inadmissible"] > 0 or st["nonfinite"] > 0, st
    s.close()


@pytest.fixture(scope="module")
def jet():
    return P.mach100_water_jet(256, 128)


def test_jet_inflow_wavespeed_and_first_step(jet):
    """The inflow's wave speeds set dt.  Its sound speed is ill-conditioned:
    the kinetic energy of the jet is ~3e4 times its internal energy, so
    rho e = E - |m|^2/(2 rho) loses ~4.5 digits and c agrees to ~1e-11 only
    (the same holds for any two correct FP64 evaluations)."""
    pr = jet
    o = oracle(pr)
    s = solver(pr)
    W = torch.from_numpy(pr.W).cuda()
    ref_sm = o.max_wavespeed(pr.W)
    got_sm = s.max_wavespeed(W)
    np.testing.assert_allclose(got_sm[:2], ref_sm[:2], rtol=1e-9)
    assert got_sm[0] > 1.5e5
    dt = s.advance_steps(W, 1, cfl=0.5)
    assert abs(dt - cfl_dt(o, pr, pr.W)) <= 1e-9 * dt
    assert_parity(W.cpu().numpy(), o.rk3_step(pr.W, dt), lambda X: o.rk3_step(X, dt), pr.W)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_jet_pp_stays_admissible(jet, precision):
    pr = jet
    s = solver(pr, precision)
    W = torch.from_numpy(pr.W).cuda()
    s.advance_steps(W, 400, cfl=0.5)
    st = s.stats()
    assert st["nonfinite"] == 0 and st["inadmissible"] == 0, st
    got = W.cpu().numpy()
    assert in_G(pr.eos, got, 2)
    assert got[0].max() > 100.0  # the jet has entered
    s.close()


def test_unlimited_blow_up_is_reported_not_faulted():
    """Failure detection on the host side of the ABI: the unlimited scheme
    drives the Sedov state out of G and then to non-finite values;
    wcns_advance_to stops at its first check after that with
    WCNS_E_INADMISSIBLE or WCNS_E_NONFINITE (it does not report reaching
    t_end), and the handle stays usable afterwards."""
    pr = P.sedov_multimaterial()
    s = solver(pr, scheme="wcns-is")
    W = torch.from_numpy(pr.W).cuda()
    with pytest.raises(WcnsError) as ei:
        s.advance_to(W, 0.0, pr.t_end, cfl=0.5)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    st = s.stats()
    assert st["nonfinite"] > 0 or st["inadmissible"] > 0
    ok = solver(pr)
    W2 = torch.from_numpy(pr.W).cuda()
    t, steps = ok.advance_to(W2, 0.0, 50 * pr.dt_fixed, cfl=0.5)
    assert t == 50 * pr.dt_fixed and steps > 0
    assert in_G(pr.eos, W2.cpu().numpy(), 1)
    s.close()
    ok.close()


def test_invalid_arguments_are_rejected():
    with pytest.raises(WcnsError):  # gamma_g > gamma_l breaks Lemma 1's convexity
        Solver((16,), (0.0,), (1.0,), (("transmissive", "transmissive"),), gamma_g=5.0, gamma_l=4.4,
               pinf_l=6e8)
    s = Solver((16, 8), (0.0, 0.0), (1.0, 1.0), (("transmissive", "transmissive"),) * 2, **P.WORKLOAD_EOS)
    with pytest.raises(WcnsError):  # the face is not a Dirichlet face
        s.set_dirichlet_face(0, 0, np.zeros((6, 8)))
    with pytest.raises(ValueError):  # wrong face size
        s.set_dirichlet_face(0, 0, np.zeros((6, 9)))
    s.close()
    with pytest.raises(WcnsError):  # tolerances must be finite and >= 0
        Solver((16,), (0.0,), (1.0,), (("transmissive", "transmissive"),), hs_tols=(-1e-11, 1e-11, 1e-9),
               **P.WORKLOAD_EOS)
