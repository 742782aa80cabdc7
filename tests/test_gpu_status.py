"""Status codes of the synchronising entry points (Sec. 2 admissible set G).

States are made outside G on the host (a negative partial density, a volume
fraction above one, a NaN) and handed to the library: the kernels run to
completion, count the cells, and wcns_advance_steps, wcns_advance_to,
wcns_advance_steps_host and wcns_batch_advance return WCNS_E_INADMISSIBLE or
WCNS_E_NONFINITE.  No GPU fault is involved; the handle stays usable.
"""
import numpy as np
import pytest

from paper_2102_05287_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300.wcns import (Batch, Solver, WcnsError, WCNS_E_INADMISSIBLE,  # noqa: E402
                                         WCNS_E_NONFINITE)


def _bad_state(kind, W):
    W = W.copy()
    nd = W.ndim - 1
    cell = tuple(s // 2 for s in W.shape[1:])
    if kind == "negative_a2r2":
        W[(1,) + cell] = -1e-3
    elif kind == "alpha1_above_one":
        W[(3 + nd,) + cell] = 1.0 + 1e-3
    elif kind == "nan_energy":
        W[(2 + nd,) + cell] = np.nan
    return W


EXPECTED = {"negative_a2r2": (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE),
            "alpha1_above_one": (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE),
            "nan_energy": (WCNS_E_NONFINITE,)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", sorted(EXPECTED))
def test_advance_steps_reports_states_outside_G(kind, precision):
    pr = P.shock_bubble_2d(64, 32, seed=7)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, precision=precision, **pr.eos)
    W = torch.from_numpy(_bad_state(kind, pr.W)).cuda()
    with pytest.raises(WcnsError) as ei:
        s.advance_steps(W, 1, dt_fixed=1e-9)
    assert ei.value.status in EXPECTED[kind], ei.value.status
    st = s.stats()
    assert st["inadmissible"] > 0 or st["nonfinite"] > 0, st
    # the same handle on an admissible state: OK again (the status is per call)
    W2 = torch.from_numpy(pr.W).cuda()
    s.advance_steps(W2, 2, cfl=0.5)
    s.close()


def test_admissible_states_return_ok_and_count_nothing():
    pr = P.shock_bubble_2d(64, 32, seed=7)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    W = torch.from_numpy(pr.W).cuda()
    t = s.advance_steps(W, 3, cfl=0.5)
    assert t > 0
    st = s.stats()
    assert st["inadmissible"] == 0 and st["nonfinite"] == 0
    s.close()


def test_advance_to_stops_with_the_status():
    pr = P.water_air_shock_tube(200)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    W = torch.from_numpy(_bad_state("negative_a2r2", pr.W)).cuda()
    with pytest.raises(WcnsError) as ei:
        s.advance_to(W, 0.0, pr.t_end, cfl=0.5)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    s.close()


def test_host_buffer_steps_copy_back_and_report():
    pr = P.water_air_shock_tube(200)
    s = Solver(pr.n, pr.lo, pr.hi, pr.bcs, **pr.eos)
    bad = _bad_state("alpha1_above_one", pr.W)
    Wh = torch.from_numpy(bad.copy())
    with pytest.raises(WcnsError) as ei:
        s.advance_steps_host(Wh, 1, dt_fixed=1e-9)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    # the host array holds the device's result, not the untouched input
    assert not np.array_equal(Wh.numpy(), bad)
    s.close()


def test_batch_advance_reports_states_outside_G():
    rb = P.riemann_batch(nprob=16)
    b = Batch(rb.sizes, [0.0] * 16, [1.0] * 16, "transmissive", "transmissive", **rb.eos)
    W = torch.from_numpy(rb.W).cuda()
    b.advance(W, 2, cfl=0.5)  # admissible: OK (tunes on the first call)
    Wb = rb.W.copy()
    Wb[1, int(rb.offsets[3]) + 5] = -1e-3  # a negative gas partial density in problem 3
    W = torch.from_numpy(Wb).cuda()
    with pytest.raises(WcnsError) as ei:
        b.advance(W, 1, cfl=0.5)
    assert ei.value.status in (WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE)
    b.close()
