"""The FP64 sweeps' division routine against CUDA's IEEE division.

The FP64 sweeps divide with their own routine (an FP32 reciprocal seed, one
Newton-Raphson step and one remainder correction, after Markstein 1990),
which uses fewer FP64-pipe operations than the IEEE division.  Called
through the C ABI (wcns_check_division) on operands spread over the whole
FP64 range, it must be within one unit in the last place of torch's CUDA
division (IEEE round-to-nearest) for every finite, normal quotient, and
equal it on the special operands (zeros, infinities, NaNs, subnormals),
which the routine hands to the IEEE division.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_05287_gb300 import wcns  # noqa: E402


def gpu_div(a, b):
    lib = wcns.load()
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    q = torch.empty_like(ta)
    st = lib.wcns_check_division(C.c_void_p(ta.data_ptr()), C.c_void_p(tb.data_ptr()), C.c_void_p(q.data_ptr()),
                                 a.size, None)
    assert st == wcns.WCNS_OK
    ieee = (ta / tb).cpu().numpy()
    torch.cuda.synchronize()
    return q.cpu().numpy(), ieee


def ulp_distance(x, y):
    """Distance in units in the last place between finite doubles of the
    same sign (lexicographic order of the bit patterns)."""
    xi, yi = x.view(np.int64), y.view(np.int64)
    xi = np.where(xi < 0, np.int64(-0x8000000000000000) - xi, xi)
    yi = np.where(yi < 0, np.int64(-0x8000000000000000) - yi, yi)
    return np.abs(xi - yi)


def test_division_within_one_ulp_over_the_fp64_range():
    rng = np.random.default_rng(2102)
    n = 1 << 21
    a = np.exp(rng.uniform(-690.0, 690.0, n)) * rng.choice([-1.0, 1.0], n)
    b = np.exp(rng.uniform(-690.0, 690.0, n)) * rng.choice([-1.0, 1.0], n)
    # operand shapes of the sweeps: quotients of comparable magnitudes
    m = n // 2
    b[:m] = a[:m] * np.exp(rng.uniform(-40.0, 40.0, m))
    q, ieee = gpu_div(a, b)
    fin = np.isfinite(ieee) & (np.abs(ieee) >= np.finfo(np.float64).tiny)
    d = ulp_distance(q[fin], ieee[fin])
    assert d.max() <= 1, d.max()
    exact = (d == 0).mean()
    print("division routine: %.4f of %d quotients correctly rounded, the rest within 1 ulp" % (exact, fin.sum()))
    assert exact > 0.99
    # quotients that overflow or underflow: the IEEE result (the routine defers or agrees)
    out = ~fin
    assert np.array_equal(np.isinf(q[out]), np.isinf(ieee[out]))
    tiny = out & np.isfinite(ieee)
    assert np.all(np.abs(q[tiny] - ieee[tiny]) <= 2 * np.finfo(np.float64).smallest_subnormal)


def test_division_special_operands():
    sub = 5e-324
    vals = np.array([0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0, np.inf, -np.inf, np.nan, sub, -sub, 1e-310,
                     np.finfo(np.float64).max, np.finfo(np.float64).tiny, 1e300, 1e-300, 7.0 / 3.0])
    a, b = np.meshgrid(vals, vals, indexing="ij")
    a, b = a.ravel().copy(), b.ravel().copy()
    q, ieee = gpu_div(a, b)
    both_nan = np.isnan(q) & np.isnan(ieee)
    same = (q == ieee) & (np.signbit(q) == np.signbit(ieee))
    close = np.isfinite(ieee) & np.isfinite(q) & (ulp_distance(q, ieee) <= 1)
    assert np.all(both_nan | same | close), [(x, y, z, w) for x, y, z, w in zip(a, b, q, ieee)
                                             if not ((np.isnan(z) and np.isnan(w)) or z == w)][:8]
