"""ctypes binding of the plain FP64 C++ oracle (oracle/wcns_oracle.cpp).

TEST INFRASTRUCTURE: this module is the parity reference and the timed CPU
baseline.  It is loaded only by tests, the smoke check, the benchmark's
CPU-baseline legs and reference arm, and opcount_table.py; the CUDA library
never imports it.

The oracle follows Wong et al., arXiv 2102.05287: EOS and mixture rules
(Section 2), HLLC (Section 3), HCS + WCNS-IS with characteristic projection
(Section 4, Appendix A), the interpolation and flux limiters (Section 5,
Algorithms 1-6) and SSPRK3 (Section 5.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wcns_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()

BC_TRANSMISSIVE, BC_PERIODIC, BC_SYMMETRY, BC_DIRICHLET = 0, 1, 2, 3
SCHEME_PP_WCNS_IS, SCHEME_HLLC1, SCHEME_WCNS_IS = 0, 1, 2
_BC_NAMES = {"transmissive": 0, "periodic": 1, "symmetry": 2, "dirichlet": 3}
_SCHEMES = {"pp-wcns-is": 0, "hllc1": 1, "wcns-is": 2}


class _Config(C.Structure):
    _fields_ = [
        ("ndim", C.c_int),
        ("n", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("bc", (C.c_int * 2) * 3),
        ("dirichlet", ((C.c_double * 7) * 2) * 3),
        ("gamma_g", C.c_double),
        ("gamma_l", C.c_double),
        ("pinf_l", C.c_double),
        ("scheme", C.c_int),
        ("eps_is", C.c_double),
        ("eps_ar", C.c_double),
        ("eps_a", C.c_double),
        ("eps_rc", C.c_double),
        ("hs_ar", C.c_double),
        ("hs_a", C.c_double),
        ("hs_rc", C.c_double),
        ("dir_face", (C.c_void_p * 2) * 3),
    ]


class OracleStats(C.Structure):
    _fields_ = [
        ("interp_limited", C.c_longlong),
        ("interp_hard", C.c_longlong),
        ("flux_limited", C.c_longlong),
        ("flux_hard", C.c_longlong),
        ("midpoints", C.c_longlong),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _compile(out, extra):
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp] + extra
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)


def build_oracle(force=False):
    """Compile the oracle and its op-counting variant (g++, -O2,
    -ffp-contract=off).  Returns the two library paths."""
    plain = os.path.join(_BUILD, "liboracle.so")
    count = os.path.join(_BUILD, "liboracle_count.so")
    with _LOCK:
        for path, extra in ((plain, []), (count, ["-DORACLE_COUNT_OPS"])):
            stale = (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(_SRC)
            if force or stale:
                _compile(path, extra)
    return plain, count


_LIBS = {}


def _lib(counting=False):
    key = bool(counting)
    if key not in _LIBS:
        plain, count = build_oracle()
        lib = C.CDLL(count if counting else plain)
        P = C.POINTER
        d = C.c_double
        cfgp = P(_Config)
        dp = P(d)
        stp = P(OracleStats)
        lib.oc_rhs.argtypes = [cfgp, dp, dp, d, stp]
        lib.oc_max_wavespeed.argtypes = [cfgp, dp, dp]
        lib.oc_rhs_smax.argtypes = [cfgp, dp, dp, d, dp, stp]
        lib.oc_rk3_step.argtypes = [cfgp, dp, d, stp]
        lib.oc_advance_to.argtypes = [cfgp, dp, d, d, d, d, C.c_long, dp, P(C.c_long), stp]
        lib.oc_thermo.argtypes = [cfgp, dp, dp]
        lib.oc_prim_to_cons.argtypes = [cfgp, dp, dp]
        lib.oc_cons_to_prim.argtypes = [cfgp, dp, dp]
        lib.oc_phys_flux.argtypes = [cfgp, C.c_int, dp, dp]
        lib.oc_hllc.argtypes = [cfgp, C.c_int, dp, dp, dp, dp]
        lib.oc_hllc_star.argtypes = [cfgp, C.c_int, dp, dp, dp, dp, dp]
        lib.oc_char_matrices.argtypes = [cfgp, C.c_int, dp, dp, dp, dp]
        lib.oc_wcnsis_left.argtypes = [dp, d, dp]
        lib.oc_hcs_recon.argtypes = [d, dp]
        lib.oc_hcs_recon.restype = d
        lib.oc_midpoint_flux.argtypes = [cfgp, C.c_int, dp, d, dp, dp, stp]
        lib.oc_interp_limit.argtypes = [cfgp, dp, dp, P(C.c_int)]
        lib.oc_flux_limit.argtypes = [cfgp, C.c_int, dp, dp, dp, dp, d, dp, dp, P(C.c_int)]
        if counting:
            lib.oc_opcount_reset.argtypes = []
            lib.oc_opcount_get.argtypes = [P(C.c_ulonglong)]
            lib.oc_opcount_rows.argtypes = [P(C.c_ulonglong)]
            lib.oc_opcount_rows.restype = C.c_int
        _LIBS[key] = lib
    return _LIBS[key]


def _dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """One problem set-up: grid, boundary conditions, EOS and scheme.

    W arrays are float64 SoA of shape (nf, n_z, n_y, n_x) (leading grid axes
    dropped for lower dimension), x fastest, interior cells only.
    """

    def __init__(self, n, lo, hi, bcs, gamma_g, gamma_l, pinf_l, scheme="pp-wcns-is",
                 eps_is=1e-40, tols=(1e-10, 1e-10, 1e-8), hs_tols=(1e-11, 1e-11, 1e-9),
                 dirichlet=None, dirichlet_face=None, counting=False):
        n = list(n)
        ndim = len(n)
        c = _Config()
        c.ndim = ndim
        for d in range(3):
            c.n[d] = n[d] if d < ndim else 1
            c.lo[d] = lo[d] if d < ndim else 0.0
            c.hi[d] = hi[d] if d < ndim else 1.0
            for s in range(2):
                kind = bcs[d][s] if d < ndim else "transmissive"
                c.bc[d][s] = _BC_NAMES[kind] if isinstance(kind, str) else int(kind)
                if dirichlet is not None and d < ndim and dirichlet[d][s] is not None:
                    for q, v in enumerate(dirichlet[d][s]):
                        c.dirichlet[d][s][q] = float(v)
        # per-face Dirichlet states: {(axis, side): array (nf, face cells)}
        self._faces = {}
        for (d, s), arr in (dirichlet_face or {}).items():
            a = np.ascontiguousarray(arr, dtype=np.float64)
            nface = int(np.prod([n[k] for k in range(ndim) if k != d]))
            assert a.size == (ndim + 4) * nface, (a.shape, nface)
            self._faces[(d, s)] = a
            c.dir_face[d][s] = a.ctypes.data
        c.gamma_g, c.gamma_l, c.pinf_l = float(gamma_g), float(gamma_l), float(pinf_l)
        c.scheme = _SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        c.eps_is = eps_is
        c.eps_ar, c.eps_a, c.eps_rc = tols
        c.hs_ar, c.hs_a, c.hs_rc = hs_tols
        self.cfg = c
        self.ndim = ndim
        self.nf = ndim + 4
        self.n = n
        self.shape = (self.nf,) + tuple(reversed(n))
        self.counting = counting
        self.lib = _lib(counting)
        self.stats = OracleStats()

    # --- whole-grid operations -------------------------------------------
    def _check(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == self.shape, (W.shape, self.shape)
        return W

    def rhs(self, W, dt):
        W = self._check(W)
        out = np.empty_like(W)
        self.lib.oc_rhs(C.byref(self.cfg), _dptr(W), _dptr(out), float(dt), C.byref(self.stats))
        return out

    def rhs_smax(self, W, dt, smax):
        """RHS with sigma_d set from the given maxima of (|u_d| + c)."""
        W = self._check(W)
        out = np.empty_like(W)
        sm = np.ascontiguousarray(np.asarray(smax, dtype=np.float64).reshape(3))
        self.lib.oc_rhs_smax(C.byref(self.cfg), _dptr(W), _dptr(out), float(dt), _dptr(sm),
                             C.byref(self.stats))
        return out

    def max_wavespeed(self, W):
        W = self._check(W)
        out = np.zeros(3)
        self.lib.oc_max_wavespeed(C.byref(self.cfg), _dptr(W), _dptr(out))
        return out

    def rk3_step(self, W, dt):
        W = self._check(W).copy()
        self.lib.oc_rk3_step(C.byref(self.cfg), _dptr(W), float(dt), C.byref(self.stats))
        return W

    def advance_to(self, W, t0, t_end, cfl=0.5, dt_fixed=0.0, max_steps=10**9):
        W = self._check(W).copy()
        t = C.c_double(0.0)
        steps = C.c_long(0)
        self.lib.oc_advance_to(C.byref(self.cfg), _dptr(W), float(t0), float(t_end), float(cfl),
                               float(dt_fixed), int(max_steps), C.byref(t), C.byref(steps),
                               C.byref(self.stats))
        return W, t.value, steps.value

    # --- pointwise helpers used by the pin tests ---------------------------
    def thermo(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros(6)
        self.lib.oc_thermo(C.byref(self.cfg), _dptr(w), _dptr(out))
        return dict(zip(("p", "rho_c2", "rho_ct2", "gamma_bar", "pinf_bar", "c"), out))

    def prim_to_cons(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.nf)
        self.lib.oc_prim_to_cons(C.byref(self.cfg), _dptr(v), _dptr(out))
        return out

    def cons_to_prim(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros(self.nf)
        self.lib.oc_cons_to_prim(C.byref(self.cfg), _dptr(w), _dptr(out))
        return out

    def phys_flux(self, d, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros(self.nf)
        self.lib.oc_phys_flux(C.byref(self.cfg), int(d), _dptr(w), _dptr(out))
        return out

    def hllc(self, d, wl, wr):
        wl = np.ascontiguousarray(wl, dtype=np.float64)
        wr = np.ascontiguousarray(wr, dtype=np.float64)
        g = np.zeros(self.nf)
        us = C.c_double(0.0)
        self.lib.oc_hllc(C.byref(self.cfg), int(d), _dptr(wl), _dptr(wr), _dptr(g), C.byref(us))
        return g, us.value

    def hllc_star(self, d, wl, wr):
        wl = np.ascontiguousarray(wl, dtype=np.float64)
        wr = np.ascontiguousarray(wr, dtype=np.float64)
        s3 = np.zeros(3)
        a = np.zeros(self.nf)
        b = np.zeros(self.nf)
        self.lib.oc_hllc_star(C.byref(self.cfg), int(d), _dptr(wl), _dptr(wr), _dptr(s3), _dptr(a),
                              _dptr(b))
        return s3, a, b

    def char_matrices(self, d, wa, wb):
        wa = np.ascontiguousarray(wa, dtype=np.float64)
        wb = np.ascontiguousarray(wb, dtype=np.float64)
        R = np.zeros((self.nf, self.nf))
        Ri = np.zeros((self.nf, self.nf))
        self.lib.oc_char_matrices(C.byref(self.cfg), int(d), _dptr(wa), _dptr(wb), _dptr(R), _dptr(Ri))
        return R, Ri

    def midpoint_flux(self, d, nodes6, lam):
        nodes6 = np.ascontiguousarray(nodes6, dtype=np.float64)
        assert nodes6.shape == (6, self.nf)
        gm = np.zeros(self.nf)
        gp = np.zeros(self.nf)
        self.lib.oc_midpoint_flux(C.byref(self.cfg), int(d), _dptr(nodes6), float(lam), _dptr(gm),
                                  _dptr(gp), C.byref(self.stats))
        return gm, gp

    def interp_limit(self, wn, wt):
        wn = np.ascontiguousarray(wn, dtype=np.float64)
        wt = np.ascontiguousarray(wt, dtype=np.float64).copy()
        hard = C.c_int(0)
        lim = self.lib.oc_interp_limit(C.byref(self.cfg), _dptr(wn), _dptr(wt), C.byref(hard))
        return wt, bool(lim), bool(hard.value)

    def flux_limit(self, d, wi, wi1, ghm, ghp, lam, gm, gp):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in (wi, wi1, ghm, ghp, gm, gp)]
        hard = C.c_int(0)
        lim = self.lib.oc_flux_limit(C.byref(self.cfg), int(d), *[_dptr(a) for a in arrs[:4]],
                                     float(lam), _dptr(arrs[4]), _dptr(arrs[5]), C.byref(hard))
        return arrs[4], arrs[5], bool(lim), bool(hard.value)

    # --- op counting --------------------------------------------------------
    def opcount_reset(self):
        assert self.counting
        self.lib.oc_opcount_reset()

    def opcount(self):
        assert self.counting
        out = (C.c_ulonglong * 5)()
        self.lib.oc_opcount_get(out)
        return dict(zip(("add", "mul", "div", "sqrt", "minmax"), [int(x) for x in out]))

    # step number -> name of the step of the method the operations belong to
    OPCOUNT_ROWS = {0: "other", 2: "node_eos", 3: "projection", 4: "wcns_is", 5: "back_projection",
                    6: "interp_limiter", 7: "midpoint_hllc", 8: "node_flux", 9: "hcs_split",
                    10: "first_order_hllc", 11: "flux_limiter", 12: "update", 13: "max_wavespeed",
                    14: "ssprk3_combine"}

    def opcount_rows(self):
        """Operation counts since the last reset, per step of the method:
        {step name: {add, mul, div, sqrt, minmax}} (steps with no work left out)."""
        assert self.counting
        out = (C.c_ulonglong * (5 * 16))()
        nrows = self.lib.oc_opcount_rows(out)
        rows = {}
        for r in range(nrows):
            c = dict(zip(("add", "mul", "div", "sqrt", "minmax"), [int(x) for x in out[5 * r:5 * r + 5]]))
            if any(c.values()):
                rows[self.OPCOUNT_ROWS.get(r, "row%d" % r)] = c
        return rows


def wcnsis_left(u5, eps=1e-40):
    """Left-biased IS interpolation at i+1/2 from u_{i-2..i+2} (Section 4.3).
    Returns dict(value, omega[4], beta[5] = (b0, b1, b01, b2, b3), tau5)."""
    u5 = np.ascontiguousarray(u5, dtype=np.float64)
    out = np.zeros(11)
    _lib().oc_wcnsis_left(_dptr(u5), float(eps), _dptr(out))
    return {"value": out[0], "omega": out[1:5].copy(), "beta": out[5:10].copy(), "tau5": out[10]}


def hcs_recon(gt, g6):
    """HCS reconstructed flux at i+1/2 (Section 4.1, psi = 256/175)."""
    g6 = np.ascontiguousarray(g6, dtype=np.float64)
    return _lib().oc_hcs_recon(float(gt), _dptr(g6))
