"""Thin ctypes binding of libwcns (include/wcns.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Functions keep the C names; ``Solver`` and ``Batch`` wrap a handle
for torch CUDA tensors (device memory and streams come from PyTorch).
If the library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwcns.so")

WCNS_OK, WCNS_E_INVALID_ARG, WCNS_E_CUDA, WCNS_E_INADMISSIBLE, WCNS_E_NONFINITE = range(5)
WCNS_E_UNSUPPORTED, WCNS_E_TOO_LARGE = 6, 7
WCNS_BC_TRANSMISSIVE, WCNS_BC_PERIODIC, WCNS_BC_SYMMETRY, WCNS_BC_DIRICHLET = range(4)
WCNS_FP64, WCNS_MIXED = 0, 1
WCNS_SCHEME_PP_WCNS_IS, WCNS_SCHEME_HLLC1, WCNS_SCHEME_WCNS_IS = 0, 1, 2
_BC = {"transmissive": 0, "periodic": 1, "symmetry": 2, "dirichlet": 3}
_SCHEME = {"pp-wcns-is": 0, "hllc1": 1, "wcns-is": 2}
_PREC = {"fp64": 0, "mixed": 1}

# Every entry point declared in include/wcns.h.
EXPORTS = [
    "wcns_create", "wcns_default_options", "wcns_set_options", "wcns_get_options", "wcns_set_dirichlet_face", "wcns_rhs",
    "wcns_max_wavespeed", "wcns_rk3_step", "wcns_set_stage_trace", "wcns_advance_steps", "wcns_advance_to",
    "wcns_advance_steps_host", "wcns_get_stats", "wcns_reset_stats", "wcns_nfields", "wcns_ncells",
    "wcns_launch_count", "wcns_rk3_step_noalloc", "wcns_profile_enable", "wcns_profile_read", "wcns_strerror", "wcns_destroy", "wcns_batch_create", "wcns_batch_set_options",
    "wcns_batch_advance", "wcns_batch_tuning", "wcns_batch_get_stats", "wcns_batch_total_cells", "wcns_batch_launch_count",
    "wcns_batch_destroy", "wcns_batch_create_grids", "wcns_check_division", "wcns_check_limiter_cert",
]


class wcns_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class wcns_bcs(C.Structure):
    _fields_ = [("kind", (C.c_int * 2) * 3), ("dirichlet", ((C.c_double * 7) * 2) * 3)]


class wcns_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("scheme", C.c_int), ("eps_is", C.c_double),
                ("eps_ar", C.c_double), ("eps_a", C.c_double), ("eps_rc", C.c_double),
                ("hs_ar", C.c_double), ("hs_a", C.c_double), ("hs_rc", C.c_double),
                ("stream", C.c_void_p)]


class wcns_stats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in ("interp_limited", "interp_hard", "flux_limited", "flux_hard",
                                            "nonfinite", "inadmissible", "midpoints", "fp64_fallbacks")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class wcns_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong * 3), ("ms", C.c_double * 3), ("dropped", C.c_longlong)]


class WcnsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, _strerror(status), status))


_lib = None


def load(path=LIB_PATH):
    """Load libwcns.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libwcns.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = C.CDLL(path)
    P, vp, d, i, ll = C.POINTER, C.c_void_p, C.c_double, C.c_int, C.c_longlong
    sig = {
        "wcns_create": ([P(wcns_grid), P(wcns_bcs), d, d, d, P(vp)], i),
        "wcns_default_options": ([P(wcns_options)], None),
        "wcns_set_options": ([vp, P(wcns_options)], i),
        "wcns_get_options": ([vp, P(wcns_options)], i),
        "wcns_set_dirichlet_face": ([vp, i, i, vp], i),
        "wcns_rhs": ([vp, vp, vp, d], i),
        "wcns_max_wavespeed": ([vp, vp, P(d)], i),
        "wcns_rk3_step": ([vp, vp, d], i),
        "wcns_set_stage_trace": ([vp, vp, vp], i),
        "wcns_advance_steps": ([vp, vp, i, d, d, P(d)], i),
        "wcns_advance_to": ([vp, vp, d, d, d, P(d), P(C.c_long)], i),
        "wcns_advance_steps_host": ([vp, vp, i, d, d, P(d)], i),
        "wcns_get_stats": ([vp, P(wcns_stats)], i),
        "wcns_reset_stats": ([vp], i),
        "wcns_nfields": ([vp], i),
        "wcns_ncells": ([vp], ll),
        "wcns_launch_count": ([vp], ll),
        "wcns_rk3_step_noalloc": ([P(wcns_grid), P(wcns_bcs), d, d, d, P(wcns_options), vp, d], i),
        "wcns_profile_enable": ([vp, i], i),
        "wcns_profile_read": ([vp, P(wcns_profile)], i),
        "wcns_strerror": ([i], C.c_char_p),
        "wcns_destroy": ([vp], None),
        "wcns_batch_create": ([i, P(i), P(d), P(d), i, i, d, d, d, P(vp)], i),
        "wcns_batch_set_options": ([vp, P(wcns_options)], i),
        "wcns_batch_advance": ([vp, vp, i, d, vp], i),
        "wcns_batch_tuning": ([vp, P(i), P(i)], i),
        "wcns_batch_get_stats": ([vp, P(wcns_stats)], i),
        "wcns_batch_total_cells": ([vp], ll),
        "wcns_batch_launch_count": ([vp], ll),
        "wcns_batch_destroy": ([vp], None),
        "wcns_batch_create_grids": ([i, i, P(i), P(d), P(d), P(wcns_bcs), d, d, d, P(vp)], i),
        "wcns_check_division": ([vp, vp, vp, ll, vp], i),
        "wcns_check_limiter_cert": ([i, i, vp, ll, d, d, d, d, d, d, vp, vp, vp], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _strerror(status):
    try:
        return load().wcns_strerror(int(status)).decode()
    except Exception:  # library itself unavailable
        return "status %d" % status


def _check(status, where):
    if status != WCNS_OK:
        raise WcnsError(status, where)


# --- C-named wrappers (marshalling only) -----------------------------------
def wcns_default_options():
    o = wcns_options()
    load().wcns_default_options(C.byref(o))
    return o


def wcns_create(grid, bcs, gamma_g, gamma_l, pinf_l):
    h = C.c_void_p()
    _check(load().wcns_create(C.byref(grid), C.byref(bcs), gamma_g, gamma_l, pinf_l, C.byref(h)),
           "wcns_create")
    return h


def wcns_destroy(h):
    load().wcns_destroy(h)


def _ptr(t):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Solver:
    """A wcns handle for one grid.  W tensors: float64 CUDA, shape
    (nf, [n_z,] [n_y,] n_x), contiguous."""

    def __init__(self, n, lo, hi, bcs, gamma_g, gamma_l, pinf_l, precision="fp64", scheme="pp-wcns-is",
                 eps_is=1e-40, tols=(1e-10, 1e-10, 1e-8), hs_tols=(1e-11, 1e-11, 1e-9), dirichlet=None,
                 dirichlet_face=None, stream=None):
        import torch
        lib = load()
        self.lib = lib
        n = list(n)
        self.ndim = len(n)
        self.nf = self.ndim + 4
        self.shape = (self.nf,) + tuple(reversed(n))
        g = wcns_grid()
        g.ndim = self.ndim
        for d in range(3):
            g.n[d] = n[d] if d < self.ndim else 1
            g.lo[d] = lo[d] if d < self.ndim else 0.0
            g.hi[d] = hi[d] if d < self.ndim else 1.0
        b = wcns_bcs()
        for d in range(self.ndim):
            for s in range(2):
                k = bcs[d][s]
                b.kind[d][s] = _BC[k] if isinstance(k, str) else int(k)
                if dirichlet is not None and dirichlet[d][s] is not None:
                    for q, v in enumerate(dirichlet[d][s]):
                        b.dirichlet[d][s][q] = float(v)
        self.h = wcns_create(g, b, gamma_g, gamma_l, pinf_l)
        o = wcns_default_options()
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.scheme = _SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        o.eps_is = eps_is
        o.eps_ar, o.eps_a, o.eps_rc = tols
        o.hs_ar, o.hs_a, o.hs_rc = hs_tols
        if stream is None:
            stream = torch.cuda.current_stream()
        o.stream = C.c_void_p(stream.cuda_stream)
        self.stream = stream
        _check(lib.wcns_set_options(self.h, C.byref(o)), "wcns_set_options")
        self.options = o
        for (d, s), arr in (dirichlet_face or {}).items():
            self.set_dirichlet_face(d, s, arr)

    def set_dirichlet_face(self, axis, side, W_face):
        """Per-face Dirichlet states: W_face array-like (nf, face cells) of
        conservative states, or None to return to the uniform state."""
        import numpy as np
        if W_face is None:
            _check(self.lib.wcns_set_dirichlet_face(self.h, int(axis), int(side), None), "wcns_set_dirichlet_face")
            return
        a = np.ascontiguousarray(W_face, dtype=np.float64)
        nface = 1
        for k in range(self.ndim):
            if k != axis:
                nface *= self.shape[self.ndim - k]
        if a.size != self.nf * nface:
            raise ValueError("face array of %d values, expected %d" % (a.size, self.nf * nface))
        _check(self.lib.wcns_set_dirichlet_face(self.h, int(axis), int(side), C.c_void_p(a.ctypes.data)),
               "wcns_set_dirichlet_face")

    def close(self):
        if getattr(self, "h", None):
            self.lib.wcns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _w(self, W):
        if tuple(W.shape) != self.shape:
            raise ValueError("state shape %s, expected %s" % (tuple(W.shape), self.shape))
        return _ptr(W)

    def rhs(self, W, dt, out=None):
        import torch
        if out is None:
            out = torch.empty_like(W)
        _check(self.lib.wcns_rhs(self.h, self._w(W), self._w(out), float(dt)), "wcns_rhs")
        return out

    def max_wavespeed(self, W):
        out = (C.c_double * 3)()
        _check(self.lib.wcns_max_wavespeed(self.h, self._w(W), out), "wcns_max_wavespeed")
        return [out[0], out[1], out[2]]

    def rk3_step(self, W, dt):
        _check(self.lib.wcns_rk3_step(self.h, self._w(W), float(dt)), "wcns_rk3_step")
        return W

    def set_stage_trace(self, W1=None, W2=None):
        """Copy the two intermediate SSPRK3 stage states of every step into
        W1, W2 (CUDA tensors shaped like the state); None, None stops."""
        self._trace = (W1, W2)  # keep the buffers alive while traced
        _check(self.lib.wcns_set_stage_trace(self.h, self._w(W1) if W1 is not None else None,
                                             self._w(W2) if W2 is not None else None), "wcns_set_stage_trace")

    def advance_steps(self, W, nsteps, cfl=0.5, dt_fixed=0.0, t=0.0):
        tt = C.c_double(t)
        _check(self.lib.wcns_advance_steps(self.h, self._w(W), int(nsteps), float(cfl), float(dt_fixed),
                                           C.byref(tt)), "wcns_advance_steps")
        return tt.value

    def advance_to(self, W, t0, t_end, cfl=0.5):
        t = C.c_double(0.0)
        steps = C.c_long(0)
        _check(self.lib.wcns_advance_to(self.h, self._w(W), float(t0), float(t_end), float(cfl), C.byref(t),
                                        C.byref(steps)), "wcns_advance_to")
        return t.value, steps.value

    def advance_steps_host(self, W_host, nsteps, cfl=0.5, dt_fixed=0.0, t=0.0):
        """W_host: contiguous float64 CPU tensor (pinned or not), updated in place."""
        if W_host.is_cuda or not W_host.is_contiguous() or tuple(W_host.shape) != self.shape:
            raise ValueError("expected a contiguous float64 CPU tensor of shape %s" % (self.shape,))
        tt = C.c_double(t)
        _check(self.lib.wcns_advance_steps_host(self.h, C.c_void_p(W_host.data_ptr()), int(nsteps),
                                                float(cfl), float(dt_fixed), C.byref(tt)),
               "wcns_advance_steps_host")
        return tt.value

    def stats(self):
        s = wcns_stats()
        _check(self.lib.wcns_get_stats(self.h, C.byref(s)), "wcns_get_stats")
        return s.as_dict()

    def reset_stats(self):
        _check(self.lib.wcns_reset_stats(self.h), "wcns_reset_stats")

    def launches(self):
        return int(self.lib.wcns_launch_count(self.h))

    def profile_enable(self, capacity=4096):
        _check(self.lib.wcns_profile_enable(self.h, int(capacity)), "wcns_profile_enable")

    def profile_read(self):
        p = wcns_profile()
        _check(self.lib.wcns_profile_read(self.h, C.byref(p)), "wcns_profile_read")
        return {"launches": list(p.launches), "ms": list(p.ms), "dropped": int(p.dropped)}


class Batch:
    """Many independent problems advanced together.  1D (the default form):
    Batch(ncells, lo, hi, bc_lo, bc_hi, ...), packed SoA (5, total).  Any
    dimension: Batch.grids(n, lo, hi, bcs, ...) with n, lo, hi of shape
    (nprob, ndim) (x first) and one boundary set for all problems, packed SoA
    (ndim + 4, total), each problem x fastest."""

    def __init__(self, ncells, lo, hi, bc_lo, bc_hi, gamma_g, gamma_l, pinf_l, precision="fp64",
                 scheme="pp-wcns-is", stream=None, _handle=None, _nf=5):
        lib = load()
        self.lib = lib
        nprob = len(ncells)
        self.nprob = nprob
        self.nf = _nf
        if _handle is None:
            nc = (C.c_int * nprob)(*[int(x) for x in ncells])
            lo_ = (C.c_double * nprob)(*[float(x) for x in lo])
            hi_ = (C.c_double * nprob)(*[float(x) for x in hi])
            h = C.c_void_p()
            _check(lib.wcns_batch_create(nprob, nc, lo_, hi_, _BC[bc_lo] if isinstance(bc_lo, str) else bc_lo,
                                         _BC[bc_hi] if isinstance(bc_hi, str) else bc_hi, gamma_g, gamma_l,
                                         pinf_l, C.byref(h)), "wcns_batch_create")
        else:
            h = _handle
        self.h = h
        self._configure(precision, scheme, stream)

    @classmethod
    def grids(cls, n, lo, hi, bcs, gamma_g, gamma_l, pinf_l, precision="fp64", scheme="pp-wcns-is",
              stream=None):
        import numpy as np
        n = np.asarray(n, dtype=np.int64)
        nprob, ndim = n.shape
        lo = np.asarray(lo, dtype=np.float64).reshape(nprob, ndim)
        hi = np.asarray(hi, dtype=np.float64).reshape(nprob, ndim)
        b = wcns_bcs()
        for d in range(ndim):
            for s in range(2):
                k = bcs[d][s]
                b.kind[d][s] = _BC[k] if isinstance(k, str) else int(k)
        n_ = (C.c_int * (nprob * ndim))(*[int(x) for x in n.ravel()])
        lo_ = (C.c_double * (nprob * ndim))(*[float(x) for x in lo.ravel()])
        hi_ = (C.c_double * (nprob * ndim))(*[float(x) for x in hi.ravel()])
        h = C.c_void_p()
        _check(load().wcns_batch_create_grids(int(ndim), int(nprob), n_, lo_, hi_, C.byref(b), gamma_g, gamma_l,
                                              pinf_l, C.byref(h)), "wcns_batch_create_grids")
        return cls([0] * nprob, None, None, None, None, gamma_g, gamma_l, pinf_l, precision=precision,
                   scheme=scheme, stream=stream, _handle=h, _nf=ndim + 4)

    def _configure(self, precision, scheme, stream):
        import torch
        lib, h = self.lib, self.h
        o = wcns_default_options()
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.scheme = _SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        if stream is None:
            stream = torch.cuda.current_stream()
        o.stream = C.c_void_p(stream.cuda_stream)
        self.stream = stream
        _check(lib.wcns_batch_set_options(h, C.byref(o)), "wcns_batch_set_options")
        self.total = int(lib.wcns_batch_total_cells(h))

    def advance(self, W, nsteps, cfl=0.5, t=None):
        if tuple(W.shape) != (self.nf, self.total):
            raise ValueError("packed state must have shape (%d, %d)" % (self.nf, self.total))
        if t is not None and tuple(t.shape) != (self.nprob,):
            raise ValueError("t must have shape (%d,): one time per problem" % self.nprob)
        tp = _ptr(t) if t is not None else None
        _check(self.lib.wcns_batch_advance(self.h, _ptr(W), int(nsteps), float(cfl), tp), "wcns_batch_advance")
        return W

    def stats(self):
        s = wcns_stats()
        _check(self.lib.wcns_batch_get_stats(self.h, C.byref(s)), "wcns_batch_get_stats")
        return s.as_dict()

    def launches(self):
        return int(self.lib.wcns_batch_launch_count(self.h))

    def tuning(self):
        tc, g = C.c_int(0), C.c_int(0)
        st = self.lib.wcns_batch_tuning(self.h, C.byref(tc), C.byref(g))
        return {"tile_cells": tc.value, "grid": g.value} if st == WCNS_OK else None

    def close(self):
        if getattr(self, "h", None):
            self.lib.wcns_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
