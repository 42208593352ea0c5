"""Python binding of the swedg C ABI (include/swedg.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. PyTorch provides device memory and streams. There is no CPU
fallback; if the library cannot be built or loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_GEOM, ERR_NEG_MEAN, ERR_NONFINITE, ERR_CUDA = 0, -1, -2, -3, -4, -5
KERNEL_CLASSES = {"volume": 0, "face": 1, "prim": 2, "av": 3, "visc_face": 4, "update": 5, "dt": 6,
                  "reduce": 7, "adjoint": 8, "adjoint_volume": 9}

SYMBOLS = ["swe_create", "swe_destroy", "swe_rhs", "swe_limit", "swe_max_dt", "swe_step", "swe_mass",
           "swe_entropy", "swe_get_epsilon", "swe_status", "swe_timing", "swe_timing_classes",
           "swe_timing_read", "swe_step_integrals", "swe_step_async",
           "swe_launches", "swe_info", "swe_last_error", "swe_integrals_noalloc", "swe_integrals",
           "swe_ens_create", "swe_ens_destroy", "swe_ens_size", "swe_ens_layout", "swe_ens_rhs",
           "swe_ens_max_dt", "swe_ens_step", "swe_ens_integrals", "swe_ens_launches", "swe_autotune",
           "swe_get_tuning", "swe_set_tuning", "swe_ens_autotune", "swe_ens_group", "swe_rhs_adjoint",
           "swe_step_adjoint", "swe_adjoint_slots", "swe_step_record", "swe_step_adjoint_recorded",
           "swe_gauge_misfit", "swe_entropy_rate"]


class Params(ctypes.Structure):
    _fields_ = [("flux", ctypes.c_int), ("av", ctypes.c_int), ("eps0", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("limiter", ctypes.c_int), ("h_tol", ctypes.c_double), ("rk", ctypes.c_int),
                ("cfl", ctypes.c_double), ("volume", ctypes.c_int), ("cfl_visc", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int), ("x", ctypes.POINTER(ctypes.c_double)),
                ("y", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("EToE", ctypes.POINTER(ctypes.c_int32)), ("EToF", ctypes.POINTER(ctypes.c_int32)),
                ("flip", ctypes.POINTER(ctypes.c_int32))]


class SweError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swedg error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) libswedg.so and declare its C ABI."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    vp, dp, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    L.swe_create.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, i32p, i32p, i32p, dp, ctypes.c_double,
                             ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.swe_destroy.argtypes = [vp]
    L.swe_destroy.restype = None
    L.swe_rhs.argtypes = [vp, vp, vp, vp]
    L.swe_limit.argtypes = [vp, vp, vp]
    L.swe_max_dt.argtypes = [vp, vp, dp, dp, vp]
    L.swe_step.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, dp, vp]
    L.swe_step_integrals.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, dp, dp, vp]
    L.swe_step_async.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp, vp]
    L.swe_mass.argtypes = [vp, vp, dp, vp]
    L.swe_entropy.argtypes = [vp, vp, dp, vp]
    L.swe_integrals.argtypes = [vp, vp, dp, vp]
    L.swe_get_epsilon.argtypes = [vp, vp, vp]
    L.swe_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
    L.swe_timing.argtypes = [vp, ctypes.c_int]
    L.swe_timing_classes.argtypes = [vp, ctypes.c_uint]
    L.swe_timing_read.argtypes = [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int64)]
    L.swe_launches.argtypes = [vp]
    L.swe_launches.restype = ctypes.c_int64
    L.swe_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)]
    L.swe_integrals_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_double, vp, vp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int)
    L.swe_ens_create.argtypes = [ctypes.c_int, ctypes.POINTER(Instance), ctypes.c_double, ctypes.POINTER(Params),
                                 ctypes.POINTER(vp)]
    L.swe_ens_destroy.argtypes = [vp]
    L.swe_ens_destroy.restype = None
    L.swe_ens_size.argtypes = [vp, i64p, ip]
    L.swe_ens_layout.argtypes = [vp, ctypes.c_int, i64p, i64p, ip, ip]
    L.swe_ens_rhs.argtypes = [vp, vp, vp, vp]
    L.swe_ens_max_dt.argtypes = [vp, vp, dp, dp, vp]
    L.swe_ens_step.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, dp, vp]
    L.swe_ens_integrals.argtypes = [vp, vp, dp, vp]
    L.swe_ens_launches.argtypes = [vp]
    L.swe_ens_launches.restype = ctypes.c_int64
    L.swe_autotune.argtypes = [vp, vp, vp]
    L.swe_get_tuning.argtypes = [vp, ip, ip]
    L.swe_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.swe_ens_autotune.argtypes = [vp, vp, vp]
    L.swe_ens_group.argtypes = [vp, ctypes.c_int, ip, ip, ip, ip]
    L.swe_rhs_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
    L.swe_step_adjoint.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp]
    L.swe_adjoint_slots.argtypes = [vp, ctypes.c_int]
    L.swe_entropy_rate.argtypes = [vp, vp, dp, dp, vp]
    L.swe_step_record.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp]
    L.swe_step_adjoint_recorded.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp, vp, vp]
    L.swe_gauge_misfit.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.swe_last_error.argtypes = []
    L.swe_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise SweError(rc, lib().swe_last_error().decode())
    return rc


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def integrals_noalloc(N, W, wJ, b, g, out4=None, stream=None):
    """swe_integrals_noalloc: mass, momenta and entropy of device state W
    without a context and without any allocation by the library (the output
    tensor out4 is allocated here unless the caller passes one).

    W is (3, K, N+1, N+1); wJ and b hold K (N+1)^2 doubles each; all tensors
    are contiguous float64 on one CUDA device, and the call runs with that
    device current (on `stream`, which must belong to it, or on its current
    stream). Shapes and devices are checked here before the library is
    called, since the kernels trust the sizes they are given."""
    import torch
    N = int(N)
    n = N + 1
    if W.dim() != 4 or W.shape[0] != 3 or W.shape[2] != n or W.shape[3] != n:
        raise ValueError(f"swe_integrals_noalloc: W must be (3, K, {n}, {n}), got {tuple(W.shape)}")
    K = int(W.shape[1])
    for name, a in (("wJ", wJ), ("b", b)):
        if a.numel() != K * n * n:
            raise ValueError(f"swe_integrals_noalloc: {name} holds {a.numel()} values, not K (N+1)^2 = {K * n * n}")
    if out4 is not None and out4.numel() < 4:
        raise ValueError("swe_integrals_noalloc: out4 must hold at least 4 values")
    tensors = (W, wJ, b) + ((out4,) if out4 is not None else ())
    for a in tensors:
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise ValueError("swe_integrals_noalloc needs contiguous float64 CUDA tensors")
    if len({a.device for a in tensors}) != 1:
        raise ValueError("swe_integrals_noalloc: W, wJ, b and out4 must be on one CUDA device")
    if stream is not None and getattr(stream, "device", W.device) != W.device:
        raise ValueError("swe_integrals_noalloc: the stream belongs to another device")
    with torch.cuda.device(W.device):
        if out4 is None:
            out4 = torch.empty(4, dtype=torch.float64, device=W.device)
        _check(lib().swe_integrals_noalloc(N, K, ctypes.c_void_p(W.data_ptr()),
                                           ctypes.c_void_p(wJ.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                           float(g), ctypes.c_void_p(out4.data_ptr()), _stream(stream)))
    return out4


class SweContext:
    """One mesh + parameter set on the current CUDA device (swe_create)."""

    def __init__(self, N, K, x, y, EToE, EToF, flip, b, g=9.81, flux=1, av=False, eps0=0.0,
                 sigma_min=math.nan, sigma_max=math.nan, limiter=False, h_tol=math.nan, rk=0, cfl=0.5, volume=0,
                 cfl_visc=0.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("swedg needs a CUDA device; there is no CPU path")
        L = lib()
        self.N, self.K, self.n = int(N), int(K), int(N) + 1
        self.params = Params(int(flux), int(av), float(eps0), float(sigma_min), float(sigma_max),
                             int(limiter), float(h_tol), int(rk), float(cfl), int(volume), float(cfl_visc))
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, b)]
        cons = [np.ascontiguousarray(a, dtype=np.int32) for a in (EToE, EToF, flip)]
        d = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        i = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        _check(L.swe_create(self.N, self.K, d(arrs[0]), d(arrs[1]), i(cons[0]), i(cons[1]), i(cons[2]),
                            d(arrs[2]), float(g), ctypes.byref(self.params), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.N, prob.K, prob.x, prob.y, prob.EToE, prob.EToF, prob.flip, prob.b, prob.g, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.swe_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

    def _state(self, W):
        import torch
        if not (isinstance(W, torch.Tensor) and W.is_cuda and W.dtype == torch.float64 and W.is_contiguous()):
            raise ValueError("state must be a contiguous float64 CUDA tensor")
        if tuple(W.shape) != (3, self.K, self.n, self.n):
            raise ValueError(f"state shape {tuple(W.shape)} != {(3, self.K, self.n, self.n)}")
        return ctypes.c_void_p(W.data_ptr())

    def rhs(self, W, R=None, stream=None):
        import torch
        if R is None:
            R = torch.empty_like(W)
        _check(lib().swe_rhs(self._h, self._state(W), self._state(R), _stream(stream)))
        return R

    def limit(self, W, stream=None):
        _check(lib().swe_limit(self._h, self._state(W), _stream(stream)))
        return W

    def max_dt(self, W, stream=None):
        dc, dp = ctypes.c_double(), ctypes.c_double()
        _check(lib().swe_max_dt(self._h, self._state(W), ctypes.byref(dc), ctypes.byref(dp), _stream(stream)))
        return dc.value, dp.value

    def step(self, W, dt=0.0, nsteps=1, stream=None, raise_on_error=True):
        dl = ctypes.c_double(0.0)
        rc = lib().swe_step(self._h, self._state(W), float(dt), int(nsteps), ctypes.byref(dl), _stream(stream))
        if raise_on_error:
            _check(rc)
        return rc, dl.value

    def step_integrals(self, W, dt=0.0, nsteps=1, stream=None):
        """step, then (mass, x momentum, y momentum, entropy) of the new
        state, with one synchronisation; returns (integrals, dt_last)."""
        dl = ctypes.c_double(0.0)
        out = (ctypes.c_double * 4)()
        _check(lib().swe_step_integrals(self._h, self._state(W), float(dt), int(nsteps), ctypes.byref(dl), out,
                                        _stream(stream)))
        return np.array(out[:]), dl.value

    def step_async(self, W, dt=0.0, nsteps=1, out=None, stream=None):
        """step and integrals enqueued without a host synchronisation; `out`
        (device, 6 doubles, allocated here unless given) receives (mass, x
        momentum, y momentum, entropy, last step size, status bits)."""
        import torch
        if out is None:
            out = torch.empty(6, dtype=torch.float64, device=W.device)
        if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.numel() < 6:
            raise ValueError("out must be a contiguous CUDA float64 tensor of 6 elements")
        _check(lib().swe_step_async(self._h, self._state(W), float(dt), int(nsteps), ctypes.c_void_p(out.data_ptr()),
                                    _stream(stream)))
        return out

    def mass(self, W, stream=None):
        out = (ctypes.c_double * 3)()
        _check(lib().swe_mass(self._h, self._state(W), out, _stream(stream)))
        return np.array(out[:])

    def entropy(self, W, stream=None):
        e = ctypes.c_double()
        _check(lib().swe_entropy(self._h, self._state(W), ctypes.byref(e), _stream(stream)))
        return e.value

    def entropy_rate(self, W, stream=None):
        """(rate, scale): sum J w w q(W).R(W) and sum J w w |q_c R_c|."""
        r, sc = ctypes.c_double(), ctypes.c_double()
        _check(lib().swe_entropy_rate(self._h, self._state(W), ctypes.byref(r), ctypes.byref(sc), _stream(stream)))
        return r.value, sc.value

    def integrals(self, W, stream=None):
        """(mass, x momentum, y momentum, entropy) in one pass."""
        out = (ctypes.c_double * 4)()
        _check(lib().swe_integrals(self._h, self._state(W), out, _stream(stream)))
        return np.array(out[:])

    def epsilon(self, stream=None):
        import torch
        eps = torch.empty(self.K, dtype=torch.float64, device="cuda")
        _check(lib().swe_get_epsilon(self._h, ctypes.c_void_p(eps.data_ptr()), _stream(stream)))
        return eps

    def status(self, stream=None):
        b = ctypes.c_int()
        _check(lib().swe_status(self._h, ctypes.byref(b), _stream(stream)))
        return b.value

    def timing(self, on=True, classes=None):
        """Events around the context's launches: every kernel class, or only
        the named ones (`classes`, names of KERNEL_CLASSES)."""
        if classes is None:
            _check(lib().swe_timing(self._h, int(on)))
            return
        mask = 0
        for name in classes:
            mask |= 1 << KERNEL_CLASSES[name]
        _check(lib().swe_timing_classes(self._h, ctypes.c_uint(mask if on else 0)))

    def timing_read(self, which):
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        w = KERNEL_CLASSES[which] if isinstance(which, str) else int(which)
        _check(lib().swe_timing_read(self._h, w, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def launches(self):
        return int(lib().swe_launches(self._h))

    # ---- adjoint ----------------------------------------------------------
    def _plane(self, b):
        import torch
        if b is None:
            return ctypes.c_void_p()
        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.float64 and b.is_contiguous()
                and tuple(b.shape) == (self.K, self.n, self.n)):
            raise ValueError("bathymetry cotangent must be a contiguous float64 CUDA tensor [K, n, n]")
        return ctypes.c_void_p(b.data_ptr())

    def rhs_adjoint(self, W, Rbar, Wbar=None, bbar=None, stream=None):
        """Wbar += (dR/dW)^T Rbar, bbar += (dR/db)^T Rbar (allocated as zeros
        when not given); returns (Wbar, bbar)."""
        import torch
        if Wbar is None:
            Wbar = torch.zeros_like(W)
        if bbar is None:
            bbar = torch.zeros((self.K, self.n, self.n), dtype=torch.float64, device=W.device)
        _check(lib().swe_rhs_adjoint(self._h, self._state(W), self._state(Rbar), self._state(Wbar),
                                     self._plane(bbar), _stream(stream)))
        return Wbar, bbar

    def step_adjoint(self, W0, dt, Wbar, bbar=None, stream=None):
        """Wbar (cotangent of step(W0, dt)) becomes the cotangent of W0; the
        step's bathymetry cotangent is added to bbar (if given)."""
        _check(lib().swe_step_adjoint(self._h, self._state(W0), float(dt), self._state(Wbar), self._plane(bbar),
                                      _stream(stream)))
        return Wbar

    def adjoint_slots(self, nslots):
        """Reserve nslots step records (swe_adjoint_slots)."""
        _check(lib().swe_adjoint_slots(self._h, int(nslots)))

    def step_record(self, W, dt, slot, stream=None):
        """One step of size dt on W in place, recorded in `slot` (swe_step_record)."""
        _check(lib().swe_step_record(self._h, self._state(W), float(dt), int(slot), _stream(stream)))
        return W

    def step_adjoint_recorded(self, slot, dt, Wbar, bbar=None, stream=None):
        """swe_step_adjoint for the step recorded in `slot`."""
        _check(lib().swe_step_adjoint_recorded(self._h, int(slot), float(dt), self._state(Wbar), self._plane(bbar),
                                               _stream(stream)))
        return Wbar

    def gauge_misfit(self, W, elem, wts, target=None, values=None, loss=None, Wbar=None, stream=None):
        """swe_gauge_misfit on device tensors (elem int32 [G], wts [G, n*n])."""
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()
        _check(lib().swe_gauge_misfit(self._h, self._state(W), int(elem.numel()), ptr(elem), ptr(wts), ptr(target),
                                      ptr(values), ptr(loss), ptr(Wbar) if Wbar is None else self._state(Wbar),
                                      _stream(stream)))

    def autotune(self, W, stream=None):
        """Time the launch shapes on W and keep the fastest; returns them."""
        _check(lib().swe_autotune(self._h, self._state(W), _stream(stream)))
        return self.tuning()

    def tuning(self):
        v, u = ctypes.c_int(), ctypes.c_int()
        _check(lib().swe_get_tuning(self._h, ctypes.byref(v), ctypes.byref(u)))
        return v.value, u.value

    def set_tuning(self, vol_threads, upd_warps):
        _check(lib().swe_set_tuning(self._h, int(vol_threads), int(upd_warps)))

    def info(self):
        N, K, nf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().swe_info(self._h, ctypes.byref(N), ctypes.byref(K), ctypes.byref(nf)))
        return N.value, K.value, nf.value


class SweEnsemble:
    """Many independent meshes of mixed degree advanced together
    (swe_ens_create). State: one flat float64 CUDA tensor of `size` doubles;
    `view(W, i)` is instance i's (3, K, n, n) view into it."""

    def __init__(self, problems, g=9.81, flux=1, av=False, eps0=0.0, sigma_min=math.nan,
                 sigma_max=math.nan, limiter=False, h_tol=math.nan, rk=0, cfl=0.5, volume=0, cfl_visc=0.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("swedg needs a CUDA device; there is no CPU path")
        L = lib()
        self.params = Params(int(flux), int(av), float(eps0), float(sigma_min), float(sigma_max),
                             int(limiter), float(h_tol), int(rk), float(cfl), int(volume), float(cfl_visc))
        self.ninst = len(problems)
        keep = []
        arr = (Instance * self.ninst)()
        d = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        i32 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        for i, p in enumerate(problems):
            x, y, b = (np.ascontiguousarray(a, dtype=np.float64) for a in (p.x, p.y, p.b))
            E, F, fl = (np.ascontiguousarray(a, dtype=np.int32) for a in (p.EToE, p.EToF, p.flip))
            keep += [x, y, b, E, F, fl]
            arr[i] = Instance(int(p.N), int(p.K), d(x), d(y), d(b), i32(E), i32(F), i32(fl))
        h = ctypes.c_void_p()
        _check(L.swe_ens_create(self.ninst, arr, float(g), ctypes.byref(self.params), ctypes.byref(h)))
        self._h = h
        tot, ng = ctypes.c_int64(), ctypes.c_int()
        _check(L.swe_ens_size(h, ctypes.byref(tot), ctypes.byref(ng)))
        self.size, self.ngroups = tot.value, ng.value
        self.layout = []
        for i in range(self.ninst):
            off, st, N, K = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
            _check(L.swe_ens_layout(h, i, ctypes.byref(off), ctypes.byref(st), ctypes.byref(N), ctypes.byref(K)))
            self.layout.append((off.value, st.value, N.value, K.value))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.swe_ens_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

    def empty(self):
        import torch
        return torch.zeros(self.size, dtype=torch.float64, device="cuda")

    def view(self, W, i):
        """Instance i's (3, K, n, n) strided view of ensemble state W."""
        off, st, N, K = self.layout[i]
        n = N + 1
        return W.as_strided((3, K, n, n), (st, n * n, n, 1), off)

    def pack(self, states, W=None):
        """Ensemble state from per-instance (3, K, n, n) arrays or tensors."""
        import torch
        W = self.empty() if W is None else W
        for i, s in enumerate(states):
            t = s if isinstance(s, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(s))
            self.view(W, i).copy_(t)
        return W

    def _state(self, W):
        import torch
        if not (isinstance(W, torch.Tensor) and W.is_cuda and W.dtype == torch.float64 and W.is_contiguous()
                and W.numel() == self.size):
            raise ValueError(f"ensemble state must be a contiguous float64 CUDA tensor of {self.size} values")
        return ctypes.c_void_p(W.data_ptr())

    def rhs(self, W, R=None, stream=None):
        import torch
        if R is None:
            R = torch.zeros_like(W)
        _check(lib().swe_ens_rhs(self._h, self._state(W), self._state(R), _stream(stream)))
        return R

    def max_dt(self, W, stream=None):
        dc = (ctypes.c_double * self.ninst)()
        dp = (ctypes.c_double * self.ninst)()
        _check(lib().swe_ens_max_dt(self._h, self._state(W), dc, dp, _stream(stream)))
        return np.array(dc[:]), np.array(dp[:])

    def step(self, W, dt=0.0, nsteps=1, stream=None, raise_on_error=True):
        dl = (ctypes.c_double * self.ninst)()
        rc = lib().swe_ens_step(self._h, self._state(W), float(dt), int(nsteps), dl, _stream(stream))
        if raise_on_error:
            _check(rc)
        return rc, np.array(dl[:])

    def entropy_rate(self, W, stream=None):
        """(rate, scale): sum J w w q(W).R(W) and sum J w w |q_c R_c|."""
        r, sc = ctypes.c_double(), ctypes.c_double()
        _check(lib().swe_entropy_rate(self._h, self._state(W), ctypes.byref(r), ctypes.byref(sc), _stream(stream)))
        return r.value, sc.value

    def integrals(self, W, stream=None):
        out = (ctypes.c_double * (4 * self.ninst))()
        _check(lib().swe_ens_integrals(self._h, self._state(W), out, _stream(stream)))
        return np.array(out[:]).reshape(self.ninst, 4)

    def launches(self):
        return int(lib().swe_ens_launches(self._h))

    def autotune(self, W, stream=None):
        _check(lib().swe_ens_autotune(self._h, self._state(W), _stream(stream)))
        return self.groups()

    def groups(self):
        """[(N, members, volume threads per block, update warps per block)] per degree group."""
        out = []
        for g in range(self.ngroups):
            v = [ctypes.c_int() for _ in range(4)]
            _check(lib().swe_ens_group(self._h, g, *[ctypes.byref(x) for x in v]))
            out.append(tuple(x.value for x in v))
        return out


class GaugeLoss:
    """Loss L = sum over steps t = 1..T and gauges g of (h_g(W_t) - target_{t,g})^2
    of an adaptive run of `nsteps` swe_step steps from W0, and its gradient
    with respect to W0 and the bathymetry through the library's adjoint
    (swe_step_adjoint, swe_gauge_misfit), recomputing states from checkpoints
    taken every `checkpoint` steps. The step sizes of the forward run are
    kept and reused by the reverse sweep. Device tensors: elem int32 [G],
    wts float64 [G, n*n], targets float64 [T, G]."""

    def __init__(self, ctx, elem, wts, targets, nsteps, checkpoint=20):
        self.ctx, self.elem, self.wts = ctx, elem, wts
        self.targets, self.nsteps, self.checkpoint = targets, int(nsteps), max(1, int(checkpoint))

    def forward(self, W0, record=None):
        """Runs the steps; returns the loss (device scalar tensor). record
        (optional [T, G] tensor) receives the gauge values."""
        import torch
        ctx = self.ctx
        W = W0.clone()
        loss = torch.zeros(1, dtype=torch.float64, device=W0.device)
        self.dts, self.ckpt = [], {0: W0.clone()}
        for t in range(self.nsteps):
            _, dt = ctx.step(W, 0.0, 1)
            self.dts.append(dt)
            vals = None if record is None else record[t]
            ctx.gauge_misfit(W, self.elem, self.wts, target=self.targets[t], values=vals, loss=loss)
            if (t + 1) % self.checkpoint == 0 and t + 1 < self.nsteps:
                self.ckpt[t + 1] = W.clone()
        return loss[0]

    def backward(self, grad_b=True, recorded=True):
        """(dL/dW0, dL/db) of the last forward run. Each segment between
        checkpoints is recomputed once; with `recorded` its steps are
        recorded on the way (swe_step_record, one record per step of the
        segment) so that the reverse sweep does not recompute them again,
        otherwise every step adjoint recomputes its step (swe_step_adjoint).
        Both give the same gradients bit for bit."""
        import torch
        ctx = self.ctx
        W0 = self.ckpt[0]
        Wbar = torch.zeros_like(W0)
        bbar = torch.zeros((ctx.K, ctx.n, ctx.n), dtype=torch.float64, device=W0.device) if grad_b else None
        T = self.nsteps
        starts = sorted(self.ckpt)
        if recorded:
            ctx.adjoint_slots(min(self.checkpoint, T))
        for c0 in reversed(starts):
            nxt = [s for s in starts if s > c0]
            c1 = nxt[0] if nxt else T
            # states W_{c0} .. W_{c1} of the segment, with the recorded step sizes
            states = [self.ckpt[c0].clone()]
            for t in range(c0, c1):
                W = states[-1].clone()
                if recorded:
                    ctx.step_record(W, self.dts[t], t - c0)
                else:
                    ctx.step(W, self.dts[t], 1)
                states.append(W)
            for t in range(c1, c0, -1):
                ctx.gauge_misfit(states[t - c0], self.elem, self.wts, target=self.targets[t - 1], Wbar=Wbar)
                if recorded:
                    ctx.step_adjoint_recorded(t - 1 - c0, self.dts[t - 1], Wbar, bbar)
                else:
                    ctx.step_adjoint(states[t - 1 - c0], self.dts[t - 1], Wbar, bbar)
        return Wbar, bbar


def gauge_loss(ctx, W0, b, elem, wts, targets, nsteps, checkpoint=20):
    """torch.autograd entry point: loss of GaugeLoss with gradients flowing to
    W0 and to b (the bathymetry tensor the context was created with)."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, W0_, b_):
            run = GaugeLoss(ctx, elem, wts, targets, nsteps, checkpoint)
            loss = run.forward(W0_)
            fctx.run = run
            return loss

        @staticmethod
        def backward(fctx, g):
            Wbar, bbar = fctx.run.backward(grad_b=True)
            return g * Wbar, (g * bbar).to(b.device).reshape(b.shape)

    return _Fn.apply(W0, b)
