"""ctypes wrapper of the C oracle (orc.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg to check and time the CUDA library. The product
path never imports this module.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orc.c")
HDR = os.path.join(HERE, "orc.h")
LIB = os.path.join(HERE, "_build", "liborc.so")

OK, ERR_ARG, ERR_GEOM, ERR_NEG_MEAN, ERR_NONFINITE = 0, -1, -2, -3, -4


def _flags(variant):
    """Compiler flags of a build variant. The default build is the checker:
    no FMA contraction, so x86-64 and aarch64 give the same results. The
    "tuned" build exists only to time the oracle as fast as the host compiler
    makes it (FMA contraction, -O3, the host's own CPU target on aarch64); its
    results are never compared with anything."""
    if variant is None:
        return ["-O2", "-ffp-contract=off"]
    if variant == "tuned":
        import platform
        f = ["-O3", "-ffp-contract=fast"]
        if platform.machine() == "aarch64":
            f.append("-mcpu=native")
        return f
    raise ValueError(f"unknown oracle build variant {variant!r}")


def lib_path(variant=None) -> str:
    return LIB if variant is None else os.path.join(HERE, "_build", f"liborc_{variant}.so")


def build(force: bool = False, variant=None) -> str:
    """Compile orc.c into _build/liborc.so (gcc, OpenMP, no FMA contraction so
    that results agree between x86-64 and aarch64 hosts), or the timing-only
    variant into _build/liborc_<variant>.so."""
    path = lib_path(variant)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    stale = (not os.path.exists(path) or
             os.path.getmtime(path) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11"] + _flags(variant) + ["-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


class Params(ctypes.Structure):
    _fields_ = [("flux", ctypes.c_int), ("av", ctypes.c_int), ("eps0", ctypes.c_double),
                ("sigma_min", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("limiter", ctypes.c_int), ("h_tol", ctypes.c_double), ("rk", ctypes.c_int),
                ("cfl", ctypes.c_double), ("volume", ctypes.c_int), ("cfl_visc", ctypes.c_double)]


_libs = {}


def lib(variant=None):
    if variant not in _libs:
        L = ctypes.CDLL(build(variant=variant))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        L.orc_basis.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ip, ip, ip, dp, ctypes.c_double,
                                 ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.orc_destroy.argtypes = [vp]
        L.orc_destroy.restype = None
        L.orc_geometry.argtypes = [vp, dp, dp, dp, dp, dp]
        L.orc_rhs.argtypes = [vp, dp, dp]
        L.orc_get_epsilon.argtypes = [vp, dp]
        L.orc_av_fields.argtypes = [vp, dp, dp, dp]
        L.orc_limit.argtypes = [vp, dp]
        L.orc_max_dt.argtypes = [vp, dp, dp, dp]
        L.orc_step.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int, dp]
        L.orc_mass.argtypes = [vp, dp, dp]
        L.orc_entropy.argtypes = [vp, dp, dp]
        L.orc_entropy_rate.argtypes = [vp, dp, dp, dp]
        L.orc_volume_flux.argtypes = [ctypes.c_double, dp, dp, dp, dp]
        L.orc_volume_flux.restype = None
        L.orc_surface_flux.argtypes = [ctypes.c_double, ctypes.c_int, dp, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_surface_flux.restype = None
        L.orc_threads.argtypes = []
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        L.orc_lsrk_coefficients.argtypes = [dp, dp]
        L.orc_lsrk_coefficients.restype = None
        _libs[variant] = L
    return _libs[variant]


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert a.dtype == np.int32
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def basis(N: int):
    n = N + 1
    xi, w = np.zeros(n), np.zeros(n)
    D, V, Vinv = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    rc = lib().orc_basis(N, _p(xi), _p(w), _p(D), _p(V), _p(Vinv))
    if rc:
        raise ValueError(f"orc_basis rc={rc}")
    return xi, w, D, V, Vinv


def volume_flux(g, Wa, Wb):
    Fs, Gs = np.zeros(3), np.zeros(3)
    lib().orc_volume_flux(g, _p(np.ascontiguousarray(Wa, dtype=np.float64)),
                          _p(np.ascontiguousarray(Wb, dtype=np.float64)), _p(Fs), _p(Gs))
    return Fs, Gs


def surface_flux(g, es, Wm, Wp, bm, bp, nx, ny):
    F = np.zeros(3)
    lib().orc_surface_flux(g, int(es), _p(np.ascontiguousarray(Wm, dtype=np.float64)),
                           _p(np.ascontiguousarray(Wp, dtype=np.float64)), bm, bp, nx, ny, _p(F))
    return F


def lsrk_coefficients():
    A, B = np.zeros(5), np.zeros(5)
    lib().orc_lsrk_coefficients(_p(A), _p(B))
    return A, B


def threads(variant=None) -> int:
    return lib(variant).orc_threads()


def set_threads(t: int, variant=None) -> None:
    """OpenMP threads of later oracle calls (for timing the oracle)."""
    lib(variant).orc_set_threads(int(t))


class Oracle:
    """Oracle instance for one Problem (see paper_1804_02221_gb300.inputs)."""

    def __init__(self, prob, flux=1, av=False, eps0=0.0, sigma_min=math.nan, sigma_max=math.nan,
                 limiter=False, h_tol=math.nan, rk=0, cfl=0.5, volume=0, cfl_visc=0.0, variant=None):
        self.prob = prob
        self._L = lib(variant)
        self.N, self.K, self.n = prob.N, prob.K, prob.N + 1
        self.params = Params(int(flux), int(av), float(eps0), float(sigma_min), float(sigma_max),
                             int(limiter), float(h_tol), int(rk), float(cfl), int(volume), float(cfl_visc))
        self._x = np.ascontiguousarray(prob.x, dtype=np.float64)
        self._y = np.ascontiguousarray(prob.y, dtype=np.float64)
        self._b = np.ascontiguousarray(prob.b, dtype=np.float64)
        self._E = np.ascontiguousarray(prob.EToE, dtype=np.int32)
        self._F = np.ascontiguousarray(prob.EToF, dtype=np.int32)
        self._fl = np.ascontiguousarray(prob.flip, dtype=np.int32)
        h = ctypes.c_void_p()
        rc = self._L.orc_create(self.N, self.K, _p(self._x), _p(self._y), _p(self._E), _p(self._F),
                              _p(self._fl), _p(self._b), float(prob.g), ctypes.byref(self.params),
                              ctypes.byref(h))
        if rc:
            raise ValueError(f"orc_create rc={rc}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and getattr(self, "_L", None) is not None:
            self._L.orc_destroy(h)
            self._h = None

    def _W(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (3, self.K, self.n, self.n), W.shape
        return W

    def geometry(self):
        shp = (self.K, self.n, self.n)
        out = [np.zeros(shp) for _ in range(5)]
        self._L.orc_geometry(self._h, *[_p(a) for a in out])
        return dict(zip(("x_xi", "x_eta", "y_xi", "y_eta", "J"), out))

    def rhs(self, W):
        W = self._W(W)
        R = np.zeros_like(W)
        rc = self._L.orc_rhs(self._h, _p(W), _p(R))
        if rc:
            raise RuntimeError(f"orc_rhs rc={rc}")
        return R

    def epsilon(self):
        e = np.zeros(self.K)
        self._L.orc_get_epsilon(self._h, _p(e))
        return e

    def av_fields(self, W):
        W = self._W(W)
        eps = np.zeros(self.K)
        grads = np.zeros((4, self.K, self.n, self.n))
        self._L.orc_av_fields(self._h, _p(W), _p(eps), _p(grads))
        return eps, grads

    def limit(self, W):
        W = self._W(W).copy()
        rc = self._L.orc_limit(self._h, _p(W))
        return W, rc

    def max_dt(self, W):
        W = self._W(W)
        dc, dp = ctypes.c_double(), ctypes.c_double()
        self._L.orc_max_dt(self._h, _p(W), ctypes.byref(dc), ctypes.byref(dp))
        return dc.value, dp.value

    def step(self, W, dt=0.0, nsteps=1):
        W = self._W(W).copy()
        dl = ctypes.c_double(0.0)
        rc = self._L.orc_step(self._h, _p(W), float(dt), int(nsteps), ctypes.byref(dl))
        return W, rc, dl.value

    def mass(self, W):
        out = np.zeros(3)
        self._L.orc_mass(self._h, _p(self._W(W)), _p(out))
        return out

    def entropy_rate(self, W):
        """(rate, scale): sum J w w q(W).R(W) and sum J w w |q_c R_c|."""
        r, sc = ctypes.c_double(), ctypes.c_double()
        rc = self._L.orc_entropy_rate(self._h, _p(self._W(W)), ctypes.byref(r), ctypes.byref(sc))
        assert rc == OK
        return r.value, sc.value

    def entropy(self, W):
        e = ctypes.c_double()
        self._L.orc_entropy(self._h, _p(self._W(W)), ctypes.byref(e))
        return e.value
