"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/swedg.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1804_02221_gb300 import build as B
from paper_1804_02221_gb300 import swedg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "swedg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swe_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("swe_create", "swe_rhs", "swe_limit", "swe_max_dt", "swe_step", "swe_mass",
              "swe_entropy", "swe_destroy", "swe_last_error"):
        assert s in syms


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} declared in swedg.h but not exported"
    # the Python binding names the same entry points
    assert set(swedg.SYMBOLS) == set(declared_symbols())


def test_last_error_callable_without_gpu():
    lib = swedg.lib()
    assert isinstance(lib.swe_last_error(), bytes)


# ---------------------------------------------------------------------------
# Argument checks that return before any CUDA call (host logic, no GPU)
# ---------------------------------------------------------------------------

def _dp():
    return ctypes.POINTER(ctypes.c_double)


def _call_create(N, K, params=None, n_elem=1):
    lib = swedg.lib()
    nn = (N + 1) ** 2
    x = (ctypes.c_double * (nn * n_elem))()
    i4 = (ctypes.c_int32 * (4 * n_elem))()
    p = params or swedg.Params(1, 0, 0.0, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 0)
    h = ctypes.c_void_p()
    rc = lib.swe_create(N, K, x, x, i4, i4, i4, x, 9.81, ctypes.byref(p), ctypes.byref(h))
    return rc, lib.swe_last_error().decode()


def test_create_rejects_empty_mesh_and_bad_degrees():
    for N, K in ((3, 0), (3, -1), (0, 4), (13, 4)):
        rc, msg = _call_create(N, K)
        assert rc == swedg.ERR_ARG, (N, K, msg)


def test_create_rejects_meshes_beyond_32_bit_node_ids():
    # N = 12 (169 nodes per element): 3 K n^2 > 2^31 - 1 from K = 4,235,629 on;
    # the size check runs before any input array is read
    rc, msg = _call_create(12, 4_300_000)
    assert rc == swedg.ERR_ARG and "32-bit" in msg


def test_create_rejects_bad_parameters():
    bad = [swedg.Params(2, 0, 0.0, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 0),   # flux
           swedg.Params(1, 0, 0.0, float("nan"), float("nan"), 0, float("nan"), 2, 0.5, 0),   # rk
           swedg.Params(1, 1, -1.0, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 0),  # eps0
           swedg.Params(1, 0, 0.0, float("nan"), float("nan"), 0, -1.0, 0, 0.5, 0),           # h_tol
           swedg.Params(1, 0, 0.0, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 3),   # volume
           swedg.Params(1, 1, 0.1, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 0, -1.0)]  # cfl_visc
    for p in bad:
        rc, _ = _call_create(3, 1, p)
        assert rc == swedg.ERR_ARG


def test_ensemble_create_rejects_empty_and_bad_members():
    lib = swedg.lib()
    p = swedg.Params(1, 0, 0.0, float("nan"), float("nan"), 0, float("nan"), 0, 0.5, 0)
    h = ctypes.c_void_p()
    assert lib.swe_ens_create(0, None, 9.81, ctypes.byref(p), ctypes.byref(h)) == swedg.ERR_ARG
    arr = (swedg.Instance * 1)()
    arr[0] = swedg.Instance(3, 0, None, None, None, None, None, None)  # K = 0
    assert lib.swe_ens_create(1, arr, 9.81, ctypes.byref(p), ctypes.byref(h)) == swedg.ERR_ARG


def test_null_contexts_are_rejected():
    lib = swedg.lib()
    assert lib.swe_rhs(None, None, None, None) == swedg.ERR_ARG
    assert lib.swe_step(None, None, 0.0, 1, None, None) == swedg.ERR_ARG
    assert lib.swe_step_integrals(None, None, 0.0, 1, None, None, None) == swedg.ERR_ARG
    assert lib.swe_step_async(None, None, 0.0, 1, None, None) == swedg.ERR_ARG
    assert lib.swe_timing_classes(None, 1) == swedg.ERR_ARG
    assert lib.swe_rhs_adjoint(None, None, None, None, None, None) == swedg.ERR_ARG
    assert lib.swe_gauge_misfit(None, None, 0, None, None, None, None, None, None, None) == swedg.ERR_ARG
    lib.swe_destroy(None)
    lib.swe_ens_destroy(None)


def test_noalloc_wrapper_checks_shapes_before_the_library(monkeypatch):
    """integrals_noalloc refuses mis-shaped or host tensors before it calls
    the library (its kernels trust the sizes they are given)."""
    torch = pytest.importorskip("torch")

    def no_library():
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(swedg, "lib", no_library)
    f64 = dict(dtype=torch.float64)
    N, K = 3, 4
    W, wJ, b = torch.zeros(3, K, 4, 4, **f64), torch.zeros(K, 4, 4, **f64), torch.zeros(K, 4, 4, **f64)
    with pytest.raises(ValueError, match="W must be"):
        swedg.integrals_noalloc(N, torch.zeros(3, K, 4, 5, **f64), wJ, b, 9.81)
    with pytest.raises(ValueError, match="W must be"):
        swedg.integrals_noalloc(N, torch.zeros(2, K, 4, 4, **f64), wJ, b, 9.81)
    with pytest.raises(ValueError, match="wJ holds"):
        swedg.integrals_noalloc(N, W, torch.zeros(K - 1, 4, 4, **f64), b, 9.81)
    with pytest.raises(ValueError, match="b holds"):
        swedg.integrals_noalloc(N, W, wJ, torch.zeros(K, 16, **f64)[:, :15], 9.81)
    with pytest.raises(ValueError, match="out4"):
        swedg.integrals_noalloc(N, W, wJ, b, 9.81, out4=torch.zeros(3, **f64))
    with pytest.raises(ValueError, match="CUDA"):
        swedg.integrals_noalloc(N, W, wJ, b, 9.81)
