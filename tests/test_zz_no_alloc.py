"""The allocation-free diagnostic integrals (swe_integrals_noalloc) agree with
the context-based swe_mass / swe_entropy.

That entry point serves callers that cannot call cudaMalloc (a host framework
owning the device memory pool, real-time loops that cannot afford the
allocator's device synchronisation, hosts with a fixed memory budget). It
keeps its partial sums in one fixed device array of the library, so this file
runs last and checks two calls in a row, with different states, against the
existing entry points.
"""
import ctypes

import numpy as np
import pytest

import refmath
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_noalloc_integrals_match_context_integrals_twice():
    from paper_1804_02221_gb300 import swedg
    p = I.random_rough(N=4, K1=9, seed=5, rotate_seed=2)
    ctx = swedg.SweContext.from_problem(p)
    geo = refmath.geometry(p.x, p.y, p.N)
    wJ = torch.from_numpy(np.ascontiguousarray(refmath.quad_weights(p.N) * geo[4])).cuda()
    b = torch.from_numpy(np.ascontiguousarray(p.b)).cuda()
    rng = np.random.default_rng(3)
    states = [p.W, p.W * (1.0 + 0.1 * rng.uniform(-1, 1, size=p.W.shape))]
    for Wn in states:  # two calls in a row, the second overwriting the first's partials
        W = torch.from_numpy(np.ascontiguousarray(Wn)).cuda()
        out = swedg.integrals_noalloc(p.N, W, wJ, b, p.g).cpu().numpy()
        mass = ctx.mass(W)
        ent = ctx.entropy(W)
        assert np.abs(out[:3] - mass).max() <= 1e-13 * np.abs(mass).max()
        assert abs(out[3] - ent) <= 1e-13 * abs(ent)


def test_noalloc_rejects_too_many_elements():
    from paper_1804_02221_gb300 import swedg
    lib = swedg.lib()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    K = 65537  # one above SWE_NOALLOC_MAX_ELEMENTS; rejected before any launch
    ptr = ctypes.c_void_p(x.data_ptr())
    rc = lib.swe_integrals_noalloc(3, K, ptr, ptr, ptr, 9.81, ptr, ctypes.c_void_p(0))
    assert rc == swedg.ERR_ARG
    assert b"exceeds" in lib.swe_last_error()


def test_noalloc_rejects_host_memory():
    """A host pointer is refused before any launch (the kernels would read
    it as a device address)."""
    from paper_1804_02221_gb300 import swedg
    lib = swedg.lib()
    host = np.zeros(3 * 4 * 16)
    dev = torch.zeros(3 * 4 * 16, dtype=torch.float64, device="cuda")
    hp, dp = ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(dev.data_ptr())
    rc = lib.swe_integrals_noalloc(3, 4, hp, dp, dp, 9.81, dp, ctypes.c_void_p(0))
    assert rc == swedg.ERR_ARG
    assert b"W" in lib.swe_last_error()
