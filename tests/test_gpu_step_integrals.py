"""swe_step_integrals: the step and the new state's integrals with one
synchronisation. W and the integrals are bitwise those of swe_step followed
by swe_integrals, for every launch shape; a failed step restores W and
leaves the integrals alone."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

AV = dict(eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,K1,rk,fixed,nsteps", [(1, 9, 0, False, 1), (3, 7, 1, False, 3), (5, 4, 0, True, 2),
                                                   (7, 3, 0, False, 1), (12, 2, 1, True, 2)])
def test_equals_step_then_integrals(N, K1, rk, fixed, nsteps):
    swedg = swe_mod()
    p = I.random_rough(N=N, K1=K1, seed=90 + N, dry_fraction=0.05)
    kw = dict(flux=1, av=True, limiter=True, rk=rk, cfl=0.4, **AV)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    # a fixed step: half the admissible one of the initial state
    dt = 0.5 * min(c.max_dt(dev(W0))) if fixed else 0.0
    Wa = dev(W0)
    _, dta = c.step(Wa, dt, nsteps)
    ref = c.integrals(Wa)
    for vol, upd in ((128, 4), (64, 2), (128, 8)):
        c.set_tuning(vol, upd)
        Wb = dev(W0)
        got, dtb = c.step_integrals(Wb, dt, nsteps)
        assert torch.equal(Wa, Wb), (vol, upd)
        assert np.array_equal(got, ref), (vol, upd)
        assert dtb == dta
    assert np.all(np.isfinite(ref)) and ref[0] > 0


def test_failed_step_restores_state_and_bad_arguments():
    swedg = swe_mod()
    p = I.random_rough(N=3, K1=4, seed=9, dry_fraction=0.5)
    kw = dict(flux=1, limiter=True, rk=1)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    W = dev(W0)
    with pytest.raises(swedg.SweError) as e:
        c.step_integrals(W, 1e-3, 0)
    assert e.value.code == swedg.ERR_ARG
    with pytest.raises(swedg.SweError) as e:
        c.step_integrals(W, 5.0, 1)   # far above the admissible step size
    assert e.value.code in (swedg.ERR_NEG_MEAN, swedg.ERR_NONFINITE)
    assert np.array_equal(W.cpu().numpy(), W0)
    # the context is usable afterwards
    dt = min(c.max_dt(W))
    got, _ = c.step_integrals(W, dt, 1)
    assert np.array_equal(got, c.integrals(W))


def test_failed_async_step_restores_state_and_its_integrals():
    """swe_step_async that fails restores W on the device; the integrals it
    leaves in out (read from the velocities, which the restore rewrites) are
    bitwise those of the restored state, and the status bits are set."""
    swedg = swe_mod()
    p = I.random_rough(N=3, K1=4, seed=9, dry_fraction=0.5)
    kw = dict(flux=1, limiter=True, rk=1)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    W = dev(W0)
    out = c.step_async(W, 5.0, 1)   # far above the admissible step size
    got = out.cpu().numpy()
    assert int(got[5]) != 0
    assert np.array_equal(W.cpu().numpy(), W0)
    assert np.array_equal(got[:4], c.integrals(W))


def test_integrals_against_oracle_after_steps():
    """Mass conservation and the oracle's integrals of the GPU state."""
    swedg = swe_mod()
    p = I.dam_break(N=4, K1=12)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    c = swedg.SweContext.from_problem(p, **kw)
    W = dev(p.W)
    m0 = c.integrals(W)
    got, _ = c.step_integrals(W, 0.0, 5)
    o = O.Oracle(p, **kw)
    Wh = W.cpu().numpy()
    mo, eo = o.mass(Wh), o.entropy(Wh)
    assert np.abs(got[:3] - mo).max() < 1e-13 * np.abs(mo).max()
    assert abs(got[3] - eo) < 1e-13 * abs(eo)
    assert abs(got[0] - m0[0]) < 1e-12 * m0[0]


def test_async_step_equals_synchronous_step():
    swedg = swe_mod()
    p = I.random_rough(N=4, K1=6, seed=31, dry_fraction=0.1)
    kw = dict(flux=1, av=True, limiter=True, rk=0, cfl=0.4, **AV)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    Wa = dev(W0)
    ints, dta = c.step_integrals(Wa, 0.0, 2)
    Wb = dev(W0)
    out = c.step_async(Wb, 0.0, 2)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert torch.equal(Wa, Wb)
    assert np.array_equal(o[:4], ints) and o[4] == dta and o[5] == 0.0


def test_async_failed_step_rolls_back_on_the_device():
    swedg = swe_mod()
    p = I.random_rough(N=3, K1=4, seed=9, dry_fraction=0.5)
    kw = dict(flux=1, limiter=True, rk=1)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    W = dev(W0)
    out = c.step_async(W, 5.0, 1)   # far above the admissible step size
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert int(o[5]) & 3
    assert np.array_equal(W.cpu().numpy(), W0)
    assert np.array_equal(o[:4], c.integrals(W))
    assert c.status() & 3
    with pytest.raises(swedg.SweError) as e:
        c.step_async(W, 1e-3, 0)
    assert e.value.code == swedg.ERR_ARG
    dt = min(c.max_dt(W))
    o2 = c.step_async(W, dt, 1).cpu().numpy()
    assert o2[5] == 0.0


@pytest.mark.parametrize("N,K1", [(3, 12), (7, 128)])
def test_async_step_replays_in_a_cuda_graph(N, K1):
    """Captured once, replayed three times: the same bits as three
    swe_step calls (adaptive step sizes computed on the device). At N = 7 on
    128 x 128 quads (2^20 nodes) the context runs its indicator, start-state
    copy and time step on its second stream, which the capture takes in
    through the fork and join events."""
    swedg = swe_mod()
    p = I.dam_break(N=N, K1=K1)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    c = swedg.SweContext.from_problem(p, **kw)
    Wr = dev(p.W)
    for _ in range(3):
        c.step(Wr, 0.0, 1)
    ref = c.integrals(Wr)
    W = dev(p.W)
    W0 = dev(p.W)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.step_async(W, 0.0, 1, out)      # warm-up outside the capture
    torch.cuda.synchronize()
    W.copy_(W0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        c.step_async(W, 0.0, 1, out)
    W.copy_(W0)                       # capture does not run the work
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(W, Wr)
    o = out.cpu().numpy()
    assert np.array_equal(o[:4], ref) and o[5] == 0.0


def _run_500(p, kw):
    swedg = swe_mod()
    c = swedg.SweContext.from_problem(p, **kw)
    W = dev(p.W)
    m0 = c.integrals(W)
    res = torch.zeros((500, 6), dtype=torch.float64, device="cuda")
    for i in range(500):
        c.step_async(W, 0.0, 1, out=res[i])
    torch.cuda.synchronize()
    return m0, res.cpu().numpy(), W


def _check_invariants(m0, r, W):
    assert np.all(r[:, 5] == 0.0), "a step failed"
    assert np.all(r[:, 4] > 0.0)
    # mass conserved on the periodic mesh (the momenta are not: the
    # bathymetry source acts on them)
    assert np.abs(r[:, 0] - m0[0]).max() <= 1e-12 * m0[0]
    # the total entropy decreases in every step (ES flux and AV dissipate)
    E = np.concatenate(([m0[3]], r[:, 3]))
    assert np.all(np.diff(E) <= 1e-13 * abs(m0[3]))
    assert E[-1] < E[0]
    assert torch.isfinite(W).all()
    assert float(W[0].min()) > 0.0


@pytest.mark.parametrize("N,K1,eps0", [(7, 64, 0.005), (3, 128, 0.01)])
def test_dam_break_500_steps_invariants(N, K1, eps0):
    """The dam break (ES flux + AV + limiter, adaptive LSRK4(5)) for 500
    asynchronous steps, in configurations where the paper's time-step rule
    (CFL and positivity, no viscous restriction) keeps the explicit AV term
    stable: every step succeeds, mass is conserved, the entropy decreases in
    every step (Thm. 1), h stays positive. (With eps0 = 0.025 at these
    sizes, or any eps0 at 256 x 256 quads and N = 7, the fixed-eps0 AV term
    outgrows the explicit step: the rule gives no viscous limit.)"""
    p = I.dam_break(N=N, K1=K1)
    kw = dict(flux=1, av=True, eps0=eps0, limiter=True, rk=0, cfl=0.5)
    _check_invariants(*_run_500(p, kw))


def test_full_size_smooth_500_steps_invariants():
    """The full-size mesh (N = 7, 256 x 256 curved quads, 4.19M nodes) with a
    smooth state (a hump on a lake at rest over a smooth bathymetry), ES flux,
    AV and limiter on, 500 asynchronous adaptive steps: every step succeeds,
    mass is conserved, the entropy decreases in every step, h stays
    positive."""
    p = I.lake_hump(N=7, K1=256, amp=0.05)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    _check_invariants(*_run_500(p, kw))
