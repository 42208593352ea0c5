"""Parity of the CUDA library (through its C ABI) with the CPU oracle on the
same seeded inputs.

Tolerances: 5e-14 per right-hand side, relative to max(|R|_inf, T) with T the
size of the largest term of the flux difference (see parity.py for why the
cancelled result alone is not the right scale near equilibrium; the plain
relative L-infinity is recorded beside it for every case); 1e-10 relative
L-infinity of the state after 100 Runge-Kutta steps.
"""
import math
import os

import numpy as np
import pytest

import refmath
from parity import check_rhs, rel
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

STEP_TOL = 1e-10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lake_hump_exact_rhs.npz")


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def pair(prob, **kw):
    return O.Oracle(prob, **kw), swe_mod().SweContext.from_problem(prob, **kw)


def dev(W):
    return torch.from_numpy(np.ascontiguousarray(W)).cuda()


def rhs_both(prob, **kw):
    o, g = pair(prob, **kw)
    Ro = o.rhs(prob.W)
    Rg = g.rhs(dev(prob.W)).cpu().numpy()
    return Ro, Rg, o, g


CASES = [
    # (N, Kx, Ky, rotate_seed)
    (1, 5, 3, None), (2, 4, 4, 1), (3, 8, 8, None), (3, 7, 5, 2), (4, 6, 6, 3), (5, 5, 4, 4),
    (6, 4, 4, None), (7, 9, 7, 5), (8, 3, 5, 6), (9, 3, 3, 7), (10, 3, 2, None), (11, 2, 3, 8),
    (12, 3, 3, 9), (3, 1, 1, None), (4, 1, 3, None), (2, 1, 1, 3),
]


@pytest.mark.parametrize("N,Kx,Ky,rot", CASES)
@pytest.mark.parametrize("flux", [0, 1])
def test_rhs_parity_inviscid(N, Kx, Ky, rot, flux):
    p = I.random_rough(N=N, K1=Kx, seed=N * 7 + Kx, rotate_seed=rot)
    if Ky != Kx:
        p = I.random_smooth(N=N, Kx=Kx, Ky=Ky, seed=N, rotate_seed=rot)
        rng = np.random.default_rng(N)
        p.W = p.W * (1 + 0.05 * rng.uniform(-1, 1, size=p.W.shape))
    Ro, Rg, _, _ = rhs_both(p, flux=flux)
    check_rhs(Rg, Ro, p)


@pytest.mark.parametrize("N,Kx,rot", [(1, 4, None), (2, 5, 1), (3, 8, 2), (4, 6, None), (5, 4, 3),
                                      (7, 5, 4), (8, 3, 5), (12, 2, None), (3, 1, None)])
def test_rhs_parity_viscous(N, Kx, rot):
    p = I.random_rough(N=N, K1=Kx, seed=100 + N, rotate_seed=rot)
    kw = dict(flux=1, av=True, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)
    Ro, Rg, o, g = rhs_both(p, **kw)
    eo = o.epsilon()
    eg = g.epsilon().cpu().numpy()
    assert eo.max() > 0 and np.all(eo < kw["eps0"]), "the case must exercise the sine ramp of App. A"
    assert np.abs(eg - eo).max() < 1e-12 * kw["eps0"]
    check_rhs(Rg, Ro, p)


@pytest.mark.parametrize("N", [3, 5])
def test_rhs_parity_partially_viscous(N):
    """Default indicator thresholds on a dam-break-like state: only some
    elements carry viscosity, so viscous lifts cross into inviscid ones."""
    p = I.dam_break(N=N, K1=10, rotate_seed=3)
    Ro, Rg, o, g = rhs_both(p, flux=1, av=True, eps0=0.025)
    eo = o.epsilon()
    assert 0 < np.count_nonzero(eo) < p.K
    assert np.abs(g.epsilon().cpu().numpy() - eo).max() < 1e-12
    check_rhs(Rg, Ro, p)


def test_rhs_parity_lake_hump_configuration():
    """The lake-plus-hump configuration (N=3, 8x8 curved periodic quads, ES
    flux, AV, limiter), at t = 0 and after 50 oracle steps: a state near
    equilibrium, where |R| is three orders of magnitude below the term scale."""
    p = I.lake_hump(N=3, K1=8)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    o, g = pair(p, **kw)
    check_rhs(g.rhs(dev(p.W)).cpu().numpy(), o.rhs(p.W), p, label="t=0")
    W, rc, _ = o.step(p.W, 0.0, 50)
    assert rc == 0
    check_rhs(g.rhs(dev(W)).cpu().numpy(), o.rhs(W), p, W, label="50 steps")


def test_rhs_lake_hump_against_exact():
    """The GPU right-hand side against the exact (40-digit) right-hand side of
    the same float64 inputs (tests/golden/lake_hump_exact_rhs.npz, written by
    the multi-precision brute force): on this near-equilibrium state the FP64
    oracle itself is ~2e-12 of |R| from the exact result, and the GPU must be
    as close as the oracle is (both ~1e-15 of T)."""
    d = np.load(GOLDEN)
    p = I.lake_hump(N=3, K1=8)
    p.x, p.y, p.b = d["x"], d["y"], d["b"]
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True)
    o, g = pair(p, **kw)
    for lab, W, R in (("exact t=0", d["W0"], d["R0"]), ("exact 50 st", d["W50"], d["R50"])):
        Rg = g.rhs(dev(W)).cpu().numpy()
        _, sg = check_rhs(Rg, R, p, W, label=lab)
        _, so = check_rhs(o.rhs(W), R, p, W, label=lab + " orc")
        assert sg <= 4 * so + 1e-15


@pytest.mark.parametrize("N,rot", [(1, None), (3, 7), (4, 8), (7, 9), (12, None)])
def test_lake_at_rest_gpu(N, rot):
    p = I.lake_at_rest_kinked(N=N, K1=5, rotate_seed=rot)
    kw = dict(flux=1, av=True, eps0=0.05, sigma_min=-9.0, sigma_max=-8.0, limiter=True)
    o, g = pair(p, **kw)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    from parity import term_scale
    assert np.abs(Rg).max() < 1e-13 * term_scale(p)
    W = dev(p.W)
    rc, dt = g.step(W, 0.0, 20)
    Wc = W.cpu().numpy()
    assert np.abs(Wc[0] + p.b - 1.0).max() < 1e-12
    assert np.abs(Wc[1:]).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 6])
def test_limiter_parity(N):
    p = I.random_rough(N=N, K1=5, seed=40 + N, rotate_seed=N)
    rng = np.random.default_rng(N)
    h = 0.1 + 0.3 * rng.uniform(-1, 1, size=p.b.shape)
    W = np.stack([h, h * rng.uniform(-1, 1, size=h.shape), h * rng.uniform(-1, 1, size=h.shape)])
    geo = refmath.geometry(p.x, p.y, N)
    ww = refmath.quad_weights(N) * geo[4]
    mean = (W[0] * ww).sum(axis=(-2, -1)) / ww.sum(axis=(-2, -1))
    W[0] += np.maximum(0.0, 0.05 - mean)[:, None, None]
    o, g = pair(p, flux=1, limiter=True)
    Wo, rc = o.limit(W)
    Wg = dev(W)
    g.limit(Wg)
    assert rc == 0 and g.status() == 0
    assert np.abs(Wg.cpu().numpy() - Wo).max() < 1e-14


@pytest.mark.parametrize("N,k", [(3, 4), (1, 5), (2, 3)])
def test_limiter_negative_mean_status(N, k):
    """An element with a negative mean sets the status bit, also when it
    shares a warp with other elements (small N: several elements per warp)."""
    p = I.random_smooth(N=N, K1=3, seed=2)
    W = p.W.copy()
    W[0, k] = -0.5
    o, g = pair(p, limiter=True)
    _, rc = o.limit(W)
    Wg = dev(W)
    g.limit(Wg)
    assert rc == O.ERR_NEG_MEAN
    assert g.status() & 1


@pytest.mark.parametrize("N,dry", [(1, 0.2), (2, 0.0), (3, 0.3), (5, 0.2)])
def test_max_dt_parity(N, dry):
    p = I.random_rough(N=N, K1=5, seed=60 + N, rotate_seed=N, dry_fraction=dry)
    o, g = pair(p, flux=1, limiter=True, cfl=0.4)
    W, _ = o.limit(p.W)
    dco, dpo = o.max_dt(W)
    dcg, dpg = g.max_dt(dev(W))
    assert abs(dcg - dco) < 1e-13 * dco
    assert abs(dpg - dpo) < 1e-13 * dpo


@pytest.mark.parametrize("N", [2, 4])
def test_mass_entropy_parity(N):
    p = I.random_rough(N=N, K1=6, seed=70 + N, rotate_seed=N)
    o, g = pair(p)
    Wg = dev(p.W)
    mo, mg = o.mass(p.W), g.mass(Wg)
    assert np.abs(mg - mo).max() < 1e-13 * np.abs(mo).max()
    eo, eg = o.entropy(p.W), g.entropy(Wg)
    assert abs(eg - eo) < 1e-13 * abs(eo)
    # deterministic: identical on repetition; the combined call agrees
    assert g.entropy(Wg) == eg
    both = g.integrals(Wg)
    assert np.array_equal(both[:3], mg) and both[3] == eg


def test_entropy_and_velocities_wide_range_of_heights():
    """1/h is a refined hardware reciprocal on the GPU (and the division for
    subnormal h): the kinetic energy and the velocities must hold over water
    heights from 1e-300 to 1e3, including subnormal and dry nodes, against
    the oracle's plain division."""
    p = I.random_rough(N=3, K1=6, seed=11, rotate_seed=1)
    rng = np.random.default_rng(12)
    W = p.W.copy()
    h = 10.0 ** rng.uniform(-300, 3, size=W[0].shape)
    flat = h.reshape(-1)
    flat[::97] = 0.0
    flat[1::97] = 5e-320          # subnormal
    flat[2::97] = 2.0 ** -1021    # normal, near the bottom of the range
    W[0] = h
    W[1] = np.where(h > 1e-100, rng.uniform(-1, 1, size=h.shape) * h, 0.0)
    W[2] = np.where(h > 1e-100, rng.uniform(-1, 1, size=h.shape) * h, 0.0)
    o, g = pair(p)
    eo, eg = o.entropy(W), g.entropy(dev(W))
    assert abs(eg - eo) < 1e-13 * abs(eo)
    # velocities enter the right-hand side: EC flux on a flat-bottom-free
    # state is finite and matches the oracle
    Ro = o.rhs(W)
    Rg = g.rhs(dev(W)).cpu().numpy()
    assert np.isfinite(Rg).all()
    check_rhs(Rg, Ro, p, W)


def test_step_parity_lake_hump_100_lsrk():
    """Lake at rest plus hump, N=3, 8x8 curved periodic quads, ES flux, AV,
    limiter, 100 LSRK4(5) steps at CFL 0.5: relative 1e-10."""
    p = I.lake_hump(N=3, K1=8)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    o, g = pair(p, **kw)
    Wo, rco, dto = o.step(p.W, 0.0, 100)
    Wg = dev(p.W)
    rcg, dtg = g.step(Wg, 0.0, 100)
    assert rco == 0 and rcg == 0
    assert abs(dtg - dto) < 1e-12 * dto
    assert rel(Wg.cpu().numpy(), Wo) < STEP_TOL
    dW = Wg.cpu().numpy() - p.W
    assert rel(Wg.cpu().numpy() - p.W, Wo - p.W) < 1e-8 and np.abs(dW).max() > 1e-4


@pytest.mark.parametrize("N,rot", [(3, None), (4, 5)])
def test_step_parity_thacker_ssp(N, rot):
    """Wet/dry oscillating lake, SSPRK3, positivity limiter and dt restriction.

    At a wet/dry front the limiter's theta = hbar/(hbar - m) and u = hu/h at
    nearly dry nodes turn rounding-level differences of R into relative
    differences of whole elements: the oracle built as is and the same oracle
    built with FMA contraction (both correct) differ by up to 4e-11 (N=3) and
    2.4e-10 (N=4) per step and by 1.2e-8 after 40 steps on this trajectory.
    So: every step's right-hand side to 5e-14 of the term scale; every step,
    from the oracle's state, to 1e-9 relative; the whole run to 1e-6, with
    non-negative water height and conserved mass.
    """
    p = I.thacker_bowl(N=N, K1=14, rotate_seed=rot)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=1, cfl=0.3)
    o, g = pair(p, **kw)
    W, _ = o.limit(p.W)
    W0 = W.copy()
    worst_step = 0.0
    Wg_run = dev(W0)
    for _ in range(40):
        Ro = o.rhs(W)
        check_rhs(g.rhs(dev(W)).cpu().numpy(), Ro, p, W, label=f"step {_}")
        Wo, rco, dto = o.step(W, 0.0, 1)
        Wg = dev(W)
        rcg, dtg = g.step(Wg, 0.0, 1)
        assert rco == 0 and rcg == 0
        assert abs(dtg - dto) < 1e-13 * dto
        worst_step = max(worst_step, rel(Wg.cpu().numpy(), Wo))
        g.step(Wg_run, 0.0, 1)
        W = Wo
    assert worst_step < 1e-9, worst_step
    Wc = Wg_run.cpu().numpy()
    assert rel(Wc, W) < 1e-6
    assert Wc[0].min() > -1e-14
    assert abs(g.mass(Wg_run)[0] - o.mass(W0)[0]) < 1e-13 * o.mass(W0)[0]


def test_step_fixed_dt_parity_ec():
    p = I.random_smooth(N=4, K1=5, seed=3, rotate_seed=4)
    kw = dict(flux=0, rk=0)
    o, g = pair(p, **kw)
    Wo, _, _ = o.step(p.W, 1e-3, 10)
    Wg = dev(p.W)
    g.step(Wg, 1e-3, 10)
    assert rel(Wg.cpu().numpy(), Wo) < STEP_TOL


def test_step_negative_mean_rolls_back():
    """A step that drives an element mean negative returns the error code and
    restores the state at the start of the failing step."""
    p = I.random_rough(N=3, K1=4, seed=9, dry_fraction=0.5)
    o, g = pair(p, flux=1, limiter=True, rk=1)
    W0, _ = o.limit(p.W)
    Wg = dev(W0)
    swedg = swe_mod()
    rc, _ = g.step(Wg, 5.0, 3, raise_on_error=False)   # far above the admissible dt
    Wo, rco, _ = o.step(W0, 5.0, 3)
    assert rco == O.ERR_NEG_MEAN
    assert rc in (swedg.ERR_NEG_MEAN, swedg.ERR_NONFINITE)
    assert np.array_equal(Wg.cpu().numpy(), W0)


def test_create_rejects_bad_inputs():
    swedg = swe_mod()
    p = I.random_smooth(N=2, K1=2)
    E = p.EToE.copy()
    E[0, 1] = -1
    with pytest.raises(swedg.SweError) as ei:
        swedg.SweContext(p.N, p.K, p.x, p.y, E, p.EToF, p.flip, p.b, p.g)
    assert ei.value.code == swedg.ERR_ARG
    x = p.x.copy()
    x[0] = x[0][:, ::-1]  # mirror one element: negative Jacobian
    with pytest.raises(swedg.SweError) as ei:
        swedg.SweContext(p.N, p.K, x, p.y, p.EToE, p.EToF, p.flip, p.b, p.g)
    assert ei.value.code == swedg.ERR_GEOM
    with pytest.raises(swedg.SweError):
        swedg.SweContext(13, p.K, p.x, p.y, p.EToE, p.EToF, p.flip, p.b, p.g)


def test_rhs_full_size_dam_break_N7():
    """The benchmark workload (N=7 on 256x256 curved quads, 4.19M nodes, ES +
    AV): every node of the GPU right-hand side against the oracle."""
    p = I.dam_break(N=7)
    kw = dict(flux=1, av=True, eps0=0.025)
    o, g = pair(p, **kw)
    Ro = o.rhs(p.W)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    check_rhs(Rg, Ro, p)
    eo = o.epsilon()
    assert np.count_nonzero(eo) > 0
    assert np.abs(g.epsilon().cpu().numpy() - eo).max() < 1e-12


@pytest.mark.parametrize("N", [1, 7])
def test_rhs_full_size_every_element_viscous(N):
    """The degree-sweep workload with the indicator thresholds set so that
    every element carries eps0: the viscous fluxes of all elements (the list
    of viscous elements, many groups per block of the viscous-flux kernel),
    every element's viscous lifts and divergence, against the oracle."""
    K1 = int(round(2048 / (N + 1)))
    p = I.dam_break(N=N, K1=K1)
    kw = dict(flux=1, av=True, eps0=0.025, sigma_min=-301.0, sigma_max=-300.0)
    o, g = pair(p, **kw)
    Ro = o.rhs(p.W)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    assert np.all(o.epsilon() == kw["eps0"])
    assert np.array_equal(g.epsilon().cpu().numpy(), o.epsilon())
    check_rhs(Rg, Ro, p)


@pytest.mark.parametrize("N", [1, 3, 12])
def test_rhs_full_size_degree_sweep(N):
    """The degree sweep's workloads (~4.2M nodes: K1 = round(2048/(N+1))
    quads per direction), ES + AV and EC without AV: every node against the
    oracle."""
    K1 = int(round(2048 / (N + 1)))
    p = I.dam_break(N=N, K1=K1)
    for kw in (dict(flux=1, av=True, eps0=0.025), dict(flux=0)):
        o, g = pair(p, **kw)
        Ro = o.rhs(p.W)
        Rg = g.rhs(dev(p.W)).cpu().numpy()
        check_rhs(Rg, Ro, p, label=str(kw))


def test_step_full_size_dam_break_N7():
    """One time step of the benchmark (LSRK4(5), CFL 0.5, ES + AV + limiter,
    the step size from the device-side CFL/positivity reduction) at full
    size against the oracle's step."""
    p = I.dam_break(N=7)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    o, g = pair(p, **kw)
    Wo, rco, dto = o.step(p.W, 0.0, 1)
    Wg = dev(p.W)
    rcg, dtg = g.step(Wg, 0.0, 1)
    assert rco == 0 and rcg == 0
    assert abs(dtg - dto) < 1e-13 * dto
    assert rel(Wg.cpu().numpy(), Wo) < STEP_TOL


@pytest.mark.parametrize("N,flux,av", [(1, 0, False), (3, 1, True), (4, 0, False), (7, 1, True)])
def test_entropy_rate_parity(N, flux, av):
    """swe_entropy_rate against the oracle's rate; for the entropy-conservative
    scheme without viscosity the GPU's rate vanishes to rounding itself."""
    p = I.random_rough(N=N, K1=4, seed=80 + N, rotate_seed=N)
    kw = dict(flux=flux, av=av, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)
    o, g = pair(p, **kw)
    ro, so = o.entropy_rate(p.W)
    rg, sg = g.entropy_rate(dev(p.W))
    assert abs(rg - ro) < 1e-11 * so
    assert abs(sg - so) < 1e-11 * so
    if flux == 0 and not av:
        assert abs(rg) < 1e-13 * sg
    else:
        assert rg < 0


def test_entropy_rate_full_size_dam_break_N7():
    """The benchmark workload two steps after the dam release (at t = 0 the
    water is at rest and the rate is exactly zero on both sides)."""
    p = I.dam_break(N=7)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5)
    o, g = pair(p, **kw)
    W, rc, _ = o.step(p.W, 0.0, 2)
    assert rc == 0
    ro, so = o.entropy_rate(W)
    rg, sg = g.entropy_rate(dev(W))
    assert so > 0 and rg < 0
    assert abs(rg - ro) < 1e-11 * so
