"""Solid walls (EToE = -1) on the GPU: parity with the oracle's walls, and the
paper's wall-bounded dam breaks (Sec. 6.1.1, Sec. 6.3) run on the library."""
import numpy as np
import pytest

from parity import check_rhs, rel
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]



def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(W):
    return torch.from_numpy(np.ascontiguousarray(W)).cuda()


def pair(prob, **kw):
    return O.Oracle(prob, **kw), swe_mod().SweContext.from_problem(prob, **kw)


CASES = [(1, 4, 3, (True, True), None), (2, 3, 3, (True, False), 1), (3, 5, 4, (True, True), 2),
         (5, 3, 4, (False, True), 3), (7, 4, 3, (True, True), 4), (12, 2, 2, (True, True), None)]


@pytest.mark.parametrize("N,Kx,Ky,walls,rot", CASES)
@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("volume", [0, 1])
def test_wall_rhs_parity(N, Kx, Ky, walls, rot, flux, volume):
    p = I.random_walls(N=N, Kx=Kx, Ky=Ky, seed=N + 50, rotate_seed=rot, walls=walls)
    o, g = pair(p, flux=flux, volume=volume)
    check_rhs(g.rhs(dev(p.W)).cpu().numpy(), o.rhs(p.W), p)


@pytest.mark.parametrize("N,Kx,Ky,walls,rot", CASES)
def test_wall_rhs_parity_viscous(N, Kx, Ky, walls, rot):
    p = I.random_walls(N=N, Kx=Kx, Ky=Ky, seed=N + 60, rotate_seed=rot, walls=walls)
    kw = dict(flux=1, av=True, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)
    o, g = pair(p, **kw)
    Ro = o.rhs(p.W)
    assert o.epsilon().max() > 0
    check_rhs(g.rhs(dev(p.W)).cpu().numpy(), Ro, p)


@pytest.mark.parametrize("N", [2, 4])
def test_wall_max_dt_parity(N):
    p = I.random_walls(N=N, Kx=4, Ky=4, seed=N, rough=False)
    o, g = pair(p, flux=1, limiter=True)
    dco, dpo = o.max_dt(p.W)
    dcg, dpg = g.max_dt(dev(p.W))
    assert abs(dcg - dco) <= 1e-13 * dco and abs(dpg - dpo) <= 1e-13 * dpo


def test_wall_lake_at_rest_steps():
    p = I.lake_at_rest_walls(N=4, Kx=6, Ky=5, rotate_seed=3)
    g = swe_mod().SweContext.from_problem(p, flux=1, av=True, eps0=0.05, sigma_min=-9.0, sigma_max=-8.0,
                                          limiter=True)
    W = dev(p.W)
    g.step(W, 0.0, 50)
    Wc = W.cpu().numpy()
    assert np.abs(Wc[0] + p.b - 1.0).max() < 1e-12
    assert np.abs(Wc[1:]).max() < 1e-12


def test_wall_step_parity_100_lsrk():
    p = I.random_walls(N=3, Kx=6, Ky=5, seed=4, rough=False, rotate_seed=8)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    o, g = pair(p, **kw)
    Wo, rc, _ = o.step(p.W, 0.0, 100)
    assert rc == 0
    Wg = dev(p.W)
    g.step(Wg, 0.0, 100)
    assert rel(Wg.cpu().numpy(), Wo) < 1e-10


def test_dry_dam_break_paper_configuration():
    """Sec. 6.1.1 as stated: N = 3, 50 x 50 Cartesian quads on [-20,20]^2,
    walls at x = +-20, periodic in y, h = 10 | 0, eps0 = 0.1, g = 9.81;
    SSPRK3 with the positivity limiter at CFL 0.2. Every step: the GPU step
    from the oracle's state matches the oracle's step (wet/dry tolerance of
    the Thacker case) for the first 10 steps; over 300 steps on the GPU the
    mass is conserved to round-off, h >= 0 and the entropy decreases."""
    p = I.dry_dam_break(N=3, K1=50)
    kw = dict(flux=1, av=True, eps0=0.1, limiter=True, rk=1, cfl=0.2)
    o, g = pair(p, **kw)
    W = p.W.copy()
    for _ in range(10):
        Wo, rco, dto = o.step(W, 0.0, 1)
        Wg = dev(W)
        rcg, dtg = g.step(Wg, 0.0, 1)
        assert rco == 0 and rcg == 0
        assert abs(dtg - dto) < 1e-12 * dto
        assert rel(Wg.cpu().numpy(), Wo) < 1e-9
        W = Wo
    Wg = dev(p.W)
    m0, _, _, E0 = g.integrals(Wg)
    for _ in range(300):
        rc, _ = g.step(Wg, 0.0, 1)
        assert rc == 0
    m1, _, _, E1 = g.integrals(Wg)
    assert abs(m1 - m0) < 1e-12 * m0
    assert float(Wg[0].min()) >= -1e-14 * float(Wg[0].max())  # the limited minimum lands on 0 up to rounding
    assert E1 < E0


def test_three_mound_dam_break_paper_configuration():
    """Sec. 6.3 as stated: N = 3 (the figure's degree), 150 x 100 quads on
    [0,75] x [0,45] closed by walls, h = 1.875 for x < 16, three conical
    mounds, eps0 = 0.2. Per-step parity with the oracle for 5 steps, then
    200 GPU steps keep mass and h >= 0."""
    p = I.three_mound_dam_break(N=3)
    kw = dict(flux=1, av=True, eps0=0.2, limiter=True, rk=1, cfl=0.2)
    o, g = pair(p, **kw)
    W = p.W.copy()
    for _ in range(5):
        Wo, rco, dto = o.step(W, 0.0, 1)
        Wg = dev(W)
        rcg, dtg = g.step(Wg, 0.0, 1)
        assert rco == 0 and rcg == 0
        assert rel(Wg.cpu().numpy(), Wo) < 1e-9
        W = Wo
    Wg = dev(p.W)
    m0 = g.integrals(Wg)[0]
    g.step(Wg, 0.0, 200)
    assert abs(g.integrals(Wg)[0] - m0) < 1e-12 * m0
    assert float(Wg[0].min()) >= -1e-14 * float(Wg[0].max())  # the limited minimum lands on 0 up to rounding


def test_ensemble_with_walled_members_matches_single_contexts():
    probs = [I.random_walls(N=3, Kx=4, Ky=3, seed=1, rough=False),
             I.lake_hump(N=3, K1=4),
             I.random_walls(N=5, Kx=3, Ky=3, seed=2, rough=False, walls=(True, False))]
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    swedg = swe_mod()
    ens = swedg.SweEnsemble(probs, **kw)
    W = ens.pack([p.W for p in probs])
    R = ens.rhs(W)
    _, dts = ens.step(W, 0.0, 5)
    for i, p in enumerate(probs):
        c = swedg.SweContext.from_problem(p, **kw)
        Ws = dev(p.W)
        assert torch.equal(c.rhs(Ws), ens.view(R, i))
        _, d = c.step(Ws, 0.0, 5)
        assert d == dts[i]
        assert torch.equal(ens.view(W, i), Ws)
