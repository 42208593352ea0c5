"""Standard (non-split) volume form (swe_params.volume = 1, Eq. VolInt second
line): parity of the CUDA library with the oracle's standard form on the
same seeded inputs, with the tolerances of the split form."""
import numpy as np
import pytest

from parity import check_rhs, rel
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

STEP_TOL = 1e-10


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(W):
    return torch.from_numpy(np.ascontiguousarray(W)).cuda()


def pair(prob, **kw):
    return O.Oracle(prob, **kw), swe_mod().SweContext.from_problem(prob, **kw)


@pytest.mark.parametrize("N,Kx,Ky,rot", [(1, 5, 3, None), (2, 4, 4, 1), (3, 7, 5, 2), (5, 5, 4, 4),
                                         (7, 9, 7, 5), (8, 3, 5, 6), (12, 3, 3, 9), (4, 1, 1, None)])
@pytest.mark.parametrize("flux", [0, 1])
def test_standard_rhs_parity_inviscid(N, Kx, Ky, rot, flux):
    p = I.random_smooth(N=N, Kx=Kx, Ky=Ky, seed=N + 3, rotate_seed=rot)
    rng = np.random.default_rng(N)
    p.W = p.W * (1 + 0.05 * rng.uniform(-1, 1, size=p.W.shape))
    o, g = pair(p, flux=flux, volume=1)
    Ro = o.rhs(p.W)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    check_rhs(Rg, Ro, p)


@pytest.mark.parametrize("N,Kx,rot", [(1, 4, None), (3, 6, 2), (5, 4, 3), (7, 5, 4), (11, 2, None)])
def test_standard_rhs_parity_viscous(N, Kx, rot):
    p = I.random_rough(N=N, K1=Kx, seed=200 + N, rotate_seed=rot)
    kw = dict(flux=1, av=True, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5, volume=1)
    o, g = pair(p, **kw)
    Ro = o.rhs(p.W)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    eo = o.epsilon()
    assert eo.max() > 0
    check_rhs(Rg, Ro, p)


def test_standard_step_parity_lake_hump():
    p = I.lake_hump(N=4, K1=6)
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5, volume=1)
    o, g = pair(p, **kw)
    Wo, rc, dto = o.step(p.W, 0.0, 40)
    assert rc == 0
    Wg = dev(p.W)
    _, dtg = g.step(Wg, 0.0, 40)
    assert rel(Wg.cpu().numpy(), Wo) < STEP_TOL
    assert abs(dtg - dto) <= 1e-12 * dto


def test_standard_form_is_not_well_balanced():
    """Lake at rest over a kinked bottom: the split form keeps R = 0, the
    standard form does not (on the GPU as in the oracle)."""
    p = I.lake_at_rest_kinked(N=4, K1=5)
    swedg = swe_mod()
    Rs = swedg.SweContext.from_problem(p, flux=1).rhs(dev(p.W)).cpu().numpy()
    Rt = swedg.SweContext.from_problem(p, flux=1, volume=1).rhs(dev(p.W)).cpu().numpy()
    assert np.abs(Rs).max() < 1e-11
    assert np.abs(Rt).max() > 1e-6
    Ro = O.Oracle(p, flux=1, volume=1).rhs(p.W)
    check_rhs(Rt, Ro, p)


def test_standard_rhs_full_size_dam_break_N7():
    """The benchmark workload in the standard form (ES interface flux, AV):
    every node against the oracle."""
    p = I.dam_break(N=7)
    kw = dict(flux=1, av=True, eps0=0.025, volume=1)
    o, g = pair(p, **kw)
    Ro = o.rhs(p.W)
    Rg = g.rhs(dev(p.W)).cpu().numpy()
    check_rhs(Rg, Ro, p)


def test_create_rejects_bad_volume_form():
    swedg = swe_mod()
    p = I.random_smooth(N=2, K1=2)
    with pytest.raises(swedg.SweError):
        swedg.SweContext.from_problem(p, volume=2)
