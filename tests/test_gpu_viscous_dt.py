"""The optional viscous restriction of the time step (swe_params.cfl_visc;
not in the paper): GPU time steps and trajectories against the oracle, the
ensemble against single contexts, and the full-size dam break of the
benchmark (N = 7, 4.19M nodes, eps0 = 0.025), which the paper's rule does
not keep stable over long runs, over 500 steps."""
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


@pytest.mark.parametrize("N,cv", [(1, 0.3), (3, 0.25), (5, 0.1), (7, 0.25), (12, 1.0)])
def test_max_dt_parity(N, cv):
    p = I.random_rough(N=N, K1=5, seed=80 + N, rotate_seed=N, dry_fraction=0.0)
    kw = dict(flux=1, av=True, limiter=True, cfl=0.4, cfl_visc=cv, **AV)
    o = O.Oracle(p, **kw)
    g = swe_mod().SweContext.from_problem(p, **kw)
    W, _ = o.limit(p.W)
    dco, dpo = o.max_dt(W)
    dcg, dpg = g.max_dt(dev(W))
    assert abs(dcg - dco) < 1e-13 * dco and abs(dpg - dpo) < 1e-13 * dpo
    # the restriction binds here (rough state: viscous elements)
    paper = O.Oracle(p, **dict(kw, cfl_visc=0.0)).max_dt(W)[0]
    assert dco < paper


@pytest.mark.parametrize("rk", [0, 1])
def test_step_parity_dam_break(rk):
    """20 adaptive steps of the dam break (N = 3, 16 x 16 quads,
    eps0 = 0.025) with the viscous restriction: relative 1e-10."""
    p = I.dam_break(N=3, K1=16)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=rk, cfl=0.5, cfl_visc=0.25)
    o = O.Oracle(p, **kw)
    g = swe_mod().SweContext.from_problem(p, **kw)
    Wo, rco, dto = o.step(p.W, 0.0, 20)
    Wg = dev(p.W)
    rcg, dtg = g.step(Wg, 0.0, 20)
    assert rco == 0 and rcg == 0
    assert abs(dtg - dto) < 1e-12 * dto
    err = np.abs(Wg.cpu().numpy() - Wo).max() / np.abs(Wo).max()
    assert err < 1e-10
    # the step is the viscous one, below the paper's rule (3.9e-4 against 7.5e-4)
    assert dto < 0.6 * min(O.Oracle(p, **dict(kw, cfl_visc=0.0)).max_dt(Wo))


def test_ensemble_matches_single_contexts():
    probs = I.ensemble(ninst=6, seed=12, sizes=(3, 6), degrees=(2, 3, 5))
    kw = dict(flux=1, av=True, eps0=0.03, limiter=True, rk=0, cfl=0.5, cfl_visc=0.3)
    swedg = swe_mod()
    ens = swedg.SweEnsemble(probs, **kw)
    W = ens.pack([p.W for p in probs])
    dc, dp = ens.max_dt(W)
    for i, p in enumerate(probs):
        assert (dc[i], dp[i]) == swedg.SweContext.from_problem(p, **kw).max_dt(dev(p.W))
    ens.step(W, 0.0, 3)
    for i, p in enumerate(probs):
        c = swedg.SweContext.from_problem(p, **kw)
        Ws = dev(p.W)
        c.step(Ws, 0.0, 3)
        assert torch.equal(ens.view(W, i), Ws), f"instance {i}"


def test_full_size_dam_break_stable_with_viscous_restriction():
    """The benchmark's workload (dam break, N = 7, 256 x 256 curved quads,
    4.19M nodes, ES flux, AV with eps0 = 0.025, limiter, adaptive LSRK4(5))
    with cfl_visc = 0.25, 500 asynchronous steps: every step succeeds, mass
    is conserved, the entropy falls in every step, |W| stays bounded and h
    positive (under the paper's rule alone this run's entropy grows and its
    time step collapses)."""
    swedg = swe_mod()
    p = I.dam_break(N=7, K1=256)
    kw = dict(flux=1, av=True, eps0=0.025, limiter=True, rk=0, cfl=0.5, cfl_visc=0.25)
    c = swedg.SweContext.from_problem(p, **kw)
    W = dev(p.W)
    m0 = c.integrals(W)
    res = torch.zeros((500, 6), dtype=torch.float64, device="cuda")
    for i in range(500):
        c.step_async(W, 0.0, 1, out=res[i])
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    assert np.all(r[:, 5] == 0.0)
    assert np.abs(r[:, 0] - m0[0]).max() <= 1e-12 * m0[0]
    E = np.concatenate(([m0[3]], r[:, 3]))
    assert np.all(np.diff(E) <= 1e-13 * abs(m0[3])) and E[-1] < E[0]
    assert r[:, 4].min() > 0.5 * r[0, 4]          # no collapse of the step
    assert float(W.abs().max()) < 3.0 and float(W[0].min()) > 0.0
