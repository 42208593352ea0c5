"""Recorded steps (swe_adjoint_slots, swe_step_record,
swe_step_adjoint_recorded): a recorded step is swe_step's step bit for bit,
its reverse sweep is swe_step_adjoint's bit for bit, and a gauge-loss
gradient through recorded segments equals the one that recomputes every
step in its step adjoint."""
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


def case(name):
    if name == "lsrk_av":
        p = I.random_smooth(N=3, K1=4, seed=9, rotate_seed=5)
        return p, dict(flux=1, av=True, rk=0, limiter=True, **AV), p.W
    if name == "ssp_limiter_wetdry":
        p = I.thacker_bowl(N=3, K1=8)
        kw = dict(flux=1, av=True, rk=1, limiter=True, eps0=0.01)
        return p, kw, O.Oracle(p, **kw).limit(p.W)[0]
    p = I.random_walls(N=4, Kx=3, Ky=3, seed=2, rough=False)
    return p, dict(flux=1, av=True, rk=1, limiter=True, **AV), p.W


@pytest.mark.parametrize("name", ["lsrk_av", "ssp_limiter_wetdry", "ssp_walls"])
def test_recorded_step_and_reverse_equal_the_plain_ones(name):
    swedg = swe_mod()
    p, kw, W0 = case(name)
    c = swedg.SweContext.from_problem(p, **kw)
    dt = min(c.max_dt(dev(W0)))
    c.adjoint_slots(3)
    Wa = dev(W0)
    c.step(Wa, dt, 1)
    Wr = dev(W0)
    c.step_record(Wr, dt, 2)
    assert torch.equal(Wa, Wr)
    rng = np.random.default_rng(3)
    wbar = rng.standard_normal(W0.shape)
    A, Ab = dev(wbar), torch.zeros_like(dev(p.b))
    c.step_adjoint(dev(W0), dt, A, Ab)   # records in slot 0, leaves slot 2 alone
    B, Bb = dev(wbar), torch.zeros_like(dev(p.b))
    c.step_adjoint_recorded(2, dt, B, Bb)
    assert torch.equal(A, B) and torch.equal(Ab, Bb)


def test_record_slot_range_and_failed_step():
    swedg = swe_mod()
    p = I.random_rough(N=3, K1=4, seed=9, dry_fraction=0.5)
    kw = dict(flux=1, limiter=True, rk=1)
    c = swedg.SweContext.from_problem(p, **kw)
    W0, _ = O.Oracle(p, **kw).limit(p.W)
    c.adjoint_slots(2)
    W = dev(W0)
    with pytest.raises(swedg.SweError) as e:
        c.step_record(W, 1e-3, 2)
    assert e.value.code == swedg.ERR_ARG
    with pytest.raises(swedg.SweError) as e:
        c.step_adjoint_recorded(-1, 1e-3, W)
    assert e.value.code == swedg.ERR_ARG
    # far above the admissible step size: the step fails and W is restored
    with pytest.raises(swedg.SweError) as e:
        c.step_record(W, 5.0, 1)
    assert e.value.code in (swedg.ERR_NEG_MEAN, swedg.ERR_NONFINITE)
    assert np.array_equal(W.cpu().numpy(), W0)


def test_gauge_loss_recorded_equals_recomputed():
    swedg = swe_mod()
    p = I.lake_hump(N=4, K1=6, amp=0.05)
    kw = dict(flux=1, av=True, eps0=0.02, sigma_min=-301.0, sigma_max=-300.0, rk=0, cfl=0.5)
    c = swedg.SweContext.from_problem(p, **kw)
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.2, 1.8, size=(6, 2))
    gw = I.gauge_weights(p, pts)
    elem = torch.tensor([k for k, _ in gw], dtype=torch.int32, device="cuda")
    wts = torch.tensor(np.stack([w.reshape(-1) for _, w in gw]), dtype=torch.float64, device="cuda")
    T = 11
    target = torch.full((T, len(gw)), 0.9, dtype=torch.float64, device="cuda")
    run = swedg.GaugeLoss(c, elem, wts, target, T, checkpoint=4)
    run.forward(dev(p.W))
    Wa, ba = run.backward(recorded=True)
    Wb, bb = run.backward(recorded=False)
    assert torch.equal(Wa, Wb) and torch.equal(ba, bb)
    assert float(Wa.abs().max()) > 0 and float(ba.abs().max()) > 0
