"""Pins of the CPU reference adjoint (oracle/adjoint_ref.py): its forward
operator is the oracle's to rounding, and its torch.autograd derivatives
match central finite differences of the oracle itself (orc.c), on states
where the decisions the adjoint holds fixed (viscosity switch, limiter
active set, h_tol cut, dt) do not change under the perturbation."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
from oracle.adjoint_ref import LSRK_A as O_LSRK_A, LSRK_B as O_LSRK_B  # noqa: E402
from oracle.adjoint_ref import Twin  # noqa: E402
gauge_weights = I.gauge_weights

AV_FLAT = dict(eps0=0.02, sigma_min=-301.0, sigma_max=-300.0)  # eps = eps0 in every element


def _problems():
    return [
        ("rough", I.random_rough(N=3, K1=3, seed=1, rotate_seed=2), dict(flux=1)),
        ("rough_ec", I.random_rough(N=4, K1=3, seed=2, rotate_seed=3), dict(flux=0)),
        ("walls", I.random_walls(N=3, Kx=3, Ky=3, seed=3, rotate_seed=4), dict(flux=1)),
        ("rough_av", I.random_rough(N=2, K1=3, seed=5, rotate_seed=1), dict(flux=1, av=True, **AV_FLAT)),
        ("walls_av", I.random_walls(N=5, Kx=3, Ky=2, seed=6, rotate_seed=7), dict(flux=1, av=True, **AV_FLAT)),
    ]


def twin_of(p, kw):
    return Twin(p, flux=kw["flux"], av=kw.get("av", False), limiter=kw.get("limiter", False),
                rk=kw.get("rk", 0))


@pytest.mark.parametrize("name,p,kw", _problems(), ids=[c[0] for c in _problems()])
def test_twin_rhs_equals_oracle(name, p, kw):
    o = O.Oracle(p, **kw)
    Ro = o.rhs(p.W)
    eps = o.epsilon() if kw.get("av") else None
    Rt = twin_of(p, kw).rhs(torch.tensor(p.W), torch.tensor(p.b), eps).numpy()
    assert np.abs(Rt - Ro).max() < 1e-13 * np.abs(Ro).max()


def _fd(fun, x, d, h):
    return (fun(x + h * d) - fun(x - h * d)) / (2 * h)


@pytest.mark.parametrize("name,p,kw", _problems(), ids=[c[0] for c in _problems()])
def test_twin_rhs_vjp_matches_oracle_fd(name, p, kw):
    rng = np.random.default_rng(11)
    o = O.Oracle(p, **kw)
    o.rhs(p.W)
    eps = o.epsilon() if kw.get("av") else None
    t = twin_of(p, kw)
    rbar = rng.standard_normal(p.W.shape)
    dW = rng.standard_normal(p.W.shape) * np.abs(p.W).max(axis=(1, 2, 3), keepdims=True)
    db = rng.standard_normal(p.b.shape)
    W = torch.tensor(p.W, requires_grad=True)
    b = torch.tensor(p.b, requires_grad=True)
    (t.rhs(W, b, eps) * torch.tensor(rbar)).sum().backward()
    gW = float((W.grad.numpy() * dW).sum())
    h = 1e-6
    fdW = float((rbar * _fd(lambda x: o.rhs(x), p.W, dW, h)).sum())
    assert abs(gW - fdW) < 1e-7 * max(abs(gW), 1.0) * 10
    # bathymetry: the oracle's mesh is rebuilt for each perturbed b
    def rhs_b(bb):
        q = I.Problem(p.name, p.N, p.Kx, p.Ky, p.x, p.y, bb, p.W, p.EToE, p.EToF, p.flip, p.g)
        return O.Oracle(q, **kw).rhs(p.W)
    gb = float((b.grad.numpy() * db).sum())
    fdb = float((rbar * _fd(rhs_b, p.b, db, h)).sum())
    assert abs(gb - fdb) < 1e-6 * max(abs(gb), 1.0)


def record_step(t, o, W, b, dt):
    """Decisions of one step (element viscosities from the oracle's indicator
    and limiter plans, per stage) from an undifferentiated pass."""
    eps, plans = [], []

    def stage_eps(Wst):
        o.rhs(Wst.numpy())
        return o.epsilon() if t.av else None

    with torch.no_grad():
        if t.rk == 0:
            Kr = torch.zeros_like(W)
            for st in range(5):
                eps.append(stage_eps(W))
                Kr = O_LSRK_A[st] * Kr + dt * t.rhs(W, b, eps[-1])
                W = W + O_LSRK_B[st] * Kr
                plans.append(t.limiter_plan(W) if t.limiter else None)
                if t.limiter:
                    W = t.limit(W, plans[-1])
        else:
            Wn = W
            for a, c in ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)):
                eps.append(stage_eps(W))
                W = a * Wn + c * (W + dt * t.rhs(W, b, eps[-1]))
                plans.append(t.limiter_plan(W) if t.limiter else None)
                if t.limiter:
                    W = t.limit(W, plans[-1])
    return eps, plans, W


@pytest.mark.parametrize("rk,limiter", [(0, False), (1, True)])
def test_twin_steps_vjp_matches_oracle_fd(rk, limiter):
    """Three steps with fixed dt; with SSPRK3 and the limiter on a wet/dry
    state whose limited elements and minimum nodes stay put under the
    perturbation."""
    if limiter:
        p = I.thacker_bowl(N=3, K1=6)
        kw = dict(flux=1, av=True, limiter=True, rk=1, **AV_FLAT)
        W0, _ = O.Oracle(p, **kw).limit(p.W)
    else:
        p = I.random_smooth(N=3, K1=3, seed=9, rotate_seed=5)
        kw = dict(flux=1, av=True, rk=0, **AV_FLAT)
        W0 = p.W
    o = O.Oracle(p, **kw)
    dt = 0.5 * min(o.max_dt(W0))
    t = twin_of(p, kw)
    b = torch.tensor(p.b)
    decisions = []
    Wd = torch.tensor(W0)
    for _ in range(3):
        e, pl, Wd = record_step(t, o, Wd, b, dt)
        decisions.append((e, pl))
    if limiter:
        assert any(bool(q[0].any()) for _, pl in decisions for q in pl), "the limiter must be active"
    W = torch.tensor(W0, requires_grad=True)
    Wt = W
    for e, pl in decisions:
        Wt = t.step(Wt, b, dt, e, pl)
    assert np.abs(Wt.detach().numpy() - o.step(W0, dt, 3)[0]).max() < 1e-12 * np.abs(W0).max()
    rng = np.random.default_rng(3)
    wbar = rng.standard_normal(W0.shape)
    (Wt * torch.tensor(wbar)).sum().backward()
    dW = rng.standard_normal(W0.shape) * np.where(W0[0] > 0.05, 1.0, 0.0)[None]
    g = float((W.grad.numpy() * dW).sum())
    h = 1e-7
    Wp, rcp, _ = o.step(W0 + h * dW, dt, 3)
    Wm, rcm, _ = o.step(W0 - h * dW, dt, 3)
    assert rcp == 0 and rcm == 0
    fd = float((wbar * (Wp - Wm)).sum() / (2 * h))
    assert abs(g - fd) < 1e-6 * max(abs(g), 1.0), (g, fd)


def test_gauge_weights_interpolate_polynomials_exactly():
    p = I.random_smooth(N=4, K1=3, seed=1, rotate_seed=3)
    # the element map itself is a degree-N polynomial, so interpolating x and
    # y at a point must return the point
    rng = np.random.default_rng(0)
    pts = rng.uniform(0.1, 1.9, size=(10, 2))
    W = gauge_weights(p, pts)
    for (k, wts), (px, py) in zip(W, pts):
        assert abs((wts * p.x[k]).sum() - px) < 1e-12
        assert abs((wts * p.y[k]).sum() - py) < 1e-12
        assert abs(wts.sum() - 1.0) < 1e-13
