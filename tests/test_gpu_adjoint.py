"""The library's adjoint (swe_rhs_adjoint, swe_step_adjoint,
swe_gauge_misfit) against the CPU reference adjoint (oracle/adjoint_ref.py,
torch autograd of the oracle's scheme, itself pinned to central differences
of the oracle) and against central differences of the oracle and of the
library's own forward run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from oracle.adjoint_ref import LSRK_A, LSRK_B, Twin  # noqa: E402
gauge_weights = I.gauge_weights

AV = dict(eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)
TOL = 1e-11


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = [
    ("rough_es", lambda: I.random_rough(N=3, K1=4, seed=1, rotate_seed=2), dict(flux=1)),
    ("rough_ec_n1", lambda: I.random_rough(N=1, K1=5, seed=2, rotate_seed=3), dict(flux=0)),
    ("smooth_n7", lambda: I.random_smooth(N=7, K1=3, seed=3, rotate_seed=4), dict(flux=1)),
    ("walls_n5", lambda: I.random_walls(N=5, Kx=3, Ky=3, seed=4, rotate_seed=5), dict(flux=1)),
    ("av_n4", lambda: I.random_rough(N=4, K1=3, seed=5, rotate_seed=6), dict(flux=1, av=True, **AV)),
    ("av_walls_n3", lambda: I.random_walls(N=3, Kx=4, Ky=3, seed=6, rotate_seed=7), dict(flux=1, av=True, **AV)),
    ("dry_n3", lambda: I.random_rough(N=3, K1=4, seed=7, dry_fraction=0.2), dict(flux=1, av=True, **AV)),
    # viscous elements next to inviscid ones, nearly dry nodes at a wet/dry front
    ("thacker_front", lambda: I.thacker_bowl(N=3, K1=8), dict(flux=1, av=True, eps0=0.01)),
    # 2^20 nodes: a context this large runs the source coefficients onto b on
    # its second stream, beside the reverse interface flux and viscosity
    ("dam_break_2p20", lambda: I.dam_break(N=7, K1=128), dict(flux=1, av=True, eps0=0.025)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_rhs_adjoint_matches_reference(name, make, kw):
    p = make()
    swedg = swe_mod()
    c = swedg.SweContext.from_problem(p, **kw)
    W = dev(p.W)
    rng = np.random.default_rng(17)
    Rbar = rng.standard_normal(p.W.shape)
    Wbar, bbar = c.rhs_adjoint(W, dev(Rbar))
    eps = c.epsilon().cpu().numpy() if kw.get("av") else None
    if kw.get("av"):
        assert eps.max() > 0
    if name == "thacker_front":
        assert eps.min() == 0.0
    t = Twin(p, flux=kw["flux"], av=kw.get("av", False))
    Wt = torch.tensor(p.W, requires_grad=True)
    bt = torch.tensor(p.b, requires_grad=True)
    (t.rhs(Wt, bt, eps) * torch.tensor(Rbar)).sum().backward()
    assert rel(Wbar.cpu().numpy(), Wt.grad.numpy()) < TOL
    assert rel(bbar.cpu().numpy(), bt.grad.numpy()) < TOL
    # accumulation: a second call adds the same amounts
    Wbar2, bbar2 = c.rhs_adjoint(W, dev(Rbar), Wbar.clone(), bbar.clone())
    assert rel(Wbar2.cpu().numpy(), 2 * Wt.grad.numpy()) < TOL


def reference_step_grad(p, kw, W0, dt, wbar, eps_of):
    """Twin gradient of <wbar, step(W0)> with the stage decisions of the twin's
    own forward pass; eps_of(state) gives the stage viscosities."""
    t = Twin(p, flux=kw["flux"], av=kw.get("av", False), limiter=kw.get("limiter", False), rk=kw.get("rk", 0))
    b = torch.tensor(p.b, requires_grad=True)
    eps, plans = [], []
    with torch.no_grad():
        W = torch.tensor(W0)
        if t.rk == 0:
            Kr = torch.zeros_like(W)
            for st in range(5):
                eps.append(eps_of(W.numpy()))
                Kr = LSRK_A[st] * Kr + dt * t.rhs(W, b, eps[-1])
                W = W + LSRK_B[st] * Kr
                plans.append(t.limiter_plan(W) if t.limiter else None)
                if t.limiter:
                    W = t.limit(W, plans[-1])
        else:
            Wn = W
            for a, c in ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)):
                eps.append(eps_of(W.numpy()))
                W = a * Wn + c * (W + dt * t.rhs(W, b, eps[-1]))
                plans.append(t.limiter_plan(W) if t.limiter else None)
                if t.limiter:
                    W = t.limit(W, plans[-1])
    Wt = torch.tensor(W0, requires_grad=True)
    out = t.step(Wt, b, dt, eps, plans)
    (out * torch.tensor(wbar)).sum().backward()
    return Wt.grad.numpy(), b.grad.numpy(), out.detach().numpy(), plans


@pytest.mark.parametrize("case", ["lsrk_av", "ssp_limiter_wetdry", "ssp_walls"])
def test_step_adjoint_matches_reference(case):
    swedg = swe_mod()
    if case == "lsrk_av":
        p = I.random_smooth(N=3, K1=4, seed=9, rotate_seed=5)
        kw = dict(flux=1, av=True, rk=0, limiter=True, **AV)
        W0 = p.W
    elif case == "ssp_limiter_wetdry":
        p = I.thacker_bowl(N=3, K1=8)
        kw = dict(flux=1, av=True, rk=1, limiter=True, eps0=0.01)
        W0, _ = O.Oracle(p, **kw).limit(p.W)
    else:
        p = I.random_walls(N=4, Kx=3, Ky=3, seed=2, rough=False)
        kw = dict(flux=1, av=True, rk=1, limiter=True, **AV)
        W0 = p.W
    c = swedg.SweContext.from_problem(p, **kw)
    dt = min(c.max_dt(dev(W0)))
    probe = swedg.SweContext.from_problem(p, **kw)

    def eps_of(Wst):
        probe.rhs(dev(Wst))
        return probe.epsilon().cpu().numpy()

    rng = np.random.default_rng(5)
    wbar = rng.standard_normal(W0.shape)
    gW, gb, out, plans = reference_step_grad(p, kw, W0, dt, wbar, eps_of)
    if case == "ssp_limiter_wetdry":
        assert any(bool(q[0].any()) for q in plans), "the limiter must act"
    Wg = dev(W0)
    c.step(Wg, dt, 1)
    assert rel(Wg.cpu().numpy(), out) < 1e-12
    Wbar = dev(wbar)
    bbar = torch.zeros_like(dev(p.b))
    c.step_adjoint(dev(W0), dt, Wbar, bbar)
    # with the limiter active the derivatives carry 1/h at nodes just above
    # h_tol and theta's d/dm0, d/dy ~ 1/(mean - min)^2 in nearly dry elements,
    # which amplify the 1e-14 forward differences between the two sides
    tol = 1e-10 if case == "lsrk_av" else 5e-9
    assert rel(Wbar.cpu().numpy(), gW) < tol
    assert rel(bbar.cpu().numpy(), gb) < tol


def _gauges(p, G, seed):
    rng = np.random.default_rng(seed)
    lo = np.array([p.x.min(), p.y.min()]) + 0.1
    hi = np.array([p.x.max(), p.y.max()]) - 0.1
    pts = rng.uniform(lo, hi, size=(G, 2))
    gw = gauge_weights(p, pts)
    elem = torch.tensor([k for k, _ in gw], dtype=torch.int32, device="cuda")
    wts = torch.tensor(np.stack([w.reshape(-1) for _, w in gw]), dtype=torch.float64, device="cuda")
    return elem, wts


def _target(p, kw, elem, wts, nsteps, seed):
    """Gauge record of a run over a perturbed bathymetry."""
    swedg = swe_mod()
    rng = np.random.default_rng(seed)
    a, bb = rng.uniform(0.01, 0.03, size=2)
    q = I.Problem(p.name, p.N, p.Kx, p.Ky, p.x, p.y,
                  p.b + a * np.sin(np.pi * p.x) * np.sin(np.pi * p.y) + bb * np.sin(2 * np.pi * p.y),
                  p.W, p.EToE, p.EToF, p.flip, p.g)
    ct = swedg.SweContext.from_problem(q, **kw)
    rec = torch.zeros(nsteps, elem.numel(), dtype=torch.float64, device="cuda")
    run = swedg.GaugeLoss(ct, elem, wts, torch.zeros_like(rec), nsteps)
    run.forward(dev(p.W), record=rec)
    return rec


def test_gauge_loss_gradient_small_vs_reference_and_fd():
    """N = 4 on 6 x 6 quads, 12 LSRK4(5) steps, 8 gauges, checkpoints every 5
    steps: dL/dW0 and dL/db against the CPU reference adjoint through the same
    steps and decisions, and a directional derivative against central
    differences of the oracle with the same step sizes."""
    swedg = swe_mod()
    p = I.lake_hump(N=4, K1=6, amp=0.05)
    kw = dict(flux=1, av=True, eps0=0.02, sigma_min=-301.0, sigma_max=-300.0, rk=0, cfl=0.5)
    c = swedg.SweContext.from_problem(p, **kw)
    elem, wts = _gauges(p, 8, seed=1)
    T = 12
    target = _target(p, kw, elem, wts, T, seed=2)
    run = swedg.GaugeLoss(c, elem, wts, target, T, checkpoint=5)
    loss = float(run.forward(dev(p.W)))
    Wbar, bbar = run.backward()
    dts = run.dts
    # CPU reference through the same steps
    t = Twin(p, flux=1, av=True, rk=0)
    eflat = np.full(p.K, 0.02)
    Wt = torch.tensor(p.W, requires_grad=True)
    bt = torch.tensor(p.b, requires_grad=True)
    tg = target.cpu().numpy()
    el = elem.cpu().numpy()
    wt = torch.tensor(wts.cpu().numpy().reshape(-1, p.N + 1, p.N + 1))
    W = Wt
    L = 0.0
    for s in range(T):
        W = t.step(W, bt, dts[s], [eflat] * 5, [None] * 5)
        hg = (W[0][el] * wt).sum(dim=(1, 2))
        L = L + ((hg - torch.tensor(tg[s])) ** 2).sum()
    assert abs(float(L.detach()) - loss) < 1e-12 * abs(loss)
    L.backward()
    assert rel(Wbar.cpu().numpy(), Wt.grad.numpy()) < 1e-9
    assert rel(bbar.cpu().numpy(), bt.grad.numpy()) < 1e-9
    # central differences of the oracle along one direction of W0 (fixed step sizes)
    o = O.Oracle(p, **kw)
    rng = np.random.default_rng(8)
    d = rng.standard_normal(p.W.shape) * np.array([0.01, 0.01, 0.01])[:, None, None, None]

    def oracle_loss(W0):
        W = W0.copy()
        tot = 0.0
        for s in range(T):
            W, rc, _ = o.step(W, dts[s], 1)
            assert rc == 0
            hg = (W[0][el] * wt.numpy()).sum(axis=(1, 2))
            tot += float(((hg - tg[s]) ** 2).sum())
        return tot

    h = 1e-5
    fd = (oracle_loss(p.W + h * d) - oracle_loss(p.W - h * d)) / (2 * h)
    g = float((Wbar.cpu().numpy() * d).sum())
    assert abs(g - fd) < 1e-6 * max(abs(fd), 1e-12), (g, fd)


def test_adjoint_configuration_full_size():
    """The adjoint workload: N = 4 on 64 x 64 curved quads, 200 adaptive
    LSRK4(5) steps, 64 seeded gauges against a run over a perturbed
    bathymetry, checkpoints every 20 steps. The gradient's directional
    derivatives along W0 and b match central differences of the library's
    own forward run with the same step sizes."""
    swedg = swe_mod()
    p = I.lake_hump(N=4, K1=64, amp=0.05)
    # viscosity on in every element (the flat branch of the switch, which
    # the adjoint holds fixed)
    kw = dict(flux=1, av=True, eps0=0.01, sigma_min=-301.0, sigma_max=-300.0, rk=0, cfl=0.5)
    c = swedg.SweContext.from_problem(p, **kw)
    elem, wts = _gauges(p, 64, seed=3)
    T = 200
    target = _target(p, kw, elem, wts, T, seed=4)
    run = swedg.GaugeLoss(c, elem, wts, target, T, checkpoint=20)
    loss = float(run.forward(dev(p.W)))
    assert loss > 0
    Wbar, bbar = run.backward()
    dts = run.dts

    def fwd_loss(W0, ctx):
        W = W0.clone()
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        for s in range(T):
            ctx.step(W, dts[s], 1)
            ctx.gauge_misfit(W, elem, wts, target=target[s], loss=tot)
        return float(tot[0])

    rng = np.random.default_rng(9)
    d = dev(rng.standard_normal(p.W.shape) * np.array([1e-3, 1e-3, 1e-3])[:, None, None, None])
    h = 1e-4
    fd = (fwd_loss(dev(p.W) + h * d, c) - fwd_loss(dev(p.W) - h * d, c)) / (2 * h)
    g = float((Wbar * d).sum())
    assert abs(g - fd) < 1e-5 * abs(fd), (g, fd)
    db = 1e-3 * np.sin(2 * np.pi * p.x) * np.cos(np.pi * p.y)
    hb = 1e-3

    def b_loss(sign):
        q = I.Problem(p.name, p.N, p.Kx, p.Ky, p.x, p.y, p.b + sign * hb * db, p.W, p.EToE, p.EToF, p.flip, p.g)
        return fwd_loss(dev(p.W), swedg.SweContext.from_problem(q, **kw))

    fdb = (b_loss(1) - b_loss(-1)) / (2 * hb)
    gb = float((bbar.cpu().numpy() * db).sum())
    assert abs(gb - fdb) < 1e-4 * abs(fdb), (gb, fdb)
