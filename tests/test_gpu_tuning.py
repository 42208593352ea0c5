"""Launch shapes (swe_autotune / swe_set_tuning): every shape of the volume
kernel and of the stage update gives bitwise the same right-hand side and
steps, so the tuner is a pure performance choice."""
import numpy as np
import pytest

from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

KW = dict(flux=1, av=True, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5, limiter=True, rk=0, cfl=0.5)
SHAPES = [(v, u) for v in (64, 128, 256) for u in (2, 4, 8)]


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(W):
    return torch.from_numpy(np.ascontiguousarray(W)).cuda()


@pytest.mark.parametrize("N,K1", [(1, 9), (2, 8), (3, 7), (5, 5), (7, 5), (8, 3), (11, 2)])
def test_every_shape_is_bitwise_identical(N, K1):
    p = I.random_rough(N=N, K1=K1, seed=40 + N, dry_fraction=0.05)
    swedg = swe_mod()
    ref = swedg.SweContext.from_problem(p, **KW)
    assert ref.tuning() == (128, 4)
    W0 = dev(p.W)
    R0 = ref.rhs(W0)
    Ws0 = W0.clone()
    ref.step(Ws0, 1e-5, 3)
    c = swedg.SweContext.from_problem(p, **KW)
    for v, u in SHAPES:
        c.set_tuning(v, u)
        assert c.tuning() == (v, u)
        assert torch.equal(c.rhs(W0), R0), (v, u)
        Ws = W0.clone()
        c.step(Ws, 1e-5, 3)
        assert torch.equal(Ws, Ws0), (v, u)


def test_autotune_keeps_results_and_picks_valid_shapes():
    p = I.dam_break(N=5, K1=48)
    swedg = swe_mod()
    c = swedg.SweContext.from_problem(p, **KW)
    W0 = dev(p.W)
    R0 = c.rhs(W0)
    v, u = c.autotune(W0)
    assert (v, u) in SHAPES
    assert torch.equal(W0, dev(p.W)), "autotune must not touch the caller's state"
    assert torch.equal(c.rhs(W0), R0)


def test_set_tuning_rejects_bad_shapes():
    swedg = swe_mod()
    p = I.random_smooth(N=12, K1=2)
    c = swedg.SweContext.from_problem(p, **KW)
    # the largest staging: 19 elements of 169 nodes, 9 planes = 225.8 KB of
    # the 227 KB a block may use (valid; the results are those of 128)
    W0 = dev(p.W)
    R0 = c.rhs(W0)
    c.set_tuning(256, 4)
    assert torch.equal(c.rhs(W0), R0)
    with pytest.raises(swedg.SweError):
        c.set_tuning(96, 4)
    with pytest.raises(swedg.SweError):
        c.set_tuning(128, 3)
    c.set_tuning(64, 8)
    assert c.tuning() == (64, 8)


def test_ensemble_autotune_then_step_matches_untuned():
    probs = I.ensemble(ninst=6, seed=21, sizes=(6, 10), degrees=(3, 5, 7))
    swedg = swe_mod()
    kw = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)
    a = swedg.SweEnsemble(probs, **kw)
    b = swedg.SweEnsemble(probs, **kw)
    Wa = a.pack([p.W for p in probs])
    Wb = b.pack([p.W for p in probs])
    a.step(Wa, 0.0, 2)          # capture with the default shapes
    groups = a.autotune(Wa)     # forces a new capture
    assert len(groups) == a.ngroups
    for N, members, v, u in groups:
        assert (v, u) in SHAPES and members > 0
    a.step(Wa, 0.0, 3)
    b.step(Wb, 0.0, 5)
    assert torch.equal(Wa, Wb)


def test_timing_of_selected_kernel_classes():
    """swe_timing brackets every launch with events; swe_timing_classes only
    the launches of the chosen classes (the launch counter counts all)."""
    swedg = swe_mod()
    p = I.dam_break(N=3, K1=16)
    c = swedg.SweContext.from_problem(p, **KW)
    W = dev(p.W)
    R0 = c.rhs(W)
    c.timing(True)
    c.rhs(W)
    torch.cuda.synchronize()
    # one launch each; the viscosity class is the indicator and the viscous
    # fluxes of the listed viscous elements (two kernels)
    for name, launches in (("volume", 1), ("face", 1), ("av", 2)):
        ms, n = c.timing_read(name)
        assert n == launches and ms > 0.0, name
    c.timing(True, classes=("volume",))
    l0 = c.launches()
    assert torch.equal(c.rhs(W), R0)
    c.step(W, 0.0, 2)  # adaptive steps (CFL 0.5)
    torch.cuda.synchronize()
    ms, n = c.timing_read("volume")
    assert n == 2 * 5 + 1 and ms > 0.0
    for name in ("face", "av", "update", "prim"):
        assert c.timing_read(name)[1] == 0, name
    assert c.launches() - l0 > n
    c.timing(False)
    c.rhs(W)
    assert c.timing_read("volume")[1] == 0
