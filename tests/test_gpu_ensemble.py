"""Ensembles (swe_ens_*): many independent meshes of mixed degree and size in
one state buffer, stepped by one CUDA graph per step.

Every kernel evaluates each element, face and node of an instance exactly as
for a single context, so the ensemble's right-hand side and steps are
compared bitwise with single contexts, and single contexts are compared with
the oracle (here for one instance directly, elsewhere for every kernel).
"""
import numpy as np
import pytest

from parity import check_rhs, rel
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

KW = dict(flux=1, av=True, eps0=0.01, limiter=True, rk=0, cfl=0.5)


def swe_mod():
    from paper_1804_02221_gb300 import swedg
    return swedg


def dev(W):
    return torch.from_numpy(np.ascontiguousarray(W)).cuda()


@pytest.fixture(scope="module")
def small():
    """Nine uneven members: degrees 2, 3 and 5, meshes of 3x3 to 7x7 quads."""
    probs = I.ensemble(ninst=9, seed=11, sizes=(3, 7), degrees=(2, 3, 5))
    assert len({p.N for p in probs}) == 3
    return probs


def singles(probs, **kw):
    return [swe_mod().SweContext.from_problem(p, **kw) for p in probs]


def test_layout_and_views(small):
    ens = swe_mod().SweEnsemble(small, **KW)
    assert ens.ngroups == 3
    W = ens.pack([p.W for p in small])
    assert W.numel() == ens.size
    seen = torch.zeros(ens.size, dtype=torch.int32, device="cuda")
    for i, p in enumerate(small):
        off, st, N, K = ens.layout[i]
        assert (N, K) == (p.N, p.K)
        assert np.array_equal(ens.view(W, i).cpu().numpy(), p.W)
        seen.as_strided((3, K * (N + 1) ** 2), (st, 1), off).add_(1)
    assert int(seen.max()) == 1, "instance planes overlap"
    for N in {p.N for p in small}:
        first = min(ens.layout[i][0] for i, p in enumerate(small) if p.N == N)
        assert first % 32 == 0, "group planes start on 256-byte boundaries"


def test_rhs_bitwise_equals_single_contexts(small):
    ens = swe_mod().SweEnsemble(small, **KW)
    W = ens.pack([p.W for p in small])
    R = ens.rhs(W)
    torch.cuda.synchronize()
    for i, (p, c) in enumerate(zip(small, singles(small, **KW))):
        Rs = c.rhs(dev(p.W))
        assert torch.equal(ens.view(R, i), Rs), f"instance {i}"


def test_rhs_one_instance_against_oracle(small):
    ens = swe_mod().SweEnsemble(small, **KW)
    W = ens.pack([p.W for p in small])
    R = ens.rhs(W)
    i = max(range(len(small)), key=lambda j: small[j].N)
    p = small[i]
    Ro = O.Oracle(p, **KW).rhs(p.W)
    check_rhs(ens.view(R, i).cpu().numpy(), Ro, p)


@pytest.mark.parametrize("dt", [0.0, 2e-4])
def test_steps_bitwise_equal_single_contexts(small, dt):
    ens = swe_mod().SweEnsemble(small, **KW)
    W = ens.pack([p.W for p in small])
    _, dts = ens.step(W, dt, 4)
    launches = ens.launches()
    assert launches > 0
    _, dts2 = ens.step(W, dt, 3)   # replays the captured graph
    assert ens.launches() > launches
    for i, (p, c) in enumerate(zip(small, singles(small, **KW))):
        Ws = dev(p.W)
        _, d1 = c.step(Ws, dt, 4)
        assert d1 == dts[i]
        _, d2 = c.step(Ws, dt, 3)
        assert d2 == dts2[i]
        assert torch.equal(ens.view(W, i), Ws), f"instance {i}"
    if dt == 0.0:
        assert len(set(dts.tolist())) > 1, "instances must take their own time steps"


def test_max_dt_and_integrals_match_single_contexts(small):
    ens = swe_mod().SweEnsemble(small, **KW)
    W = ens.pack([p.W for p in small])
    dc, dp = ens.max_dt(W)
    ints = ens.integrals(W)
    for i, (p, c) in enumerate(zip(small, singles(small, **KW))):
        Ws = dev(p.W)
        assert (dc[i], dp[i]) == c.max_dt(Ws)
        s = c.integrals(Ws)
        assert np.abs(ints[i] - s).max() <= 1e-14 * max(np.abs(s).max(), 1.0)


def test_step_parity_with_oracle_100_steps():
    """Three members, 100 adaptive LSRK4(5) steps, against the oracle
    stepping each member alone (1e-10 relative L-infinity)."""
    probs = I.ensemble(ninst=3, seed=3, sizes=(4, 6), degrees=(3, 5))
    ens = swe_mod().SweEnsemble(probs, **KW)
    W = ens.pack([p.W for p in probs])
    ens.step(W, 0.0, 100)
    for i, p in enumerate(probs):
        Wo, rc, _ = O.Oracle(p, **KW).step(p.W, 0.0, 100)
        assert rc == 0
        assert rel(ens.view(W, i).cpu().numpy(), Wo) < 1e-10


def test_nonfinite_rolls_back_every_instance(small):
    """A NaN in one instance: the step reports a non-finite state and every
    instance is restored to the start of the step."""
    swedg = swe_mod()
    ens = swedg.SweEnsemble(small, **KW)
    W = ens.pack([p.W for p in small])
    ens.step(W, 0.0, 2)
    W0 = W.clone()
    v = ens.view(W, 4)
    v[0, 0, 1, 1] = float("nan")
    Wbad = W.clone()
    rc, _ = ens.step(W, 0.0, 3, raise_on_error=False)
    assert rc == swedg.ERR_NONFINITE
    assert torch.equal(torch.isnan(W), torch.isnan(Wbad))
    assert torch.equal(torch.nan_to_num(W), torch.nan_to_num(Wbad))
    # other instances untouched by the failed call
    for i in range(len(small)):
        if i != 4:
            assert torch.equal(ens.view(W, i), ens.view(W0, i))


def test_single_context_nonfinite_rolls_back():
    swedg = swe_mod()
    p = I.lake_hump(N=3, K1=4)
    c = swedg.SweContext.from_problem(p, **KW)
    W = dev(p.W)
    W[1, 2, 0, 3] = float("nan")
    Wbad = W.clone()
    rc, _ = c.step(W, 1e-4, 2, raise_on_error=False)
    assert rc == swedg.ERR_NONFINITE
    assert torch.equal(torch.isnan(W), torch.isnan(Wbad))
    assert torch.equal(torch.nan_to_num(W), torch.nan_to_num(Wbad))


def test_create_rejects_cross_instance_connectivity(small):
    swedg = swe_mod()
    bad = [p for p in small[:2]]
    E = bad[1].EToE.copy()
    E[0, 0] = bad[1].K  # outside the instance
    import dataclasses
    bad[1] = dataclasses.replace(bad[1], EToE=E)
    with pytest.raises(swedg.SweError) as ei:
        swedg.SweEnsemble(bad, **KW)
    assert ei.value.code == swedg.ERR_ARG
    with pytest.raises(swedg.SweError):
        swedg.SweEnsemble([], **KW)


def test_full_size_ensemble_sampled_members():
    """The 256-member ensemble (16x16 to 96x96 quads, N in {3, 5, 7}, about
    40M nodes): after one adaptive step of the whole ensemble, sampled
    members equal single contexts bitwise, and their right-hand sides
    match the oracle."""
    probs = I.ensemble(256)
    ens = swe_mod().SweEnsemble(probs, **KW)
    W = ens.pack([p.W for p in probs])
    R = ens.rhs(W)
    sample = [0, 97, 255] + [min(range(256), key=lambda j: probs[j].K)]
    for i in sample:
        p = probs[i]
        if p.K <= 400:
            Ro = O.Oracle(p, **KW).rhs(p.W)
            check_rhs(ens.view(R, i).cpu().numpy(), Ro, p)
    _, dts = ens.step(W, 0.0, 1)
    for i in sample:
        p = probs[i]
        c = swe_mod().SweContext.from_problem(p, **KW)
        Ws = dev(p.W)
        assert torch.equal(c.rhs(Ws), ens.view(R, i))
        _, d = c.step(Ws, 0.0, 1)
        assert d == dts[i]
        assert torch.equal(ens.view(W, i), Ws)
