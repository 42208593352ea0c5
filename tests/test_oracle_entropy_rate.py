"""Pins of the oracle's discrete entropy rate orc_entropy_rate (Sec. 2: the
entropy variables of Eq. entropyVariables contracted with the semi-discrete
operator): it is the time derivative of the total entropy (orc_entropy)
along R, zero for the entropy-conservative scheme (Lemma ESDGSEM), and its
entropy-stable part is the interface dissipation identity."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I
from test_oracle_scheme import es_dissipation_sum


@pytest.mark.parametrize("N,rot,flux,av", [(2, None, 0, False), (3, 5, 1, False), (4, 2, 1, True)])
def test_rate_is_the_time_derivative_of_the_entropy(N, rot, flux, av):
    """(E(W + d R) - E(W - d R)) / 2d -> sum J w w q(W).R (the chain rule
    with q = de/dw, independent of how the rate is summed)."""
    p = I.random_smooth(N=N, K1=3, seed=40 + N, rotate_seed=rot)
    o = O.Oracle(p, flux=flux, av=av, eps0=0.03, sigma_min=-6.0, sigma_max=-0.5)
    rate, scale = o.entropy_rate(p.W)
    R = o.rhs(p.W)
    d = 1e-4 / np.abs(R).max()
    fd = (o.entropy(p.W + d * R) - o.entropy(p.W - d * R)) / (2 * d)
    assert abs(fd - rate) < 1e-7 * scale, (fd, rate, scale)


@pytest.mark.parametrize("N,rot", [(1, None), (3, 5), (6, 3)])
def test_rate_of_the_ec_scheme_vanishes(N, rot):
    p = I.random_rough(N=N, K1=3, seed=50 + N, rotate_seed=rot)
    rate, scale = O.Oracle(p, flux=0).entropy_rate(p.W)
    assert scale > 0
    assert abs(rate) < 1e-13 * scale


@pytest.mark.parametrize("N,rot", [(2, None), (5, 4)])
def test_rate_of_the_es_scheme_is_the_interface_dissipation(N, rot):
    p = I.random_rough(N=N, K1=3, seed=60 + N, rotate_seed=rot)
    es, scale = O.Oracle(p, flux=1).entropy_rate(p.W)
    ec, _ = O.Oracle(p, flux=0).entropy_rate(p.W)
    diss = es_dissipation_sum(p)
    assert diss < 0 and es < 0
    assert abs((es - ec) - diss) < 1e-12 * scale
