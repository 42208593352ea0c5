"""The FP64 oracle against an independent multi-precision evaluation of the
right-hand side (oracle/bruteforce.py: 40-digit arithmetic, neighbours
matched by physical coordinates instead of the connectivity tables, strong
form with explicit surface corrections, strong-form BR1).

* Small meshes, N = 1 and 2, on 1, 2 and 4 elements: periodic self-connected
  elements, rotated element frames (faces meeting with reversed node order),
  solid walls; EC and ES interface fluxes, and the BR1 viscosity with every
  element at eps0. These pin the oracle's face bookkeeping (owner and
  neighbour slots, the sign of the contravariant interface flux per face,
  the flip), which the identity pins cannot see when a mistake is symmetric.
* The full-size N = 12 dam-break mesh (158 x 158 quads, 4.2M nodes): the
  oracle's right-hand side on elements at the far corner of the domain
  (coordinates ~2, element size 0.0127, the 3 x 3 patch wrapping across the
  periodic seam) against the exact one. This pins the conditioning of the
  metric terms: differentiating the absolute coordinates instead of the
  element-relative ones puts an error ~1e-12 of the term scale there.
* The stored exact right-hand side of the lake-plus-hump configuration
  (tests/golden/lake_hump_exact_rhs.npz): it is reproduced by the brute
  force, and the oracle's distance to it is the rounding floor of an FP64
  evaluation on that near-equilibrium state.
"""
import os

import numpy as np
import pytest

from parity import term_scale
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

mp = pytest.importorskip("mpmath")
from oracle.bruteforce import BruteForce  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lake_hump_exact_rhs.npz")
TOL = 1e-13
AV = dict(av=True, eps0=0.02, sigma_min=-301.0, sigma_max=-300.0)  # eps = eps0 in every element

# (N, Kx, Ky, rotate_seed, walls)
CASES = [
    (1, 1, 1, None, None), (1, 2, 1, 3, None), (1, 2, 2, 4, None),
    (2, 1, 1, 2, None), (2, 2, 1, 7, None), (2, 2, 2, 5, None),
    (2, 2, 2, 2, (True, True)), (1, 2, 1, 5, (True, False)), (2, 1, 1, None, (True, True)),
]


def problem(N, Kx, Ky, rot, walls):
    if walls is None:
        p = I.random_smooth(N=N, Kx=Kx, Ky=Ky, seed=N + Kx, rotate_seed=rot)
        rng = np.random.default_rng(N * 10 + Kx)
        p.W = p.W * (1 + 0.2 * rng.uniform(-1, 1, size=p.W.shape))
        periods = [(2.0, 0.0), (0.0, 2.0)]
    else:
        p = I.random_walls(N=N, Kx=Kx, Ky=Ky, seed=3, rotate_seed=rot, walls=walls)
        periods = [] if walls == (True, True) else ([(0.0, 2.0)] if walls[0] else [(2.0, 0.0)])
    return p, periods


def test_cases_cover_the_face_bookkeeping():
    flips = sum(int(problem(*c)[0].flip.any()) for c in CASES)
    selfconn = problem(1, 1, 1, None, None)[0]
    assert flips >= 3
    assert np.all(selfconn.EToE == 0)
    assert any((problem(*c)[0].EToE < 0).any() for c in CASES)


@pytest.mark.parametrize("N,Kx,Ky,rot,walls", CASES)
def test_rhs_against_bruteforce(N, Kx, Ky, rot, walls):
    p, periods = problem(N, Kx, Ky, rot, walls)
    bf = BruteForce(N, p.x, p.y, p.b, p.g, periods=periods)
    nwall = sum(v is None for v in bf.partner.values())
    assert nwall == int((p.EToE < 0).sum()) * (N + 1)
    for flux in (0, 1):
        Rb = bf.rhs(p.W, flux=flux)
        Ro = O.Oracle(p, flux=flux).rhs(p.W)
        assert np.abs(Ro - Rb).max() <= TOL * np.abs(Rb).max(), flux
    o = O.Oracle(p, flux=1, **AV)
    Ro = o.rhs(p.W)
    assert np.all(o.epsilon() == AV["eps0"])
    Rb = bf.rhs(p.W, flux=1, eps=o.epsilon())
    assert np.abs(Ro - Rb).max() <= TOL * np.abs(Rb).max()


def test_full_size_N12_far_corner_against_bruteforce():
    """Metric terms at |x| ~ 160 element sizes from the origin (reading: the
    coordinates are differentiated relative to the element's first node)."""
    N, K1 = 12, 158
    p = I.dam_break(N=N, K1=K1)
    rng = np.random.default_rng(0)
    W = p.W * (1 + 0.01 * rng.uniform(-1, 1, size=p.W.shape))
    T = term_scale(p)
    Ro = O.Oracle(p, flux=1).rhs(W)
    for cx, cy in ((K1 - 1, K1 - 1), (K1 - 1, K1 // 2)):
        ks = [((cy + dy) % K1) * K1 + (cx + dx) % K1 for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        bf = BruteForce(N, p.x[ks], p.y[ks], p.b[ks], p.g)
        Rb = bf.rhs(W[:, ks], flux=1, elements=[4])
        assert np.abs(Ro[:, ks[4]] - Rb[:, 4]).max() <= 1e-13 * T


def test_lake_hump_exact_rhs_golden():
    d = np.load(GOLDEN)
    p = I.lake_hump(N=3, K1=8)
    p.x, p.y, p.b = d["x"], d["y"], d["b"]
    # the stored exact right-hand side is what the brute force gives
    bf = BruteForce(p.N, p.x, p.y, p.b, p.g)
    assert np.array_equal(bf.rhs(d["W0"], flux=1), d["R0"])
    o = O.Oracle(p, flux=1, av=True, eps0=0.01, limiter=True)
    T = term_scale(p)
    for W, R in ((d["W0"], d["R0"]), (d["W50"], d["R50"])):
        Ro = o.rhs(W)
        assert o.epsilon().max() == 0.0
        err = np.abs(Ro - R).max()
        # the FP64 oracle's own distance to the exact result: ~1e-15 of T,
        # which is ~2e-12 of |R| on this state (T/|R| ~ 2000)
        assert err <= 2e-15 * T
        assert T / np.abs(R).max() > 1000
