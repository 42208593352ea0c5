"""Pins of the oracle's pointwise two-point fluxes.

Volume flux (Eq. volumeFluxes) and interface flux (Eqs. surfaceFluxes,
fesandges, App. B) are checked against: consistency with the physical flux,
symmetry, Tadmor's entropy-conservation condition [[q]].F = [[psi]] (flat
bottom, psi = g h^2 u / 2), the Roe-type limit of the dissipation
(1/2 |A_n| [[w]] for nearby states, |A_n| from numpy's eigendecomposition of
the normal flux Jacobian), the sign of the entropy production, and the
compact first component of App. B.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

G = 9.81


def phys(W, g=G):
    h, hu, hv = W
    u, v = hu / h, hv / h
    return (np.array([hu, hu * u + 0.5 * g * h * h, hu * v]),
            np.array([hv, hv * u, hv * v + 0.5 * g * h * h]))


def qvars(W, b, g=G):
    h, hu, hv = W
    u, v = hu / h, hv / h
    return np.array([g * (h + b) - 0.5 * (u * u + v * v), u, v])


def rand_state(rng, hmin=0.2):
    h = rng.uniform(hmin, 2.0)
    return np.array([h, h * rng.uniform(-1.5, 1.5), h * rng.uniform(-1.5, 1.5)])


def test_volume_flux_consistency_and_symmetry():
    rng = np.random.default_rng(0)
    for _ in range(200):
        Wa, Wb = rand_state(rng), rand_state(rng)
        Fs, Gs = O.volume_flux(G, Wa, Wa)
        f, g = phys(Wa)
        assert np.allclose(Fs, f, rtol=1e-14, atol=1e-13)
        assert np.allclose(Gs, g, rtol=1e-14, atol=1e-13)
        F1, G1 = O.volume_flux(G, Wa, Wb)
        F2, G2 = O.volume_flux(G, Wb, Wa)
        assert np.allclose(F1, F2, rtol=1e-15, atol=1e-14)
        assert np.allclose(G1, G2, rtol=1e-15, atol=1e-14)


def test_volume_flux_tadmor_condition():
    rng = np.random.default_rng(1)
    for _ in range(200):
        Wa, Wb = rand_state(rng), rand_state(rng)
        Fs, Gs = O.volume_flux(G, Wa, Wb)
        dq = qvars(Wb, 0.0) - qvars(Wa, 0.0)
        psi_x = lambda W: 0.5 * G * W[0] * W[1]
        psi_y = lambda W: 0.5 * G * W[0] * W[2]
        assert abs(dq @ Fs - (psi_x(Wb) - psi_x(Wa))) < 1e-12 * (1 + abs(psi_x(Wa)))
        assert abs(dq @ Gs - (psi_y(Wb) - psi_y(Wa))) < 1e-12 * (1 + abs(psi_y(Wa)))


def unit(rng):
    a = rng.uniform(0, 2 * math.pi)
    return math.cos(a), math.sin(a)


@pytest.mark.parametrize("es", [0, 1])
def test_surface_flux_consistency(es):
    rng = np.random.default_rng(2)
    for _ in range(200):
        W = rand_state(rng)
        b = rng.uniform(-0.5, 0.5)
        nx, ny = unit(rng)
        F = O.surface_flux(G, es, W, W, b, b, nx, ny)
        f, g = phys(W)
        assert np.allclose(F, nx * f + ny * g, rtol=1e-13, atol=1e-12)


def test_surface_flux_ec_tadmor_condition():
    rng = np.random.default_rng(3)
    for _ in range(200):
        Wm, Wp = rand_state(rng), rand_state(rng)
        nx, ny = unit(rng)
        F = O.surface_flux(G, 0, Wm, Wp, 0.0, 0.0, nx, ny)
        psi = lambda W: 0.5 * G * W[0] * (nx * W[1] + ny * W[2])
        dq = qvars(Wp, 0.0) - qvars(Wm, 0.0)
        assert abs(dq @ F - (psi(Wp) - psi(Wm))) < 1e-12 * (1 + abs(psi(Wm)))


def normal_jacobian(W, nx, ny, g=G):
    h, hu, hv = W
    u, v = hu / h, hv / h
    A = np.array([[0, 1, 0], [g * h - u * u, 2 * u, 0], [-u * v, v, u]])
    B = np.array([[0, 0, 1], [-u * v, v, u], [g * h - v * v, 0, 2 * v]])
    return nx * A + ny * B


def test_surface_flux_dissipation_roe_limit():
    """For W+ = W- + d with |d| -> 0 the dissipation F_ec - F_es tends to
    (1/2)|A_n(W)| d with |A_n| = R |Lambda| R^-1 of the normal flux Jacobian."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        W = rand_state(rng, 0.5)
        nx, ny = unit(rng)
        d0 = rng.standard_normal(3)
        An = normal_jacobian(W, nx, ny)
        lam, Rv = np.linalg.eig(An)
        absA = (Rv @ np.diag(np.abs(lam)) @ np.linalg.inv(Rv)).real
        errs = []
        for s in (1e-3, 5e-4):
            d = s * d0
            Wm, Wp = W - 0.5 * d, W + 0.5 * d
            diss = O.surface_flux(G, 0, Wm, Wp, 0.1, 0.1, nx, ny) - O.surface_flux(G, 1, Wm, Wp, 0.1, 0.1, nx, ny)
            errs.append(np.max(np.abs(diss - 0.5 * absA @ d)))
            assert errs[-1] < 50 * s * s * (1 + np.max(np.abs(absA)))
        # the remainder is second order in |d|
        assert errs[1] < 0.35 * errs[0] + 1e-13


def test_surface_flux_entropy_production_sign():
    rng = np.random.default_rng(5)
    for _ in range(500):
        Wm, Wp = rand_state(rng, 0.05), rand_state(rng, 0.05)
        bm = rng.uniform(-0.3, 0.3)
        nx, ny = unit(rng)
        Fes = O.surface_flux(G, 1, Wm, Wp, bm, bm, nx, ny)
        Fec = O.surface_flux(G, 0, Wm, Wp, bm, bm, nx, ny)
        dq = qvars(Wp, bm) - qvars(Wm, bm)
        # rotate [[q]]'s velocity part into the physical frame dot product
        assert dq @ (Fes - Fec) <= 1e-12 * (1 + np.abs(dq).max() * np.abs(Fes).max())


def test_surface_flux_compact_first_component():
    """App. B: F1*,es = {h}{u~} - (A [[g h + g b]] + {c} B [[u~]]) / (4 g)."""
    rng = np.random.default_rng(6)
    for _ in range(500):
        Wm, Wp = rand_state(rng, 0.0), rand_state(rng, 0.0)
        bm, bp = rng.uniform(-0.3, 0.3, size=2)
        nx, ny = unit(rng)
        F = O.surface_flux(G, 1, Wm, Wp, bm, bp, nx, ny)
        um = (nx * Wm[1] + ny * Wm[2]) / Wm[0]
        up = (nx * Wp[1] + ny * Wp[2]) / Wp[0]
        ua = 0.5 * (um + up)
        ca = 0.5 * (math.sqrt(G * Wm[0]) + math.sqrt(G * Wp[0]))
        A = abs(ua + ca) + abs(ua - ca)
        B = abs(ua + ca) - abs(ua - ca)
        F1 = 0.5 * (Wm[0] + Wp[0]) * ua - (A * (G * (Wp[0] + bp) - G * (Wm[0] + bm)) + ca * B * (up - um)) / (4 * G)
        assert abs(F[0] - F1) < 1e-13 * (1 + abs(F1))


def test_surface_flux_dry_states():
    """Both sides dry: zero flux; one side dry: finite flux and u = 0 there."""
    z = np.zeros(3)
    F = O.surface_flux(G, 1, z, z, 0.0, 0.0, 0.6, 0.8)
    assert np.all(F == 0.0)
    W = np.array([1.0, 0.5, -0.2])
    F = O.surface_flux(G, 1, W, z, 0.0, 0.0, 1.0, 0.0)
    assert np.all(np.isfinite(F))
