"""Pins of the oracle's LGL basis (Sec. 2.2, App. A) against closed forms and
numpy's Legendre routines."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import refmath
from oracle import oracle as O

NS = list(range(1, 17))


@pytest.mark.parametrize("N", NS)
def test_lgl_nodes_and_weights(N):
    xi, w, D, V, Vinv = O.basis(N)
    ref_xi, ref_w = refmath.lgl(N)
    assert np.max(np.abs(xi - ref_xi)) < 1e-14
    assert np.max(np.abs(w - ref_w)) < 1e-13
    assert abs(w.sum() - 2.0) < 1e-13
    # LGL quadrature is exact for polynomials of degree <= 2N-1
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * xi ** k) - exact) < 1e-13
    # end weight omega_0 = 2/(N(N+1)) (the value Lemma PosPres needs)
    assert abs(w[0] - 2.0 / (N * (N + 1))) < 1e-15


@pytest.mark.parametrize("N", NS)
def test_derivative_matrix(N):
    xi, w, D, V, Vinv = O.basis(N)
    # exact on monomials up to degree N
    for k in range(N + 1):
        d = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        assert np.max(np.abs(D @ xi ** k - d)) < 1e-11 * max(1, k) * N ** 2
    # matches the Vandermonde route
    assert np.max(np.abs(D - refmath.dmat(N))) < 1e-10 * N ** 2
    # SBP property (Eq. SBP_def)
    M = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    assert np.max(np.abs(M @ D + (M @ D).T - B)) < 1e-13 * N ** 2
    # closed-form corner entries of the LGL derivative matrix
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-12 * N ** 2
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-12 * N ** 2
    # D~ = 2D + S has a vanishing diagonal and M D~ is skew apart from the corners
    S = np.diag([1.0 / w[0]] + [0.0] * (N - 1) + [-1.0 / w[N]]) if N > 1 else np.diag([1.0 / w[0], -1.0 / w[N]])
    Dt = 2 * D + S
    assert np.max(np.abs(np.diag(Dt))) < 1e-12 * N ** 2


@pytest.mark.parametrize("N", NS)
def test_vandermonde(N):
    xi, w, D, V, Vinv = O.basis(N)
    n = N + 1
    for j in range(n):
        ref = npleg.legval(xi, [0] * j + [1]) * math.sqrt(j + 0.5)
        assert np.max(np.abs(V[:, j] - ref)) < 1e-13
    assert np.max(np.abs(Vinv @ V - np.eye(n))) < 1e-12
    # App. A's Gauss-quadrature formula for V^-1 (exact for these degrees):
    # Vinv_ij = sum_l Ltilde_i(xg_l) l_j(xg_l) wg_l
    xg, wg = npleg.leggauss(n)
    lag = np.zeros((n, n))  # lag[l, j] = l_j(xg_l)
    for j in range(n):
        others = np.delete(xi, j)
        lag[:, j] = np.prod((xg[:, None] - others[None, :]) / (xi[j] - others[None, :]), axis=1)
    Lt = np.stack([npleg.legval(xg, [0] * i + [1]) * math.sqrt(i + 0.5) for i in range(n)])
    ref = (Lt * wg[None, :]) @ lag
    assert np.max(np.abs(Vinv - ref)) < 1e-11 * n
