"""Independent numpy restatements used to pin the oracle.

Everything here is derived by a route different from the oracle's: the
derivative matrix from the Legendre Vandermonde matrix and its derivative,
LGL nodes from numpy's root finder, face geometry from numpy array slicing.
Nothing here is used by the CUDA library or by the oracle.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def lgl(N):
    inner = npleg.Legendre.basis(N).deriv().roots()
    xi = np.concatenate(([-1.0], np.sort(np.real(inner)), [1.0]))
    PN = npleg.legval(xi, [0] * N + [1])
    w = 2.0 / (N * (N + 1) * PN ** 2)
    return xi, w


def dmat(N):
    """D = V' V^-1 with the Legendre Vandermonde matrix V and its derivative."""
    xi, _ = lgl(N)
    n = N + 1
    V = np.zeros((n, n))
    Vd = np.zeros((n, n))
    for j in range(n):
        c = [0] * j + [1]
        V[:, j] = npleg.legval(xi, c)
        Vd[:, j] = npleg.legval(xi, npleg.legder(c)) if j > 0 else 0.0
    return Vd @ np.linalg.inv(V)


def geometry(x, y, N):
    """Metric terms and Jacobian with D applied along the xi (last) and eta
    (middle) axes of [K, n, n] arrays."""
    D = dmat(N)
    x_xi = np.einsum("im,kjm->kji", D, x)
    y_xi = np.einsum("im,kjm->kji", D, y)
    x_eta = np.einsum("jm,kmi->kji", D, x)
    y_eta = np.einsum("jm,kmi->kji", D, y)
    J = x_xi * y_eta - x_eta * y_xi
    return x_xi, x_eta, y_xi, y_eta, J


def face_slice(a, f):
    """Values of a nodal [K, n, n] array (or [..., K, n, n]) on face f,
    ordered along the face: shape [..., K, n]."""
    if f == 0:
        return a[..., 0, :]
    if f == 1:
        return a[..., :, -1]
    if f == 2:
        return a[..., -1, :]
    return a[..., :, 0]


def outward_normal(geo, f):
    x_xi, x_eta, y_xi, y_eta, _ = geo
    if f == 0:
        return face_slice(y_xi, 0), -face_slice(x_xi, 0)
    if f == 1:
        return face_slice(y_eta, 1), -face_slice(x_eta, 1)
    if f == 2:
        return -face_slice(y_xi, 2), face_slice(x_xi, 2)
    return -face_slice(y_eta, 3), face_slice(x_eta, 3)


def unique_faces(prob):
    """(k, f, kk, ff, flip) once per interface."""
    out = []
    for k in range(prob.K):
        for f in range(4):
            kk, ff = int(prob.EToE[k, f]), int(prob.EToF[k, f])
            if kk > k or (kk == k and ff > f):
                out.append((k, f, kk, ff, int(prob.flip[k, f])))
    return out


def primitives(W):
    h, hu, hv = W
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(h > 0, hu / np.where(h > 0, h, 1.0), 0.0)
        v = np.where(h > 0, hv / np.where(h > 0, h, 1.0), 0.0)
    return h, u, v


def entropy_vars(W, b, g):
    h, u, v = primitives(W)
    return np.stack([g * (h + b) - 0.5 * (u * u + v * v), u, v])


def physical_flux(W, g):
    h, u, v = primitives(W)
    f = np.stack([h * u, h * u * u + 0.5 * g * h * h, h * u * v])
    gg = np.stack([h * v, h * u * v, h * v * v + 0.5 * g * h * h])
    return f, gg


def quad_weights(N):
    _, w = lgl(N)
    return np.outer(w, w)  # [j, i]
