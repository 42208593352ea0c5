"""Error measures of the parity tests.

The right-hand side is a small difference of large terms for states near
equilibrium (flux differencing against the well-balanced source, metric
derivatives cancelling by the discrete metric identities), so two correct
FP64 evaluations that round differently disagree in proportion to the size
of those terms, not to the size of the result: an oracle whose derivative
matrix alone is computed by another (equally exact) formula moves R by
9e-12 relative to max|R| on the lake-plus-hump state. The scale is
  T = g max(h)^2 max_nodes (|a_xi| + |a_eta|)/J * N(N+1)/2,
the largest single term of the flux difference (N(N+1)/2 = 1/omega_0 is the
largest entry of D~), and the right-hand-side error is measured relative to
max(|R|_inf, T).
"""
import numpy as np

import refmath


def term_scale(prob, W=None):
    W = prob.W if W is None else W
    x_xi, x_eta, y_xi, y_eta, J = refmath.geometry(prob.x, prob.y, prob.N)
    a = (np.hypot(y_eta, x_eta) + np.hypot(y_xi, x_xi)) / J
    return prob.g * np.abs(W[0]).max() ** 2 * a.max() * prob.N * (prob.N + 1) / 2.0


def rhs_err(Rg, Ro, prob, W=None):
    """|Rg - Ro|_inf / max(|Ro|_inf, T)."""
    return np.abs(Rg - Ro).max() / max(np.abs(Ro).max(), term_scale(prob, W))


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
