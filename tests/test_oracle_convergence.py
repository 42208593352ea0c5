"""Order of accuracy of the assembled scheme on a manufactured smooth
solution (Sec. 2.2, Eq. CurvilinearECDGSEMviscous without viscosity).

A smooth periodic exact solution W_e(x, y, t) on the curved [0,2]^2 mesh of
the lake-plus-hump configuration (x += 0.05 sin(pi x) sin(pi y), same for y)
over the bathymetry b = 0.1 + 0.05 sin(pi x) cos(pi y); the forcing
S = W_t + div F(W_e) + g h grad b of the exact solution is added at the
nodes in every stage (dW/dt = R(W) + S(x, t)), and the semi-discrete system
is advanced with the oracle's right-hand side (entropy-stable interface
flux; no viscosity and no limiter, which would cut the order on purpose) by
the five-stage 2N-storage LSRK4(5) with the oracle's coefficients. The L2
error at t = 0.2 must fall at rate >= N + 0.8 between the two finest meshes.
The time step is the CFL rule's; a step four times smaller changes none of
the errors in their first four digits, so the time error is negligible.

Planted mistakes this fails on (each run once by hand): a surface lift
weight 1/w_1 instead of 1/w_0, the source's printed factor 2D (twice the
continuous source), the printed pairing of {x_xi} with F# in G~.
"""
import math

import numpy as np
import pytest

import refmath
from oracle import oracle as O
from paper_1804_02221_gb300 import inputs as I

sp = pytest.importorskip("sympy")

G = 9.81
T_END = 0.2


def exact():
    X, Y, t = sp.symbols("x y t")
    b = 0.1 + 0.05 * sp.sin(sp.pi * X) * sp.cos(sp.pi * Y)
    h = 1.5 + 0.1 * sp.sin(sp.pi * (X + Y - t)) - b
    u = 0.3 + 0.1 * sp.cos(sp.pi * (X - Y) - sp.pi * t / 2)
    v = 0.2 + 0.1 * sp.sin(sp.pi * (X + 2 * Y) + sp.pi * t / 3)
    W = [h, h * u, h * v]
    f = [h * u, h * u ** 2 + G * h ** 2 / 2, h * u * v]
    g = [h * v, h * u * v, h * v ** 2 + G * h ** 2 / 2]
    src = [0, G * h * sp.diff(b, X), G * h * sp.diff(b, Y)]
    S = [sp.diff(W[c], t) + sp.diff(f[c], X) + sp.diff(g[c], Y) + src[c] for c in range(3)]
    return (sp.lambdify((X, Y, t), W, "numpy"), sp.lambdify((X, Y, t), S, "numpy"),
            sp.lambdify((X, Y), b, "numpy"))


def stage_times(A, B):
    """c_s of the 2N-storage scheme: the stage values of y' = 1, y(0) = 0."""
    c, y, k = [], 0.0, 0.0
    for s in range(len(A)):
        c.append(y)
        k = A[s] * k + 1.0
        y += B[s] * k
    assert abs(y - 1.0) < 1e-14
    return c


def l2_error(N, K1, Wf, Sf, bf):
    x, y, xw, yw, E, F, fl = I.periodic_mesh(N, K1, K1, (0.0, 2.0, 0.0, 2.0),
                                             lambda A, B: (0.05 * np.sin(np.pi * A) * np.sin(np.pi * B),) * 2,
                                             rotate_seed=K1)
    field = lambda fun, t: np.stack([np.broadcast_to(a, xw.shape) for a in fun(xw, yw, t)]).astype(float)
    b = bf(xw, yw) * np.ones_like(xw)
    p = I.Problem("manufactured", N, K1, K1, x, y, b, np.ascontiguousarray(field(Wf, 0.0)), E, F, fl, G)
    o = O.Oracle(p, flux=1, cfl=0.5)
    A, B = O.lsrk_coefficients()
    c = stage_times(A, B)
    dtc, _ = o.max_dt(p.W)
    nst = int(math.ceil(T_END / dtc))
    dt = T_END / nst
    W, Kr, t = p.W.copy(), np.zeros_like(p.W), 0.0
    for _ in range(nst):
        for s in range(5):
            Kr = A[s] * Kr + dt * (o.rhs(W) + field(Sf, t + c[s] * dt))
            W = W + B[s] * Kr
        t += dt
    ww = refmath.quad_weights(N) * refmath.geometry(x, y, N)[4]
    return math.sqrt(np.sum(ww * (W - field(Wf, T_END)) ** 2) / np.sum(ww))


@pytest.mark.parametrize("N,meshes", [(2, (8, 16, 32)), (3, (8, 16, 32)), (4, (4, 8, 16)), (5, (4, 8, 16))])
def test_manufactured_solution_order(N, meshes):
    Wf, Sf, bf = exact()
    errs = [l2_error(N, K1, Wf, Sf, bf) for K1 in meshes]
    rate = math.log2(errs[-2] / errs[-1])
    assert rate >= N + 0.8, (errs, rate)
    assert errs[-1] < errs[-2] < errs[-3]
