"""Seeded synthetic inputs: meshes, bathymetries and initial states.

This module holds none of the scheme's arithmetic. It evaluates analytic
mappings and fields at Legendre-Gauss-Lobatto positions (taken from numpy's
Legendre-polynomial roots) and builds periodic quadrilateral connectivity.
Both the CUDA library's tests and the oracle's tests draw their inputs here.

Array layout (shared with the library's C-ABI):
  x, y, b          float64 [K, n, n]     index [k, j, i], i along xi (fastest)
  W                float64 [3, K, n, n]  (h, hu, hv)
  EToE, EToF, flip int32   [K, 4]        faces 0: eta=-1, 1: xi=+1, 2: eta=+1, 3: xi=-1

Face node p runs along increasing xi (faces 0, 2) or eta (faces 1, 3); node p of
face (k, f) meets node (N - p if flip else p) of face (EToE[k, f], EToF[k, f]).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def lgl_points(N: int) -> np.ndarray:
    """LGL positions -1, roots of L_N', +1 (numpy polynomial root finder)."""
    if N < 1:
        raise ValueError("N >= 1 required")
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots()
    return np.concatenate(([-1.0], np.sort(np.real(inner)), [1.0]))


@dataclasses.dataclass
class Problem:
    """One synthetic instance: mesh, bathymetry, gravity and initial state."""

    name: str
    N: int
    Kx: int
    Ky: int
    x: np.ndarray
    y: np.ndarray
    b: np.ndarray
    W: np.ndarray
    EToE: np.ndarray
    EToF: np.ndarray
    flip: np.ndarray
    g: float = 9.81
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def K(self) -> int:
        return self.x.shape[0]

    @property
    def n(self) -> int:
        return self.N + 1

    @property
    def nodes(self) -> int:
        return self.K * self.n * self.n


# ---------------------------------------------------------------------------
# Mesh: periodic structured quads, optionally with rotated element frames
# ---------------------------------------------------------------------------

def _local_to_canonical(N: int, r: int, ii: np.ndarray, jj: np.ndarray):
    """Canonical node (i, j) of local node (ii, jj) of an element whose local
    frame is rotated by r quarter turns."""
    if r == 0:
        return ii, jj
    if r == 1:
        return N - jj, ii
    if r == 2:
        return N - ii, N - jj
    return jj, N - ii


def _face_local_nodes(N: int, f: int):
    p = np.arange(N + 1)
    if f == 0:
        return p, np.zeros_like(p)
    if f == 1:
        return np.full_like(p, N), p
    if f == 2:
        return p, np.full_like(p, N)
    return np.zeros_like(p), p


def _canonical_face_of(N: int, i: np.ndarray, j: np.ndarray) -> int:
    if np.all(j == 0):
        return 0
    if np.all(i == N):
        return 1
    if np.all(j == N):
        return 2
    return 3


def periodic_mesh(N: int, Kx: int, Ky: int, domain, mapping, rotate_seed=None, walls=(False, False)):
    """Periodic Kx x Ky quad mesh of the box domain=(x0, x1, y0, y1).

    ``mapping(X, Y)`` returns the displacement (dx, dy) of the lattice point
    (X, Y) given in wrapped coordinates; it must be periodic. Returns
    (x, y, xw, yw, EToE, EToF, flip) where (xw, yw) are the physical
    coordinates wrapped into the periodic box (identical bit patterns on both
    sides of every face, so fields evaluated there agree across faces).
    Element k = ky*Kx + kx; with rotate_seed the local frame of every element
    is turned by a random number of quarter turns. walls = (in x, in y):
    the faces on x = x0, x1 (resp. y = y0, y1) become solid walls
    (EToE = -1) instead of periodic, and those coordinates are not wrapped.
    """
    x0, x1, y0, y1 = domain
    Lx, Ly = x1 - x0, y1 - y0
    n = N + 1
    r = lgl_points(N)
    K = Kx * Ky
    rng = np.random.default_rng(rotate_seed) if rotate_seed is not None else None
    rot = rng.integers(0, 4, size=K) if rng is not None else np.zeros(K, dtype=np.int64)

    # canonical lattice coordinates (exact at element corners)
    ex = np.arange(Kx)[:, None] + (r[None, :] + 1.0) / 2.0  # [Kx, n]
    ey = np.arange(Ky)[:, None] + (r[None, :] + 1.0) / 2.0
    Xc = x0 + Lx * ex / Kx
    Yc = y0 + Ly * ey / Ky
    Xcw = Xc if walls[0] else np.where(Xc >= x1, Xc - Lx, Xc)
    Ycw = Yc if walls[1] else np.where(Yc >= y1, Yc - Ly, Yc)

    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # [j, i]
    ci_tab = np.stack([_local_to_canonical(N, q, ii, jj)[0] for q in range(4)])  # [4, n, n]
    cj_tab = np.stack([_local_to_canonical(N, q, ii, jj)[1] for q in range(4)])
    k = np.arange(K)
    kx, ky = k % Kx, k // Kx
    CI, CJ = ci_tab[rot], cj_tab[rot]  # [K, n, n]
    X = Xc[kx[:, None, None], CI]
    Y = Yc[ky[:, None, None], CJ]
    XW = Xcw[kx[:, None, None], CI]
    YW = Ycw[ky[:, None, None], CJ]
    dx, dy = mapping(XW, YW)
    x, y, xw, yw = X + dx, Y + dy, XW + dx, YW + dy

    # local face f of a frame turned by q quarter turns lies on canonical face
    # (f + q) % 4; rev_tab[q, f]: its node order runs against the canonical one
    rev_tab = np.zeros((4, 4), dtype=bool)
    for q in range(4):
        for f in range(4):
            li, lj = _face_local_nodes(N, f)
            ci, cj = _local_to_canonical(N, q, li, lj)
            F = _canonical_face_of(N, ci, cj)
            assert F == (f + q) % 4
            pos = ci if F in (0, 2) else cj
            rev_tab[q, f] = pos[0] == N
    f = np.arange(4)[None, :]
    F = (f + rot[:, None]) % 4  # [K, 4]
    nkx = np.where(F == 1, (kx[:, None] + 1) % Kx, np.where(F == 3, (kx[:, None] - 1) % Kx, kx[:, None]))
    nky = np.where(F == 0, (ky[:, None] - 1) % Ky, np.where(F == 2, (ky[:, None] + 1) % Ky, ky[:, None]))
    nb = nky * Kx + nkx
    fn = ((F + 2) % 4 - rot[nb]) % 4
    EToE = nb.astype(np.int32)
    EToF = fn.astype(np.int32)
    flip = (rev_tab[rot[:, None], f] != rev_tab[rot[nb], fn]).astype(np.int32)
    wall = np.zeros((K, 4), dtype=bool)
    if walls[0]:
        wall |= ((F == 1) & (kx[:, None] == Kx - 1)) | ((F == 3) & (kx[:, None] == 0))
    if walls[1]:
        wall |= ((F == 0) & (ky[:, None] == 0)) | ((F == 2) & (ky[:, None] == Ky - 1))
    EToE[wall] = -1
    EToF[wall] = 0
    flip[wall] = 0
    return x, y, xw, yw, EToE, EToF, flip


# ---------------------------------------------------------------------------
# Mappings and fields
# ---------------------------------------------------------------------------

def _sine_map(amp: float, freq: float):
    def mapping(X, Y):
        d = amp * np.sin(freq * X) * np.sin(freq * Y)
        return d, d
    return mapping


def _gaussian_sum_periodic(xw, yw, a, c, s, Lx, Ly):
    B = np.zeros_like(xw)
    for ak, ck, sk in zip(a, c, s):
        for sx in (-Lx, 0.0, Lx):
            for sy in (-Ly, 0.0, Ly):
                B += ak * np.exp(-((xw - ck[0] - sx) ** 2 + (yw - ck[1] - sy) ** 2) / sk ** 2)
    return B


def _gaussian_sum_periodic_separable(xw, yw, a, c, s, Lx, Ly):
    """The same sum of periodic Gaussian images, factored per direction."""
    B = np.zeros_like(xw)
    for ak, ck, sk in zip(a, c, s):
        ex = sum(np.exp(-((xw - ck[0] - sx) / sk) ** 2) for sx in (-Lx, 0.0, Lx))
        ey = sum(np.exp(-((yw - ck[1] - sy) / sk) ** 2) for sy in (-Ly, 0.0, Ly))
        B += ak * ex * ey
    return B


def _smooth_periodic_field(rng, xw, yw, Lx, Ly, modes=3):
    """Random smooth periodic field of unit-order amplitude."""
    f = np.zeros_like(xw)
    for p in range(modes + 1):
        for q in range(modes + 1):
            a, bb, c, d = rng.standard_normal(4) / (1.0 + p * p + q * q)
            kx, ky = 2 * math.pi * p / Lx, 2 * math.pi * q / Ly
            f += a * np.cos(kx * xw) * np.cos(ky * yw) + bb * np.sin(kx * xw) * np.cos(ky * yw)
            f += c * np.cos(kx * xw) * np.sin(ky * yw) + d * np.sin(kx * xw) * np.sin(ky * yw)
    return f / max(1e-300, np.max(np.abs(f)))


def _state(h, u, v):
    return np.ascontiguousarray(np.stack([h, h * u, h * v]))


def lake_hump(N=3, K1=8, seed=0, rotate_seed=None, g=9.81, amp=0.01) -> Problem:
    """Lake at rest h+b=1 on b=0.1+0.05 sin(pi x)cos(pi y) plus a seeded
    Gaussian hump (amplitude 0.01, width 0.2) on the curved periodic
    [0,2]^2 mesh x += 0.05 sin(pi x) sin(pi y) (same for y)."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, K1, K1, (0.0, 2.0, 0.0, 2.0),
                                           _sine_map(0.05, math.pi), rotate_seed)
    rng = np.random.default_rng(seed)
    c0 = rng.uniform(0.5, 1.5, size=2)
    b = 0.1 + 0.05 * np.sin(math.pi * xw) * np.cos(math.pi * yw)
    h = 1.0 - b + amp * np.exp(-((xw - c0[0]) ** 2 + (yw - c0[1]) ** 2) / 0.2 ** 2)
    z = np.zeros_like(h)
    return Problem("lake_hump", N, K1, K1, x, y, b, _state(h, z, z), E, F, fl, g,
                   {"hump_center": c0.tolist()})


def lake_at_rest_kinked(N=3, K1=6, rotate_seed=None, g=9.81, H=1.0) -> Problem:
    """h+b=H, u=v=0 on the curved [0,2]^2 mesh with b continuous but not
    smooth: the lake_hump bathymetry plus a cone 0.1 max(0, 1 - r/0.5)."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, K1, K1, (0.0, 2.0, 0.0, 2.0),
                                           _sine_map(0.05, math.pi), rotate_seed)
    r = np.sqrt((xw - 0.93) ** 2 + (yw - 1.07) ** 2)
    b = 0.1 + 0.05 * np.sin(math.pi * xw) * np.cos(math.pi * yw) + 0.1 * np.maximum(0.0, 1.0 - r / 0.5)
    h = H - b
    z = np.zeros_like(h)
    return Problem("lake_at_rest_kinked", N, K1, K1, x, y, b, _state(h, z, z), E, F, fl, g)


def dam_break(N=7, K1=None, seed=1, rotate_seed=None, g=9.81) -> Problem:
    """Degree-sweep workload: periodic curved [0,2]^2 mesh with K1 x K1 quads
    (default round(2048/(N+1)), about 4.2M nodes), bathymetry 0.3 B/max B with
    B a sum of 8 seeded Gaussians (periodic images), total height H = 2.0
    where x < 1 + 0.25 sin(pi y) and 0.5 elsewhere, at rest."""
    if K1 is None:
        K1 = int(round(2048 / (N + 1)))
    x, y, xw, yw, E, F, fl = periodic_mesh(N, K1, K1, (0.0, 2.0, 0.0, 2.0),
                                           _sine_map(0.05, math.pi), rotate_seed)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 1.0, size=8)
    c = rng.uniform(0.0, 2.0, size=(8, 2))
    s = rng.uniform(0.1, 0.4, size=8)
    B = _gaussian_sum_periodic(xw, yw, a, c, s, 2.0, 2.0)
    b = 0.3 * B / B.max()
    H = np.where(xw < 1.0 + 0.25 * np.sin(math.pi * yw), 2.0, 0.5)
    h = H - b
    z = np.zeros_like(h)
    return Problem("dam_break", N, K1, K1, x, y, b, _state(h, z, z), E, F, fl, g,
                   {"K1": K1})


def thacker_bowl(N=4, K1=128, g=9.81, h0=0.25, a=1.0, sigma=0.5, rotate_seed=None) -> Problem:
    """Oscillating lake in the parabolic bowl b = h0 (x^2+y^2)/a^2 on [-2,2]^2
    (curved map x += 0.05 sin(pi x/2) sin(pi y/2), same for y), initial state
    of the analytic solution at t = 0: wet disc (x-sigma)^2 + y^2 < a^2."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, K1, K1, (-2.0, 2.0, -2.0, 2.0),
                                           _sine_map(0.05, math.pi / 2), rotate_seed)
    b = h0 * (xw ** 2 + yw ** 2) / a ** 2
    W = thacker_state(xw, yw, b, 0.0, g, h0, a, sigma)
    p = Problem("thacker_bowl", N, K1, K1, x, y, b, W, E, F, fl, g,
                {"h0": h0, "a": a, "sigma": sigma, "omega": math.sqrt(2 * g * h0) / a})
    p.meta["xw"], p.meta["yw"] = xw, yw
    return p


def thacker_state(xw, yw, b, t, g=9.81, h0=0.25, a=1.0, sigma=0.5):
    """Analytic oscillating-lake solution at time t (Sec. 6.2)."""
    om = math.sqrt(2 * g * h0) / a
    h = np.maximum(0.0, sigma * h0 / a ** 2 * (2 * xw * math.cos(om * t) + 2 * yw * math.sin(om * t) - sigma)
                   + h0 - b)
    u = np.where(h > 0, -sigma * om * math.sin(om * t), 0.0)
    v = np.where(h > 0, sigma * om * math.cos(om * t), 0.0)
    return _state(h, u, v)


def random_smooth(N=3, K1=4, seed=0, rotate_seed=None, g=9.81, dh=0.2, du=0.5,
                  flat=False, Kx=None, Ky=None) -> Problem:
    """Smooth random periodic state (h in [1-dh, 1+dh], |u|,|v| <= du) on the
    curved [0,2]^2 mesh with a smooth random bathymetry (flat if asked)."""
    Kx = Kx or K1
    Ky = Ky or K1
    x, y, xw, yw, E, F, fl = periodic_mesh(N, Kx, Ky, (0.0, 2.0, 0.0, 2.0),
                                           _sine_map(0.05, math.pi), rotate_seed)
    rng = np.random.default_rng(seed)
    b = np.zeros_like(xw) if flat else 0.1 * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    h = 1.0 + dh * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    u = du * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    v = du * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    return Problem("random_smooth", N, Kx, Ky, x, y, b, _state(h, u, v), E, F, fl, g)


def random_rough(N=3, K1=4, seed=0, rotate_seed=None, g=9.81, dry_fraction=0.0) -> Problem:
    """Non-smooth random nodal state (independent noise per node) on a smooth
    bathymetry; with dry_fraction > 0 that share of nodes is set dry."""
    p = random_smooth(N, K1, seed, rotate_seed, g)
    rng = np.random.default_rng(seed + 1000)
    h = 1.0 + 0.3 * rng.uniform(-1, 1, size=p.b.shape)
    u = 0.5 * rng.uniform(-1, 1, size=p.b.shape)
    v = 0.5 * rng.uniform(-1, 1, size=p.b.shape)
    if dry_fraction > 0:
        dry = rng.uniform(size=p.b.shape) < dry_fraction
        h = np.where(dry, 0.0, h)
        u = np.where(dry, 0.0, u)
        v = np.where(dry, 0.0, v)
    p.W = _state(h, u, v)
    p.name = "random_rough"
    return p


def lake_at_rest_walls(N=3, Kx=5, Ky=4, rotate_seed=None, g=9.81, walls=(True, True)) -> Problem:
    """Lake at rest h + b = 1 in the curved box [0,2]^2 closed by solid walls
    (x += 0.05 sin(pi x) sin(pi y), same for y, which keeps the walls
    straight), over the kinked bathymetry of lake_at_rest_kinked."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, Kx, Ky, (0.0, 2.0, 0.0, 2.0), _sine_map(0.05, math.pi),
                                           rotate_seed, walls)
    r = np.sqrt((xw - 0.93) ** 2 + (yw - 1.07) ** 2)
    b = 0.1 + 0.05 * np.sin(math.pi * xw) * np.cos(math.pi * yw) + 0.1 * np.maximum(0.0, 1.0 - r / 0.5)
    z = np.zeros_like(b)
    return Problem("lake_at_rest_walls", N, Kx, Ky, x, y, b, _state(1.0 - b, z, z), E, F, fl, g)


def random_walls(N=3, Kx=4, Ky=3, seed=0, rotate_seed=None, g=9.81, walls=(True, True),
                 rough=True) -> Problem:
    """Random state (independent noise per node when rough, else smooth) on a
    smooth random bathymetry in the curved box [0,2]^2 with solid walls."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, Kx, Ky, (0.0, 2.0, 0.0, 2.0), _sine_map(0.05, math.pi),
                                           rotate_seed, walls)
    rng = np.random.default_rng(seed)
    b = 0.1 * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    if rough:
        h = 1.0 + 0.3 * rng.uniform(-1, 1, size=b.shape)
        u = 0.5 * rng.uniform(-1, 1, size=b.shape)
        v = 0.5 * rng.uniform(-1, 1, size=b.shape)
    else:
        h = 1.0 + 0.2 * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
        u = 0.5 * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
        v = 0.5 * _smooth_periodic_field(rng, xw, yw, 2.0, 2.0)
    return Problem("random_walls", N, Kx, Ky, x, y, b, _state(h, u, v), E, F, fl, g)


def dry_dam_break(N=3, K1=50, g=9.81, rotate_seed=None) -> Problem:
    """Dam break into a dry region (Sec. 6.1.1): [-20,20]^2, solid walls at
    x = +-20, periodic in y, flat bottom, h = 10 for x < 0 and 0 elsewhere,
    at rest, Cartesian K1 x K1 mesh."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, K1, K1, (-20.0, 20.0, -20.0, 20.0),
                                           lambda X, Y: (0.0 * X, 0.0 * Y), rotate_seed, (True, False))
    b = np.zeros_like(xw)
    h = np.where(xw < 0.0, 10.0, 0.0)
    z = np.zeros_like(h)
    return Problem("dry_dam_break", N, K1, K1, x, y, b, _state(h, z, z), E, F, fl, g)


def three_mound_dam_break(N=3, Kx=150, Ky=100, g=9.81, rotate_seed=None) -> Problem:
    """Dam break over three mounds (Sec. 6.3): [0,75] x [0,45] closed by solid
    walls, h = 1.875 for x < 16 and dry elsewhere, at rest, bottom
    b = max(0, M1, M2, M3) (Eq. ThreeMoundBottom), Cartesian Kx x Ky mesh."""
    x, y, xw, yw, E, F, fl = periodic_mesh(N, Kx, Ky, (0.0, 75.0, 0.0, 45.0),
                                           lambda X, Y: (0.0 * X, 0.0 * Y), rotate_seed, (True, True))
    m1 = 1.0 - 0.1 * np.sqrt((xw - 30.0) ** 2 + (yw - 22.5) ** 2)
    m2 = 1.0 - 0.1 * np.sqrt((xw - 30.0) ** 2 + (yw - 7.5) ** 2)
    m3 = 2.8 - 0.28 * np.sqrt((xw - 47.5) ** 2 + (yw - 15.0) ** 2)
    b = np.maximum(np.maximum(0.0, m1), np.maximum(m2, m3))
    h = np.where(xw < 16.0, np.maximum(1.875 - b, 0.0), 0.0)
    z = np.zeros_like(h)
    return Problem("three_mound_dam_break", N, Kx, Ky, x, y, b, _state(h, z, z), E, F, fl, g)


def ensemble_member(i: int, seed=5, sizes=(16, 96), degrees=(3, 5, 7), g=9.81) -> Problem:
    """Member i of the uneven ensemble: degree drawn from `degrees`, an s x s
    curved periodic [0,2]^2 mesh with s uniform in `sizes` (inclusive), a
    bathymetry 0.3 B/max B with B a sum of 8 seeded Gaussians, and a lake at
    rest h + b = 1 with a Gaussian hump (amplitude 0.1, width 0.2)."""
    rng = np.random.default_rng([seed, i])
    N = int(rng.choice(np.asarray(degrees)))
    s = int(rng.integers(sizes[0], sizes[1] + 1))
    x, y, xw, yw, E, F, fl = periodic_mesh(N, s, s, (0.0, 2.0, 0.0, 2.0), _sine_map(0.05, math.pi))
    a = rng.uniform(0.2, 1.0, size=8)
    c = rng.uniform(0.0, 2.0, size=(8, 2))
    w = rng.uniform(0.1, 0.4, size=8)
    B = _gaussian_sum_periodic_separable(xw, yw, a, c, w, 2.0, 2.0)
    b = 0.3 * B / B.max()
    c0 = rng.uniform(0.5, 1.5, size=2)
    h = 1.0 - b + 0.1 * np.exp(-((xw - c0[0]) ** 2 + (yw - c0[1]) ** 2) / 0.2 ** 2)
    z = np.zeros_like(h)
    return Problem("ensemble_member", N, s, s, x, y, b, _state(h, z, z), E, F, fl, g,
                   {"member": i, "seed": seed})


def ensemble(ninst=256, seed=5, sizes=(16, 96), degrees=(3, 5, 7), g=9.81) -> list:
    """The uneven ensemble: `ninst` independent members (see ensemble_member)."""
    return [ensemble_member(i, seed, sizes, degrees, g) for i in range(ninst)]


def gauge_weights(prob, points):
    """Gauges of a loss functional: for each physical point the element that
    contains it and the (n, n) tensor-product Lagrange weights at its
    reference coordinates (found by Newton on the element map), so that a
    nodal field's value there is sum(weights * field[element])."""
    N, n = prob.N, prob.N + 1
    xi = lgl_points(N)

    def lag(r):
        L = np.ones(n)
        for j in range(n):
            for m in range(n):
                if m != j:
                    L[j] *= (r - xi[m]) / (xi[j] - xi[m])
        return L

    def dlag(r):
        d = np.zeros(n)
        for j in range(n):
            for l in range(n):
                if l == j:
                    continue
                t = 1.0 / (xi[j] - xi[l])
                for m in range(n):
                    if m != j and m != l:
                        t *= (r - xi[m]) / (xi[j] - xi[m])
                d[j] += t
        return d

    cx = prob.x.mean(axis=(1, 2))
    cy = prob.y.mean(axis=(1, 2))
    out = []
    for (px, py) in points:
        order = np.argsort((cx - px) ** 2 + (cy - py) ** 2)
        for k in order[:9]:
            r = s = 0.0
            for _ in range(50):
                Lr, Ls, dLr, dLs = lag(r), lag(s), dlag(r), dlag(s)
                X = Ls @ prob.x[k] @ Lr
                Y = Ls @ prob.y[k] @ Lr
                Xr, Xs = Ls @ prob.x[k] @ dLr, dLs @ prob.x[k] @ Lr
                Yr, Ys = Ls @ prob.y[k] @ dLr, dLs @ prob.y[k] @ Lr
                det = Xr * Ys - Xs * Yr
                dr = (Ys * (px - X) - Xs * (py - Y)) / det
                ds = (-Yr * (px - X) + Xr * (py - Y)) / det
                r, s = r + dr, s + ds
                if abs(dr) + abs(ds) < 1e-15:
                    break
            if abs(r) <= 1 + 1e-12 and abs(s) <= 1 + 1e-12:
                out.append((int(k), np.outer(lag(s), lag(r))))
                break
        else:
            raise ValueError(f"gauge point {(px, py)} not found in the mesh")
    return out


CONFIGS = {
    "lake_hump": lake_hump,
    "dam_break": dam_break,
    "thacker_bowl": thacker_bowl,
    "random_smooth": random_smooth,
    "random_rough": random_rough,
    "lake_at_rest_kinked": lake_at_rest_kinked,
    "lake_at_rest_walls": lake_at_rest_walls,
    "random_walls": random_walls,
    "dry_dam_break": dry_dam_break,
    "three_mound_dam_break": three_mound_dam_break,
}
