"""Multi-precision brute-force evaluation of the semi-discrete operator.

TEST INFRASTRUCTURE ONLY: a second, independent restatement of the scheme's
right-hand side, used to pin the FP64 oracle (orc.c) and to write the exact
right-hand side stored under tests/golden/. Only the tests and the golden
scripts use it; the product path never does. It shares no code with orc.c
or with the CUDA library, and it is arranged differently from orc.c on
purpose:

* arithmetic in mpmath at 40 significant digits (the float64 inputs are
  exact binary fractions, so the result is the exact right-hand side of the
  given inputs up to ~1e-38);
* LGL nodes from the roots of L_N' in multi-precision, weights
  2/(N(N+1) L_N(xi)^2), and the derivative matrix from the definition of the
  Lagrange basis (the sum over products, no barycentric or product formula);
* neighbours found by matching the physical coordinates of face nodes up to a
  period shift (with opposite outward normals), not through EToE, EToF and
  flip: every element evaluates the interface flux of each of its own face
  nodes from its own side, with its own outward normal; a face with no
  partner is a solid wall (mirror state);
* the strong form with 2D and explicit surface corrections
  (1/w_end)(F*_out - f~_out) at every face node (Sec. 2.2, Eq. fluxDiffFormF
  with D~ = 2D + S unfolded), where orc.c sums D~ and adds F* alone;
* the BR1 gradients (Eq. BR1, metrics outside the derivative) in strong form
  with (U* - u) lifts, where orc.c uses the weak operator D^ with U* lifts.

What it computes (W_t = R): J R = -(L_xi + L_eta) + S + L^v with
  L_xi  = sum_m 2 D_im F~(i,m),  F~ = F# {y_eta} - G# {x_eta}     (Eq. Fmij)
  L_eta = sum_m 2 D_jm G~(j,m),  G~ = -F# {y_xi} + G# {x_xi}
  F#, G# the entropy-conservative well-balanced fluxes of Eq. volumeFluxes,
  surface corrections (1/w_end)(J^surf F*(W_own, W_nb, n) - f(W_own).n~),
  F* the rotated EC flux of Eq. surfaceFluxes minus, for the entropy-stable
  flux, 1/2 R|L|R^T [[q]] (Eqs. RightEigenvectors2DCurved,
  ScalingMatrix2DCurved), rotated back (Eq. surfaceFlux2DRotated);
  S = (0, -g/2 h beta_x, +g/2 h beta_y) with the split bathymetry derivatives
  beta_x = y_eta D_xi b + D_xi(y_eta b) - y_xi D_eta b - D_eta(y_xi b),
  beta_y = x_eta D_xi b + D_xi(x_eta b) - x_xi D_eta b - D_eta(x_xi b)
  (Eq. SourceDisc read with plain D and the sign that makes the lake at rest
  exact); L^v the BR1 viscous divergence of Eq. ViscTermsDisc with the
  element viscosities passed in (the smoothness indicator is not restated).
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

DPS = 40


def _mp(a):
    return mp.mpf(float(a))


def lgl(N):
    """LGL nodes, weights and the derivative matrix D_ij = l_j'(xi_i) in
    multi-precision (roots of L_N' by mpmath, D from the Lagrange basis)."""
    with mp.workdps(DPS + 10):
        # Legendre coefficients of L_N in the monomial basis (Bonnet recursion)
        P = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
        for k in range(1, N):
            a = [mp.mpf(0)] + [(2 * k + 1) * c for c in P[k]]
            b = [k * c for c in P[k - 1]] + [mp.mpf(0), mp.mpf(0)]
            P.append([(a[i] - b[i]) / (k + 1) for i in range(k + 2)])
        LN = P[N]
        dLN = [i * LN[i] for i in range(1, N + 1)]  # ascending
        inner = []
        if N >= 2:
            roots = mp.polyroots(list(reversed(dLN)), maxsteps=200, extraprec=200)
            inner = sorted(mp.re(r) for r in roots)
        xi = [mp.mpf(-1)] + inner + [mp.mpf(1)]
        LNv = lambda x: sum(c * x ** i for i, c in enumerate(LN))
        w = [mp.mpf(2) / (N * (N + 1) * LNv(x) ** 2) for x in xi]
        n = N + 1
        D = [[mp.mpf(0)] * n for _ in range(n)]
        for i in range(n):
            for j in range(n):
                s = mp.mpf(0)
                for m in range(n):
                    if m == j:
                        continue
                    prod = mp.mpf(1) / (xi[j] - xi[m])
                    for l in range(n):
                        if l in (j, m):
                            continue
                        prod *= (xi[i] - xi[l]) / (xi[j] - xi[l])
                    s += prod
                D[i][j] = s
    return xi, w, D


def _face_nodes(N, f):
    """(i, j) of the face nodes of face f (0: eta=-1, 1: xi=+1, 2: eta=+1, 3: xi=-1)."""
    p = range(N + 1)
    if f == 0:
        return [(q, 0) for q in p]
    if f == 1:
        return [(N, q) for q in p]
    if f == 2:
        return [(q, N) for q in p]
    return [(0, q) for q in p]


class BruteForce:
    """Right-hand side of one problem (x, y, b as [K][n][n] float arrays
    indexed [k, j, i]) in multi-precision. periods: the lattice of shifts
    under which the mesh is periodic (e.g. [(2, 0), (0, 2)])."""

    def __init__(self, N, x, y, b, g, periods=((2.0, 0.0), (0.0, 2.0)), tol=1e-9):
        mp.mp.dps = DPS
        self.N, self.n = N, N + 1
        self.K = x.shape[0]
        self.g = _mp(g)
        self.xf, self.yf = np.asarray(x, float), np.asarray(y, float)
        self.xi, self.w, self.D = lgl(N)
        n, K = self.n, self.K
        X = [[[_mp(x[k, j, i]) for i in range(n)] for j in range(n)] for k in range(K)]
        Y = [[[_mp(y[k, j, i]) for i in range(n)] for j in range(n)] for k in range(K)]
        self.b = [[[_mp(b[k, j, i]) for i in range(n)] for j in range(n)] for k in range(K)]
        D = self.D
        self.x_xi, self.x_eta, self.y_xi, self.y_eta, self.J = ([] for _ in range(5))
        for k in range(K):
            dx = lambda F, i, j: sum(D[i][m] * F[j][m] for m in range(n))
            de = lambda F, i, j: sum(D[j][m] * F[m][i] for m in range(n))
            xx = [[dx(X[k], i, j) for i in range(n)] for j in range(n)]
            xe = [[de(X[k], i, j) for i in range(n)] for j in range(n)]
            yx = [[dx(Y[k], i, j) for i in range(n)] for j in range(n)]
            ye = [[de(Y[k], i, j) for i in range(n)] for j in range(n)]
            self.x_xi.append(xx)
            self.x_eta.append(xe)
            self.y_xi.append(yx)
            self.y_eta.append(ye)
            self.J.append([[xx[j][i] * ye[j][i] - xe[j][i] * yx[j][i] for i in range(n)] for j in range(n)])
        self._match(periods, tol)

    # --- geometry -----------------------------------------------------------

    def normal(self, k, f, i, j):
        """Outward unscaled normal at node (i, j) of face f of element k."""
        if f == 1:
            return self.y_eta[k][j][i], -self.x_eta[k][j][i]
        if f == 3:
            return -self.y_eta[k][j][i], self.x_eta[k][j][i]
        if f == 2:
            return -self.y_xi[k][j][i], self.x_xi[k][j][i]
        return self.y_xi[k][j][i], -self.x_xi[k][j][i]

    def _match(self, periods, tol):
        """partner[(k, f, i, j)] = (k', i', j') or None (wall), from coordinates."""
        shifts = [(0.0, 0.0)]
        for a in ((-1, 0, 1) if periods else ()):
            for c in (-1, 0, 1):
                s = (a * periods[0][0] + c * periods[1][0], a * periods[0][1] + c * periods[1][1]) \
                    if len(periods) == 2 else (a * periods[0][0], a * periods[0][1])
                if s not in shifts:
                    shifts.append(s)
        N, K = self.N, self.K
        faces = [(k, f) for k in range(K) for f in range(4)]
        pos = {(k, f): [(self.xf[k, j, i], self.yf[k, j, i]) for (i, j) in _face_nodes(N, f)]
               for (k, f) in faces}
        self.partner = {}
        for (k, f) in faces:
            found = None
            for (kk, ff) in faces:
                for s in shifts:
                    if (kk, ff) == (k, f) and s == (0.0, 0.0):
                        continue
                    pairs = []
                    for p, (px, py) in enumerate(pos[(k, f)]):
                        q = [q for q, (qx, qy) in enumerate(pos[(kk, ff)])
                             if abs(qx - px - s[0]) < tol and abs(qy - py - s[1]) < tol]
                        if len(q) != 1:
                            break
                        pairs.append((p, q[0]))
                    if len(pairs) != N + 1:
                        continue
                    # outward normals must be opposite at matched nodes
                    ok = True
                    for p, q in pairs:
                        i, j = _face_nodes(N, f)[p]
                        ii, jj = _face_nodes(N, ff)[q]
                        a = self.normal(k, f, i, j)
                        c = self.normal(kk, ff, ii, jj)
                        if a[0] * c[0] + a[1] * c[1] >= 0:
                            ok = False
                    if ok:
                        found = (kk, ff, pairs)
                        break
                if found:
                    break
            for p, (i, j) in enumerate(_face_nodes(N, f)):
                if found is None:
                    self.partner[(k, f, i, j)] = None
                else:
                    kk, ff, pairs = found
                    q = dict(pairs)[p]
                    ii, jj = _face_nodes(N, ff)[q]
                    self.partner[(k, f, i, j)] = (kk, ii, jj)

    # --- pointwise physics --------------------------------------------------

    def _vel(self, h, m):
        return m / h if h > 0 else mp.mpf(0)

    def _phys(self, W):
        g = self.g
        h, hu, hv = W
        u, v = self._vel(h, hu), self._vel(h, hv)
        p = g * h * h / 2
        return [hu, hu * u + p, hu * v], [hv, hv * u, hv * v + p]

    def _two_point(self, Wa, Wb):
        g = self.g
        ha, hb = Wa[0], Wb[0]
        ua, va = self._vel(ha, Wa[1]), self._vel(ha, Wa[2])
        ub, vb = self._vel(hb, Wb[1]), self._vel(hb, Wb[2])
        hu = (Wa[1] + Wb[1]) / 2
        hv = (Wa[2] + Wb[2]) / 2
        um, vm = (ua + ub) / 2, (va + vb) / 2
        p = g * ha * hb / 2  # g {h}^2 - g/2 {h^2}
        return [hu, hu * um + p, hu * vm], [hv, hv * um, hv * vm + p]

    def _interface(self, Wm, Wp, bm, bp, nx, ny, es):
        """F*(W-, W+) through the unit normal (nx, ny), physical frame."""
        g = self.g
        T = [[nx, ny], [-ny, nx]]
        def rot(W):
            h = W[0]
            u, v = self._vel(h, W[1]), self._vel(h, W[2])
            return h, T[0][0] * u + T[0][1] * v, T[1][0] * u + T[1][1] * v
        hm, um, vm = rot(Wm)
        hp, up, vp = rot(Wp)
        ha, ua, va = (hm + hp) / 2, (um + up) / 2, (vm + vp) / 2
        Fr = [ha * ua, ha * ua * ua + g * (hm * hm + hp * hp) / 4, ha * ua * va]
        if es:
            ca = (mp.sqrt(g * max(hm, 0)) + mp.sqrt(g * max(hp, 0))) / 2
            q = lambda h, b, u, v: [g * (h + b) - (u * u + v * v) / 2, u, v]
            dq = [a - c for a, c in zip(q(hp, bp, up, vp), q(hm, bm, um, vm))]
            Rm = mp.matrix([[1, 0, 1], [ua + ca, 0, ua - ca], [va, 1, va]])
            Lm = mp.diag([abs(ua + ca) / (2 * g), abs(ha * ua), abs(ua - ca) / (2 * g)])
            d = Rm * Lm * Rm.T * mp.matrix(dq)
            Fr = [Fr[c] - d[c] / 2 for c in range(3)]
        # back to the physical frame: momentum components by T^T
        return [Fr[0], T[0][0] * Fr[1] + T[1][0] * Fr[2], T[0][1] * Fr[1] + T[1][1] * Fr[2]]

    # --- operator -----------------------------------------------------------

    def rhs(self, W, flux=1, eps=None, elements=None):
        """R(W) as float64 [3][K][n][n]; eps: per-element viscosity (None: no
        AV); elements: evaluate only these elements (the rest stay zero)."""
        N, n, K, g = self.N, self.n, self.K, self.g
        D, w = self.D, self.w
        S = [[[[_mp(W[c, k, j, i]) for i in range(n)] for j in range(n)] for k in range(K)]
             for c in range(3)]
        st = lambda k, i, j: [S[0][k][j][i], S[1][k][j][i], S[2][k][j][i]]
        bb = lambda k, i, j: self.b[k][j][i]

        def neighbour_state(k, f, i, j):
            nb = self.partner[(k, f, i, j)]
            Wo = st(k, i, j)
            if nb is not None:
                kk, ii, jj = nb
                return st(kk, ii, jj), bb(kk, ii, jj), nb
            nx, ny = self.normal(k, f, i, j)
            js = mp.sqrt(nx * nx + ny * ny)
            nx, ny = nx / js, ny / js
            mn = Wo[1] * nx + Wo[2] * ny
            return [Wo[0], Wo[1] - 2 * mn * nx, Wo[2] - 2 * mn * ny], bb(k, i, j), None

        # BR1 gradients and viscous fluxes (element viscosities given)
        visc = eps is not None and any(float(e) != 0.0 for e in eps)
        if visc:
            vel = lambda k, i, j: (self._vel(S[0][k][j][i], S[1][k][j][i]),
                                   self._vel(S[0][k][j][i], S[2][k][j][i]))
            grad = {}
            for k in range(K):
                for j in range(n):
                    for i in range(n):
                        out = []
                        for c in range(2):
                            f_ = lambda a, b_: vel(k, a, b_)[c]
                            dxi = sum(D[i][m] * f_(m, j) for m in range(n))
                            det = sum(D[j][m] * f_(i, m) for m in range(n))
                            for fc, end, sgn, along in ((1, N, 1, "xi"), (3, 0, -1, "xi"),
                                                        (2, N, 1, "eta"), (0, 0, -1, "eta")):
                                if (i if along == "xi" else j) != end:
                                    continue
                                nb = self.partner[(k, fc, i, j)]
                                own = f_(i, j)
                                star = own if nb is None else (own + vel(*nb)[c]) / 2
                                if along == "xi":
                                    dxi += sgn * (star - own) / w[end]
                                else:
                                    det += sgn * (star - own) / w[end]
                            ye, yx = self.y_eta[k][j][i], self.y_xi[k][j][i]
                            xe, xx = self.x_eta[k][j][i], self.x_xi[k][j][i]
                            Jn = self.J[k][j][i]
                            out.append(((ye * dxi - yx * det) / Jn, (-xe * dxi + xx * det) / Jn))
                        grad[(k, i, j)] = out  # [(U1, U2), (V1, V2)]

            def vflux(k, i, j):
                he = S[0][k][j][i] * _mp(eps[k])
                (U1, U2), (V1, V2) = grad[(k, i, j)]
                return [0, he * U1, he * V1], [0, he * U2, he * V2]

        R = np.zeros((3, K, n, n))
        for k in (range(K) if elements is None else elements):
            for j in range(n):
                for i in range(n):
                    Wo = st(k, i, j)
                    L = [mp.mpf(0)] * 3
                    for m in range(n):
                        Fs, Gs = self._two_point(Wo, st(k, m, j))
                        ye = (self.y_eta[k][j][i] + self.y_eta[k][j][m]) / 2
                        xe = (self.x_eta[k][j][i] + self.x_eta[k][j][m]) / 2
                        for c in range(3):
                            L[c] += 2 * D[i][m] * (Fs[c] * ye - Gs[c] * xe)
                        Fs, Gs = self._two_point(Wo, st(k, i, m))
                        yx = (self.y_xi[k][j][i] + self.y_xi[k][m][i]) / 2
                        xx = (self.x_xi[k][j][i] + self.x_xi[k][m][i]) / 2
                        for c in range(3):
                            L[c] += 2 * D[j][m] * (-Fs[c] * yx + Gs[c] * xx)
                    f_o, g_o = self._phys(Wo)
                    Lv = [mp.mpf(0)] * 3
                    if visc:
                        for c in (1, 2):
                            sx = mp.mpf(0)
                            for m in range(n):
                                Fv, Gv = vflux(k, m, j)
                                sx += D[i][m] * (self.y_eta[k][j][m] * Fv[c] - self.x_eta[k][j][m] * Gv[c])
                                Fv, Gv = vflux(k, i, m)
                                sx += D[j][m] * (-self.y_xi[k][m][i] * Fv[c] + self.x_xi[k][m][i] * Gv[c])
                            Lv[c] = sx
                    for f in range(4):
                        if (i, j) not in _face_nodes(N, f):
                            continue
                        wend = w[N] if f in (1, 2) else w[0]
                        nx, ny = self.normal(k, f, i, j)
                        js = mp.sqrt(nx * nx + ny * ny)
                        Wn, bn, nb = neighbour_state(k, f, i, j)
                        Fst = self._interface(Wo, Wn, bb(k, i, j), bn, nx / js, ny / js, flux)
                        for c in range(3):
                            L[c] += (js * Fst[c] - (f_o[c] * nx + g_o[c] * ny)) / wend
                        if visc:
                            Fo, Go = vflux(k, i, j)
                            for c in (1, 2):
                                own = Fo[c] * nx + Go[c] * ny
                                if nb is None:
                                    avg = mp.mpf(0)
                                else:
                                    Fn, Gn = vflux(*nb)
                                    avg = (own + Fn[c] * nx + Gn[c] * ny) / 2
                                Lv[c] += (avg - own) / wend
                    # split bathymetry derivatives
                    bk = self.b[k]
                    ye, yx = self.y_eta[k], self.y_xi[k]
                    xe, xx = self.x_eta[k], self.x_xi[k]
                    Dx = lambda F: sum(D[i][m] * F(m, j) for m in range(n))
                    De = lambda F: sum(D[j][m] * F(i, m) for m in range(n))
                    bx_ = Dx(lambda a, c_: bk[c_][a])
                    be_ = De(lambda a, c_: bk[c_][a])
                    beta_x = (ye[j][i] * bx_ + Dx(lambda a, c_: ye[c_][a] * bk[c_][a])
                              - yx[j][i] * be_ - De(lambda a, c_: yx[c_][a] * bk[c_][a]))
                    beta_y = (xe[j][i] * bx_ + Dx(lambda a, c_: xe[c_][a] * bk[c_][a])
                              - xx[j][i] * be_ - De(lambda a, c_: xx[c_][a] * bk[c_][a]))
                    src = [mp.mpf(0), -g * Wo[0] * beta_x / 2, g * Wo[0] * beta_y / 2]
                    Jn = self.J[k][j][i]
                    for c in range(3):
                        R[c, k, j, i] = float((-L[c] + src[c] + Lv[c]) / Jn)
        return R
