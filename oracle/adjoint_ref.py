"""CPU reference of the discrete adjoint.

TEST INFRASTRUCTURE ONLY: the tests use it to check the CUDA library's
adjoint kernels; the product path never imports it.

The scheme of orc.c (split-form volume term of Eq. fluxDiffFormF with the
fluxes of Eqs. Fmij and volumeFluxes, the interface flux of Eq. fesandges in
the rotated frame of App. B, the well-balanced source of Eq. SourceDisc, the
BR1 viscous terms of Eqs. BR1 and ViscTermsDisc, solid walls by the mirror
state, the limiter of Eq. PosPres and the LSRK4(5) / SSPRK3 steps) restated
with plain float64 PyTorch operations on the CPU, element-vectorised but
with no other restructuring, so that torch.autograd gives exact
vector-Jacobian products of the discrete operator. It follows orc.c term by
term and is pinned to it by the tests (same right-hand side to rounding) and
to central finite differences of orc.c (same derivatives).

What the adjoint holds fixed, as decided on the forward pass: the element
viscosities eps_k (the viscosity switch of App. A), the limiter's active
set (which elements are limited and the node attaining their minimum; theta
itself is differentiated), the nodes cut by h_tol, and the step sizes dt.
"""
from __future__ import annotations


import numpy as np
import torch

from . import oracle as O

LSRK_A = [0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0]
LSRK_B = [1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
          1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
          2277821191437.0 / 14882151754819.0]

_T = dict(dtype=torch.float64)


def _face_nodes(N, f):
    p = np.arange(N + 1)
    if f == 0:
        return p, np.zeros_like(p)
    if f == 1:
        return np.full_like(p, N), p
    if f == 2:
        return p, np.full_like(p, N)
    return np.zeros_like(p), p


class Twin:
    """The discrete scheme of one problem as differentiable torch functions.

    Arrays follow the library's layout: nodal [K, n, n] indexed [k, j, i]
    (i along xi), states [3, K, n, n]."""

    def __init__(self, prob, flux=1, av=False, limiter=False, h_tol=1e-4, rk=0):
        self.N, self.K, self.n = prob.N, prob.K, prob.N + 1
        self.g = float(prob.g)
        self.flux, self.av, self.limiter, self.h_tol, self.rk = int(flux), bool(av), bool(limiter), h_tol, rk
        N, n, K = self.N, self.n, self.K
        xi, w, D, V, Vinv = O.basis(N)
        self.w = torch.tensor(w, **_T)
        self.D = torch.tensor(D, **_T)
        S = np.zeros((n, n))
        S[0, 0], S[N, N] = 1.0 / w[0], -1.0 / w[N]
        self.Dt = torch.tensor(2.0 * D + S, **_T)                      # D~ = 2D + S
        self.Dh = torch.tensor(-(D.T * w[None, :]) / w[:, None], **_T)  # D^ = -M^-1 D^T M
        x = torch.tensor(np.ascontiguousarray(prob.x), **_T)
        y = torch.tensor(np.ascontiguousarray(prob.y), **_T)
        self.x_xi, self.y_xi = self.dxi(x), self.dxi(y)
        self.x_eta, self.y_eta = self.deta(x), self.deta(y)
        self.J = self.x_xi * self.y_eta - self.x_eta * self.y_xi
        self.wJ = self.w[None, :, None] * self.w[None, None, :] * self.J
        self._faces(prob)

    # ---- derivative operators along xi (last axis) and eta (middle axis) ----
    def dxi(self, f, M=None):
        return torch.einsum("im,...jm->...ji", self.D if M is None else M, f)

    def deta(self, f, M=None):
        return torch.einsum("jm,...mi->...ji", self.D if M is None else M, f)

    # ---- connectivity ----------------------------------------------------
    def _faces(self, prob):
        N, n, K = self.N, self.n, self.K
        E, F, fl = prob.EToE, prob.EToF, prob.flip
        own_face, own_nodes, nb_nodes, nb_slots, own_slots = [], [], [], [], []
        wall_slots, wall_nodes = [], []
        for k in range(K):
            for f in range(4):
                i, j = _face_nodes(N, f)
                nodes = k * n * n + j * n + i
                slots = (k * 4 + f) * n + np.arange(n)
                kk, ff = int(E[k, f]), int(F[k, f])
                if kk < 0:
                    wall_slots.append(slots)
                    wall_nodes.append(nodes)
                    continue
                if not (kk > k or (kk == k and ff > f)):
                    continue
                q = np.arange(n)[::-1] if fl[k, f] else np.arange(n)
                ii, jj = _face_nodes(N, ff)
                own_face.append((k, f))
                own_nodes.append(nodes)
                own_slots.append(slots)
                nb_nodes.append(kk * n * n + jj[q] * n + ii[q])
                nb_slots.append((kk * 4 + ff) * n + q)
        cat = lambda L: torch.tensor(np.concatenate(L) if L else np.zeros(0, dtype=np.int64), dtype=torch.long)
        self.f_own, self.f_nb = cat(own_nodes), cat(nb_nodes)
        self.f_town, self.f_tnb = cat(own_slots), cat(nb_slots)
        self.w_slot, self.w_node = cat(wall_slots), cat(wall_nodes)
        # owner's outward unscaled normal at every unique face node and wall node
        nx_all, ny_all = self._side_normals()
        self.f_nx = nx_all[self.f_town]
        self.f_ny = ny_all[self.f_town]
        self.w_nx = nx_all[self.w_slot]
        self.w_ny = ny_all[self.w_slot]

    def _side_normals(self):
        """Outward unscaled normal at every element side node, [K*4*n]."""
        N = self.N
        out_x, out_y = [], []
        sl = {0: (slice(None), 0, slice(None)), 1: (slice(None), slice(None), N),
              2: (slice(None), N, slice(None)), 3: (slice(None), slice(None), 0)}
        for f in range(4):
            s = sl[f]
            if f == 0:
                nx, ny = self.y_xi[s], -self.x_xi[s]
            elif f == 1:
                nx, ny = self.y_eta[s], -self.x_eta[s]
            elif f == 2:
                nx, ny = -self.y_xi[s], self.x_xi[s]
            else:
                nx, ny = -self.y_eta[s], self.x_eta[s]
            out_x.append(nx)
            out_y.append(ny)
        return torch.stack(out_x, 1).reshape(-1), torch.stack(out_y, 1).reshape(-1)

    # ---- pointwise pieces --------------------------------------------------
    @staticmethod
    def velocity(h, hu):
        pos = h > 0
        return torch.where(pos, hu / torch.where(pos, h, torch.ones_like(h)), torch.zeros_like(h))

    def celerity(self, h):
        """c = sqrt(g max(h, 0)); its derivative is taken as 0 where h <= 0."""
        wet = h > 0
        return torch.where(wet, torch.sqrt(self.g * torch.where(wet, h, torch.ones_like(h))), torch.zeros_like(h))

    def surface_flux(self, Wm, Wp, bm, bp, nx, ny):
        """Eq. fesandges in the rotated frame (App. B), rotated back."""
        g = self.g
        hm, hp = Wm[0], Wp[0]
        um, vm = self.velocity(hm, Wm[1]), self.velocity(hm, Wm[2])
        up, vp = self.velocity(hp, Wp[1]), self.velocity(hp, Wp[2])
        utm, vtm = nx * um + ny * vm, -ny * um + nx * vm
        utp, vtp = nx * up + ny * vp, -ny * up + nx * vp
        ha, h2a = 0.5 * (hm + hp), 0.5 * (hm * hm + hp * hp)
        ua, va = 0.5 * (utm + utp), 0.5 * (vtm + vtp)
        F = [ha * ua, ha * ua * ua + 0.5 * g * h2a, ha * ua * va]
        if self.flux:
            cm, cp = self.celerity(hm), self.celerity(hp)
            ca = 0.5 * (cm + cp)
            qm = [g * (hm + bm) - 0.5 * (utm * utm + vtm * vtm), utm, vtm]
            qp = [g * (hp + bp) - 0.5 * (utp * utp + vtp * vtp), utp, vtp]
            dq = [qp[a] - qm[a] for a in range(3)]
            one, zero = torch.ones_like(ha), torch.zeros_like(ha)
            R = [[one, zero, one], [ua + ca, zero, ua - ca], [va, one, va]]
            lam = [torch.abs(ua + ca) / (2 * g), torch.abs(ha * ua), torch.abs(ua - ca) / (2 * g)]
            t = [lam[a] * sum(R[c][a] * dq[c] for c in range(3)) for a in range(3)]
            F = [F[a] - 0.5 * sum(R[a][c] * t[c] for c in range(3)) for a in range(3)]
        return torch.stack([F[0], nx * F[1] - ny * F[2], ny * F[1] + nx * F[2]])

    # ---- the right-hand side ---------------------------------------------
    def rhs(self, W, b, eps=None):
        """R(W) of Eq. CurvilinearECDGSEMviscous divided by J; b enters the
        source and the interface flux; eps [K] (no gradient) when av."""
        N, n, K, g = self.N, self.n, self.K, self.g
        h, hu, hv = W[0], W[1], W[2]
        u, v = self.velocity(h, hu), self.velocity(h, hv)
        # volume term, xi pairs (node i, partner m along the same eta-line)
        Lxi = self._pairs(h, hu, hv, u, v, axis="xi")
        Leta = self._pairs(h, hu, hv, u, v, axis="eta")
        # interface flux of every side slot
        Fs = self._interface(W, b)
        Fs = Fs.reshape(3, K, 4, n)
        Lxi = Lxi.clone()
        Leta = Leta.clone()
        Lxi[:, :, :, N] = Lxi[:, :, :, N] + Fs[:, :, 1, :] / self.w[N]
        Lxi[:, :, :, 0] = Lxi[:, :, :, 0] + Fs[:, :, 3, :] / self.w[0]
        Leta[:, :, N, :] = Leta[:, :, N, :] + Fs[:, :, 2, :] / self.w[N]
        Leta[:, :, 0, :] = Leta[:, :, 0, :] + Fs[:, :, 0, :] / self.w[0]
        # split-form source (Eq. SourceDisc, reading of orc.c)
        bx, be = self.dxi(b), self.deta(b)
        beta_x = self.y_eta * bx + self.dxi(self.y_eta * b) - self.y_xi * be - self.deta(self.y_xi * b)
        beta_y = self.x_eta * bx + self.dxi(self.x_eta * b) - self.x_xi * be - self.deta(self.x_xi * b)
        S = torch.stack([torch.zeros_like(h), -0.5 * g * h * beta_x, 0.5 * g * h * beta_y])
        R = -Lxi - Leta + S
        if self.av:
            R = R + self._viscous(W, u, v, eps)
        return R / self.J

    def _pairs(self, h, hu, hv, u, v, axis):
        g = self.g
        if axis == "xi":
            a = lambda f: f[:, :, :, None]   # node (j, i)
            c = lambda f: f[:, :, None, :]   # partner (j, m)
            my, mx = self.y_eta, self.x_eta
            sgn = 1.0
        else:
            a = lambda f: f.transpose(1, 2)[:, :, :, None]   # node, indexed [k, i, j]
            c = lambda f: f.transpose(1, 2)[:, :, None, :]   # partner (m, i)
            my, mx = self.y_xi, self.x_xi
            sgn = -1.0
        ha, hb = a(h), c(h)
        havg, h2avg = 0.5 * (ha + hb), 0.5 * (ha * ha + hb * hb)
        huavg, hvavg = 0.5 * (a(hu) + c(hu)), 0.5 * (a(hv) + c(hv))
        uavg, vavg = 0.5 * (a(u) + c(u)), 0.5 * (a(v) + c(v))
        p = g * havg * havg - 0.5 * g * h2avg
        Fs = [huavg, huavg * uavg + p, huavg * vavg]
        Gs = [hvavg, hvavg * uavg, hvavg * vavg + p]
        myavg, mxavg = 0.5 * (a(my) + c(my)), 0.5 * (a(mx) + c(mx))
        out = []
        for q in range(3):
            Ft = sgn * (Fs[q] * myavg - Gs[q] * mxavg)  # xi: F# y_eta - G# x_eta; eta: -F# y_xi + G# x_xi
            L = torch.einsum("im,kxim->kxi", self.Dt, Ft)
            out.append(L if axis == "xi" else L.transpose(1, 2))
        return torch.stack(out)

    def _interface(self, W, b):
        """Outward interface flux x Jsurf at every side slot, [3, K*4*n]."""
        K, n = self.K, self.n
        Wf = W.reshape(3, -1)
        bf = b.reshape(-1)
        Fs = torch.zeros(3, K * 4 * n, **_T)
        if self.f_own.numel():
            js = torch.sqrt(self.f_nx ** 2 + self.f_ny ** 2)
            F = self.surface_flux(Wf[:, self.f_own], Wf[:, self.f_nb], bf[self.f_own], bf[self.f_nb],
                                  self.f_nx / js, self.f_ny / js) * js
            Fs = Fs.index_copy(1, self.f_town, F)
            Fs = Fs.index_copy(1, self.f_tnb, -F)
        if self.w_slot.numel():
            js = torch.sqrt(self.w_nx ** 2 + self.w_ny ** 2)
            nx, ny = self.w_nx / js, self.w_ny / js
            Wm = Wf[:, self.w_node]
            mn = Wm[1] * nx + Wm[2] * ny
            Wg = torch.stack([Wm[0], Wm[1] - 2.0 * mn * nx, Wm[2] - 2.0 * mn * ny])
            F = self.surface_flux(Wm, Wg, bf[self.w_node], bf[self.w_node], nx, ny) * js
            Fs = Fs.index_copy(1, self.w_slot, F)
        return Fs

    def _viscous(self, W, u, v, eps):
        """BR1 (Eq. BR1, weak form with D^) and Eq. ViscTermsDisc with eps fixed."""
        N, n, K = self.N, self.n, self.K
        eps = torch.as_tensor(eps, **_T).detach()
        uf, vf = u.reshape(-1), v.reshape(-1)
        Us = torch.zeros(2, K * 4 * n, **_T)
        if self.f_own.numel():
            us = 0.5 * (uf[self.f_own] + uf[self.f_nb])
            vs = 0.5 * (vf[self.f_own] + vf[self.f_nb])
            st = torch.stack([us, vs])
            Us = Us.index_copy(1, self.f_town, st)
            Us = Us.index_copy(1, self.f_tnb, st)
        if self.w_slot.numel():
            Us = Us.index_copy(1, self.w_slot, torch.stack([uf[self.w_node], vf[self.w_node]]))
        Us = Us.reshape(2, K, 4, n)
        wi = self.w[None, None, :]
        wj = self.w[None, :, None]
        grads = []
        for c, f in enumerate((u, v)):
            dx, de = self.dxi(f, self.Dh), self.deta(f, self.Dh)
            # U* at xi = +-1 (faces 1, 3) and eta = +-1 (faces 2, 0), signed by the side
            Lx = torch.zeros_like(f)
            Le = torch.zeros_like(f)
            Lx[:, :, N] = Us[c, :, 1, :]
            Lx[:, :, 0] = -Us[c, :, 3, :]
            Le[:, N, :] = Us[c, :, 2, :]
            Le[:, 0, :] = -Us[c, :, 0, :]
            J1 = self.y_eta * dx - self.y_xi * de + self.y_eta / wi * Lx - self.y_xi / wj * Le
            J2 = -self.x_eta * dx + self.x_xi * de - self.x_eta / wi * Lx + self.x_xi / wj * Le
            grads.append((J1 / self.J, J2 / self.J))
        (U1, U2), (V1, V2) = grads
        he = W[0] * eps[:, None, None]
        Fv = [he * U1, he * V1]
        Gv = [he * U2, he * V2]
        # interface average {F^v . n} with the owner's unscaled normal, zero at walls
        Fvs = torch.zeros(2, K * 4 * n, **_T)
        if self.f_own.numel():
            avgs = []
            for c in range(2):
                a = Fv[c].reshape(-1)
                bb = Gv[c].reshape(-1)
                avgs.append(0.5 * ((self.f_nx * a[self.f_own] + self.f_ny * bb[self.f_own]) +
                                   (self.f_nx * a[self.f_nb] + self.f_ny * bb[self.f_nb])))
            avg = torch.stack(avgs)
            Fvs = Fvs.index_copy(1, self.f_town, avg)
            Fvs = Fvs.index_copy(1, self.f_tnb, -avg)
        Fvs = Fvs.reshape(2, K, 4, n)
        out = [torch.zeros_like(W[0])]
        for c in range(2):
            Ft = self.y_eta * Fv[c] - self.x_eta * Gv[c]
            Gt = -self.y_xi * Fv[c] + self.x_xi * Gv[c]
            sx = self.dxi(Ft)
            se = self.deta(Gt)
            sx = sx.clone()
            se = se.clone()
            sx[:, :, N] = sx[:, :, N] + (Fvs[c, :, 1, :] - Ft[:, :, N]) / self.w[N]
            sx[:, :, 0] = sx[:, :, 0] + (Fvs[c, :, 3, :] + Ft[:, :, 0]) / self.w[0]
            se[:, N, :] = se[:, N, :] + (Fvs[c, :, 2, :] - Gt[:, N, :]) / self.w[N]
            se[:, 0, :] = se[:, 0, :] + (Fvs[c, :, 0, :] + Gt[:, 0, :]) / self.w[0]
            out.append(sx + se)
        return torch.stack(out)

    # ---- limiter with a frozen active set -----------------------------------
    def limiter_plan(self, W):
        """Active set of Eq. PosPres on W (no gradient): limited elements,
        the node of their minimum, and the h_tol cut mask of the result."""
        with torch.no_grad():
            vol = self.wJ.sum(dim=(1, 2))
            mean = (self.wJ * W[0]).sum(dim=(1, 2)) / vol
            flat = W[0].reshape(self.K, -1)
            hmin, arg = flat.min(dim=1)
            active = (hmin < 0.0) & (mean - hmin > 0.0)
            Wl = self.limit(W, (active, arg, None))
            cut = Wl[0] < self.h_tol
        return active, arg, cut

    def limit(self, W, plan):
        active, arg, cut = plan
        vol = self.wJ.sum(dim=(1, 2))
        means = (self.wJ[None] * W).sum(dim=(2, 3)) / vol[None]        # [3, K]
        hmin = W[0].reshape(self.K, -1).gather(1, arg[:, None])[:, 0]
        denom = torch.where(active, means[0] - hmin, torch.ones_like(hmin))
        theta = torch.where(active, torch.minimum(torch.ones_like(hmin), means[0] / denom), torch.ones_like(hmin))
        th = theta[None, :, None, None]
        mb = means[:, :, None, None]
        Wl = torch.where(active[None, :, None, None], th * (W - mb) + mb, W)
        if cut is not None:
            zero = torch.zeros_like(Wl[1])
            Wl = torch.stack([Wl[0], torch.where(cut, zero, Wl[1]), torch.where(cut, zero, Wl[2])])
        return Wl

    # ---- one step with frozen decisions -------------------------------------
    def step(self, W, b, dt, eps_list, plans):
        """One LSRK4(5) or SSPRK3 step with the stage viscosities eps_list and
        the limiter plans (one per stage, None without limiter)."""
        if self.rk == 0:
            Kr = torch.zeros_like(W)
            for st in range(5):
                R = self.rhs(W, b, eps_list[st])
                Kr = LSRK_A[st] * Kr + dt * R
                W = W + LSRK_B[st] * Kr
                if self.limiter:
                    W = self.limit(W, plans[st])
            return W
        Wn = W
        W = Wn + dt * self.rhs(Wn, b, eps_list[0])
        if self.limiter:
            W = self.limit(W, plans[0])
        W = 0.75 * Wn + 0.25 * (W + dt * self.rhs(W, b, eps_list[1]))
        if self.limiter:
            W = self.limit(W, plans[1])
        W = Wn / 3.0 + 2.0 / 3.0 * (W + dt * self.rhs(W, b, eps_list[2]))
        if self.limiter:
            W = self.limit(W, plans[2])
        return W
