// Adjoint (vector-Jacobian product) kernels of the right-hand side and of
// the Runge-Kutta stage update with the positivity limiter, for gradients of
// a loss of the final or intermediate states with respect to the state and
// the bathymetry. The paper has no adjoint; these kernels differentiate the
// discrete forward kernels of this library exactly (up to rounding), with
// the decisions of the forward pass held fixed: the element viscosities
// eps_k, the limiter's active set (which elements are limited and the node
// of their minimum; theta itself is differentiated), the nodes cut by h_tol
// and the step size. At dry nodes (h <= 0) the velocity u = hu/h and the
// celerity c = sqrt(g max(h, 0)) are constant (zero derivative).
//
// Reverse order of one right-hand side (each step's input cotangents come
// from the previous one):
//   volume adjoint     R^ -> node cotangents of (h, hu, hv, u, v), the
//                      interface-flux and viscous-flux cotangents per side
//                      slot, the contravariant viscous-flux cotangents, the
//                      source-coefficient cotangents;
//   viscous face       viscous interface average -> side-node viscous fluxes;
//   viscosity (BR1)    viscous fluxes -> h, u, v and the BR1 interface values;
//   interface flux     per face node -> both sides' (h, u, v, b);
//   gather             slots -> nodes, u = hu/h -> (h, hu, hv), source
//                      coefficients -> b; accumulated into the caller's
//                      cotangents.
// Every cotangent is written by exactly one thread (no atomics), so the
// results are deterministic.
#include <math.h>

#include "kcommon.cuh"

namespace swe {
namespace {

constexpr int F_H = 0, F_HU = 1, F_HV = 2, F_U = 3, F_V = 4, F_A1 = 5, F_A2 = 6, F_A3 = 7;
constexpr int F_GH = 8, F_GHU = 9, F_GHV = 10, F_GU = 11, F_GV = 12, F_ADJ = 13;

template <int N>
constexpr int adj_ne() {
    return (128 / (N + 1)) > 0 ? 128 / (N + 1) : 1;
}

template <int N>
constexpr size_t adj_vol_smem() {
    return sizeof(double) * ((size_t)F_ADJ * adj_ne<N>() * (N + 1) * (N + 1) + (N + 1) * (N + 1));
}

template <int N>
__host__ __device__ constexpr int pair_index_adj(int i, int q) {
    return i * (N + 1) - i * (i + 1) / 2 + (q - i - 1);
}

// Pair loop of one line in reverse: for every pair (i, q), i < q, with
// d = A^(i) - A^(q) (the forward adds to node i and subtracts from node q):
//   Q^ = 2 d1 + (u_i + u_q) d2 + (v_i + v_q) d3,  P^ = 2g (S_x d2 + S_y d3),
//   u^_{i,q} += Q d2, v^_{i,q} += Q d3, hu^_{i,q} += S_x Q^, hv^_{i,q} += S_y Q^,
//   h^_i += h_q P^, h^_q += h_i P^.
// Q^ is formed from the per-node theta = 2 A^1 + u A^2 + v A^3 (staged in
// place of A^1): Q^ = theta_i - theta_q + u_q A^2_i - u_i A^2_q
// + v_q A^3_i - v_i A^3_q, which needs neither d1 nor the velocity sums.
// The factor 2g of P^ is applied once per node after both lines (gH holds
// h^ / 2g), and every cotangent sum is a fused multiply-add: 23 FP64
// instructions per pair.
template <int N, int BLK>
__device__ __forceinline__ void pair_loop_adj(const double* __restrict__ s, int base, int stride,
                                              const double* __restrict__ pmk, double* gH, double* gHU,
                                              double* gHV, double* gU, double* gV) {
    constexpr int n = N + 1;
    const double* sH = s + F_H * BLK;
    const double* sHU = s + F_HU * BLK;
    const double* sHV = s + F_HV * BLK;
    const double* sU = s + F_U * BLK;
    const double* sV = s + F_V * BLK;
    const double* sA1 = s + F_A1 * BLK;
    const double* sA2 = s + F_A2 * BLK;
    const double* sA3 = s + F_A3 * BLK;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int ni = base + i * stride;
        const double h_i = sH[ni], hu_i = sHU[ni], hv_i = sHV[ni], u_i = sU[ni], v_i = sV[ni];
        const double th_i = sA1[ni], a2 = sA2[ni], a3 = sA3[ni];
#pragma unroll
        for (int q = i + 1; q < n; ++q) {
            const int nq = base + q * stride;
            const int pr = pair_index_adj<N>(i, q);
            const double2 c = __ldg(reinterpret_cast<const double2*>(pmk + 2 * pr * n));
            const double sx = c.x, sy = c.y;
            const double a2q = sA2[nq], a3q = sA3[nq];
            const double d2 = a2 - a2q, d3 = a3 - a3q;
            const double Q = fma(hu_i + sHU[nq], sx, (hv_i + sHV[nq]) * sy);
            const double Qb =
                fma(-v_i, a3q, fma(sV[nq], a3, fma(-u_i, a2q, fma(sU[nq], a2, th_i - sA1[nq]))));
            const double Pb = fma(sy, d3, sx * d2);
            gU[i] = fma(Q, d2, gU[i]);
            gU[q] = fma(Q, d2, gU[q]);
            gV[i] = fma(Q, d3, gV[i]);
            gV[q] = fma(Q, d3, gV[q]);
            gHU[i] = fma(sx, Qb, gHU[i]);
            gHU[q] = fma(sx, Qb, gHU[q]);
            gHV[i] = fma(sy, Qb, gHV[i]);
            gHV[q] = fma(sy, Qb, gHV[q]);
            gH[i] = fma(sH[nq], Pb, gH[i]);
            gH[q] = fma(h_i, Pb, gH[q]);
        }
    }
}

struct VolAdjArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Rb;    // [3][KN] cotangent of R
    const double* eps;
    double* Ga;          // [3][KN] out: cotangents of (h, hu, hv), direct paths
    double* Guv;         // [2][KN] out: cotangents of (u, v)
    double* Gfo;         // [3][KS] out: cotangents of the outward interface flux
    double* Gsrc;        // [2][KN] out: cotangents of the source coefficients
    double* Gfvt;        // [4][KN] out (AV): cotangents of the contravariant viscous fluxes
    double* Gfvo;        // [2][KS] out (AV): cotangents of the viscous interface flux
    int acc_src;         // add to Gsrc (a sum over stages) instead of overwriting it
};

template <int N, bool AV>
__global__ void __launch_bounds__(adj_ne<N>() * (N + 1)) k_volume_adj(VolAdjArgs a) {
    constexpr int n = N + 1, nn = n * n, NE = adj_ne<N>(), NT = NE * n, BLK = NE * nn;
    constexpr int NP = N * (N + 1) / 2;
    extern __shared__ double sm[];
    const DeviceMesh& m = a.m;
    const int t = threadIdx.x;
    const long long k0 = (long long)blockIdx.x * NE;
    auto S = [&](int f) { return sm + f * BLK; };
    double* sD = sm + F_ADJ * BLK;
    for (int idx = t; idx < nn; idx += NT) sD[idx] = Dm<N>(idx / n, idx % n);

    // ---- stage: state, velocities and A^ = -R^/(w_i w_j J) -----------------
    for (int idx = t; idx < BLK; idx += NT) {
        const int e = idx / nn;
        const long long k = k0 + e;
        double h = 0, hu = 0, hv = 0, u = 0, v = 0, b1 = 0, b2 = 0, b3 = 0;
        if (k < m.K) {
            const long long gid = k * nn + (idx - e * nn);
            h = a.W[gid];
            hu = a.W[m.KN + gid];
            hv = a.W[2 * m.KN + gid];
            u = a.uv[gid];
            v = a.uv[m.KN + gid];
            const double f = m.fwJ[gid];
            b1 = f * a.Rb[gid];
            b2 = f * a.Rb[m.KN + gid];
            b3 = f * a.Rb[2 * m.KN + gid];
        }
        S(F_H)[idx] = h;
        S(F_HU)[idx] = hu;
        S(F_HV)[idx] = hv;
        S(F_U)[idx] = u;
        S(F_V)[idx] = v;
        S(F_A1)[idx] = fma(v, b3, fma(u, b2, 2.0 * b1));  // theta
        S(F_A2)[idx] = b2;
        S(F_A3)[idx] = b3;
    }
    __syncthreads();

    const int e = t / n, l = t - e * n;
    const long long k = k0 + e;
    const bool valid = k < m.K;
    const double* pmx = m.pm + ((size_t)(valid ? k : 0) * 2 * NP * n + l) * 2;
    const double* pme = pmx + (size_t)NP * n * 2;
    const double g2 = 2.0 * m.g;
    double gH[n], gHU[n], gHV[n], gU[n], gV[n];
#pragma unroll
    for (int p = 0; p < n; ++p) gH[p] = gHU[p] = gHV[p] = gU[p] = gV[p] = 0.0;

    // ---- xi-line j = l ------------------------------------------------------
    if (valid) pair_loop_adj<N, BLK>(sm, e * nn + l * n, 1, pmx, gH, gHU, gHV, gU, gV);
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const int id = e * nn + l * n + p;
        S(F_GH)[id] = gH[p];
        S(F_GHU)[id] = gHU[p];
        S(F_GHV)[id] = gHV[p];
        S(F_GU)[id] = gU[p];
        S(F_GV)[id] = gV[p];
    }
    __syncthreads();
    // ---- eta-line i = l, continuing the node sums ----------------------------
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const int id = e * nn + p * n + l;
        gH[p] = S(F_GH)[id];
        gHU[p] = S(F_GHU)[id];
        gHV[p] = S(F_GHV)[id];
        gU[p] = S(F_GU)[id];
        gV[p] = S(F_GV)[id];
    }
    if (valid) pair_loop_adj<N, BLK>(sm, e * nn + l, n, pme, gH, gHU, gHV, gU, gV);
    if (!valid) return;

    const long long KN = m.KN, KS = m.KS, side = k * 4 * n;
    const double ek = AV ? a.eps[k] : 0.0;
    const bool visc = AV && ek > 0.0;
    const int eb = e * nn;
    // ---- nodes (i = l, j = p): source, interface lifts, outputs -------------
    const int i = l;
    const double wi = wq<N>(i);
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const int j = p;
        const long long gid = k * nn + j * n + i;
        const double rb2 = a.Rb[KN + gid], rb3 = a.Rb[2 * KN + gid];
        const double h = S(F_H)[eb + j * n + i];
        // R2 = h srcx + f a2, R3 = h srcy + f a3
        a.Ga[gid] = fma(g2, gH[p], fma(rb2, m.srcx[gid], rb3 * m.srcy[gid]));
        a.Ga[KN + gid] = gHU[p];
        a.Ga[2 * KN + gid] = gHV[p];
        a.Guv[gid] = gU[p];
        a.Guv[KN + gid] = gV[p];
        if (a.acc_src) {
            a.Gsrc[gid] = fma(h, rb2, a.Gsrc[gid]);
            a.Gsrc[KN + gid] = fma(h, rb3, a.Gsrc[KN + gid]);
        } else {
            a.Gsrc[gid] = h * rb2;
            a.Gsrc[KN + gid] = h * rb3;
        }
        const double b2 = S(F_A2)[eb + j * n + i], b3 = S(F_A3)[eb + j * n + i];
        // a_c += wt F_out,c  =>  F_out^ = wt a^_c;  a_c -= wt (Fv_out - own)  =>  Fv_out^ = -wt a^_c
        // (every element takes the viscous interface flux, viscous or not)
        auto lift = [&](int f, int pn, double wt) {
            const long long sl = side + f * n + pn;
            a.Gfo[sl] = wt * (m.fwJ[gid] * a.Rb[gid]);  // A^1 (the plane holds theta)
            a.Gfo[KS + sl] = wt * b2;
            a.Gfo[2 * KS + sl] = wt * b3;
            if (AV) {
                a.Gfvo[sl] = -wt * b2;
                a.Gfvo[KS + sl] = -wt * b3;
            }
        };
        if (j == 0) lift(0, i, wi);
        if (j == N) lift(2, i, wi);
    }
    // the xi-side slots (sides 1 and 3) of row j = l: every lane takes the
    // two end nodes of its row, rather than two lanes of eight in the loop
    {
        const double wl = wq<N>(l);
#pragma unroll
        for (int end = 0; end < 2; ++end) {
            const int pi = end == 0 ? N : 0, f = end == 0 ? 1 : 3;
            const int nd = eb + l * n + pi;
            const long long gnd = k * nn + l * n + pi;
            const double b1 = m.fwJ[gnd] * a.Rb[gnd], b2 = S(F_A2)[nd], b3 = S(F_A3)[nd];
            const long long sl = side + f * n + l;
            a.Gfo[sl] = wl * b1;
            a.Gfo[KS + sl] = wl * b2;
            a.Gfo[2 * KS + sl] = wl * b3;
            if (AV) {
                a.Gfvo[sl] = -wl * b2;
                a.Gfvo[KS + sl] = -wl * b3;
            }
        }
    }
    if (!visc) return;
    // ---- viscous divergence: a_c -= w_i w_j (sum_q D_iq Ft_c[j][q] + sum_q D_jq Gt_c[q][i])
    // and the own-flux part of the viscous lift. Thread l owns the xi-line j = l
    // for Ft^ and the eta-line i = l for Gt^.
    {
        const int jl = l;  // xi-line
        const double wjl = wq<N>(jl);
#pragma unroll
        for (int q = 0; q < n; ++q) {
            double f2 = 0.0, f3 = 0.0;
#pragma unroll
            for (int ii = 0; ii < n; ++ii) {
                const double c = -wq<N>(ii) * wjl * sD[ii * n + q];
                f2 = fma(c, S(F_A2)[eb + jl * n + ii], f2);
                f3 = fma(c, S(F_A3)[eb + jl * n + ii], f3);
            }
            // own outward viscous flux at the xi faces: +Ft on face 1, -Ft on face 3
            if (q == N) {
                f2 = fma(wjl, S(F_A2)[eb + jl * n + q], f2);
                f3 = fma(wjl, S(F_A3)[eb + jl * n + q], f3);
            }
            if (q == 0) {
                f2 = fma(-wjl, S(F_A2)[eb + jl * n + q], f2);
                f3 = fma(-wjl, S(F_A3)[eb + jl * n + q], f3);
            }
            const long long gid = k * nn + jl * n + q;
            a.Gfvt[gid] = f2;
            a.Gfvt[KN + gid] = f3;
        }
        const int il = l;  // eta-line
        const double wil = wq<N>(il);
#pragma unroll
        for (int q = 0; q < n; ++q) {
            double g2v = 0.0, g3v = 0.0;
#pragma unroll
            for (int jj = 0; jj < n; ++jj) {
                const double c = -wil * wq<N>(jj) * sD[jj * n + q];
                g2v = fma(c, S(F_A2)[eb + jj * n + il], g2v);
                g3v = fma(c, S(F_A3)[eb + jj * n + il], g3v);
            }
            // own outward viscous flux at the eta faces: +Gt on face 2, -Gt on face 0
            if (q == N) {
                g2v = fma(wil, S(F_A2)[eb + q * n + il], g2v);
                g3v = fma(wil, S(F_A3)[eb + q * n + il], g3v);
            }
            if (q == 0) {
                g2v = fma(-wil, S(F_A2)[eb + q * n + il], g2v);
                g3v = fma(-wil, S(F_A3)[eb + q * n + il], g3v);
            }
            const long long gid = k * nn + q * n + il;
            a.Gfvt[2 * KN + gid] = g2v;
            a.Gfvt[3 * KN + gid] = g3v;
        }
    }
}

// ---------------------------------------------------------------------------
// Viscous interface average {F^v . n}: both side slots' physical viscous
// fluxes receive half of the face's cotangent times the normal.
// ---------------------------------------------------------------------------
__global__ void k_visc_face_adj(DeviceMesh m, const double* __restrict__ Gfvo, double* __restrict__ Gfvtr) {
    const long long total = (long long)m.nfaces * m.n;
    const long long S = m.KS;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long tm = m.f_tm[t], tp = m.f_tp[t];
        const double nx = 4.0 * m.f_nx[t] * m.f_js8[t], ny = 4.0 * m.f_ny[t] * m.f_js8[t];
        const double a2 = Gfvo[tm] - Gfvo[tp], a3 = Gfvo[S + tm] - Gfvo[S + tp];
        const double f2 = nx * a2, g2 = ny * a2, f3 = nx * a3, g3 = ny * a3;
        Gfvtr[tm] = f2;
        Gfvtr[S + tm] = f3;
        Gfvtr[2 * S + tm] = g2;
        Gfvtr[3 * S + tm] = g3;
        Gfvtr[tp] = f2;
        Gfvtr[S + tp] = f3;
        Gfvtr[2 * S + tp] = g2;
        Gfvtr[3 * S + tp] = g3;
    }
}

// ---------------------------------------------------------------------------
// BR1 and the viscous fluxes in reverse, one warp per viscous element: the
// warps of a fixed grid stride over the list of viscous elements (built with
// the forward quantities). The BR1 interface-value cotangents of the other
// elements are zero (cleared before the launch), and a viscous element
// writes all of its side slots.
// ---------------------------------------------------------------------------
constexpr int AVA_WPB = 4;

struct AvAdjArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Ustar;
    const double* eps;
    const double* Gfvt;
    const double* Gfvtr;
    double* Ga;    // += h cotangent
    double* Guv;   // += (u, v) cotangents
    double* GUs;   // [2][KS] out: cotangents of the BR1 interface values
    const int* vlist;   // the viscous elements, vcount of them
    const int* vcount;
};

template <int N>
__global__ void __launch_bounds__(32 * AVA_WPB) k_av_adj(AvAdjArgs a) {
    constexpr int n = N + 1, nn = n * n, PER = (nn + 31) / 32;
    __shared__ double sD[nn];
    __shared__ double sG[AVA_WPB][4][nn];  // cotangents of u_xi, u_eta, v_xi, v_eta
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) sD[idx] = Dm<N>(idx / n, idx % n);
    __syncthreads();
    const DeviceMesh& m = a.m;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long KN = m.KN, KS = m.KS;
    constexpr double iw0 = N * (N + 1) / 2.0;
    const int count = *a.vcount;
    for (int li = blockIdx.x * AVA_WPB + w; li < count; li += gridDim.x * AVA_WPB) {
        const long long k = a.vlist[li];
        const double ep = a.eps[k];
        const long long base = k * nn, side = k * 4 * n;
        double ubar[PER], vbar[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            ubar[r] = vbar[r] = 0.0;
            if (node >= nn) continue;
            const int i = node % n, j = node / n;
            const long long gid = base + node;
            // forward gradient of u, v at the node
            double ux = 0.0, ue = 0.0, vx = 0.0, ve = 0.0;
#pragma unroll
            for (int q = 0; q < n; ++q) {
                const double di = sD[i * n + q], dj = sD[j * n + q];
                ux = fma(di, a.uv[base + j * n + q], ux);
                vx = fma(di, a.uv[KN + base + j * n + q], vx);
                ue = fma(dj, a.uv[base + q * n + i], ue);
                ve = fma(dj, a.uv[KN + base + q * n + i], ve);
            }
            const double u = a.uv[gid], v = a.uv[KN + gid];
            if (i == N) { const long long sl = side + 1 * n + j; ux += iw0 * (a.Ustar[sl] - u); vx += iw0 * (a.Ustar[KS + sl] - v); }
            if (i == 0) { const long long sl = side + 3 * n + j; ux -= iw0 * (a.Ustar[sl] - u); vx -= iw0 * (a.Ustar[KS + sl] - v); }
            if (j == N) { const long long sl = side + 2 * n + i; ue += iw0 * (a.Ustar[sl] - u); ve += iw0 * (a.Ustar[KS + sl] - v); }
            if (j == 0) { const long long sl = side + 0 * n + i; ue -= iw0 * (a.Ustar[sl] - u); ve -= iw0 * (a.Ustar[KS + sl] - v); }
            const double axx = m.axx[gid], axy = m.axy[gid], aex = m.aex[gid], aey = m.aey[gid];
            // cotangents of the physical viscous fluxes (F2, G2, F3, G3)
            const double ft2 = a.Gfvt[gid], ft3 = a.Gfvt[KN + gid], gt2 = a.Gfvt[2 * KN + gid],
                         gt3 = a.Gfvt[3 * KN + gid];
            double F2 = fma(axx, ft2, aex * gt2), G2 = fma(axy, ft2, aey * gt2);
            double F3 = fma(axx, ft3, aex * gt3), G3 = fma(axy, ft3, aey * gt3);
            auto take = [&](int f, int p) {
                const long long sl = side + f * n + p;
                F2 += a.Gfvtr[sl];
                F3 += a.Gfvtr[KS + sl];
                G2 += a.Gfvtr[2 * KS + sl];
                G3 += a.Gfvtr[3 * KS + sl];
            };
            if (j == 0) take(0, i);
            if (i == N) take(1, j);
            if (j == N) take(2, i);
            if (i == 0) take(3, j);
            const double rJ = m.rJ[gid];
            const double h = a.W[gid];
            const double he = h * ep * rJ;
            // F2 = he (axx ux + aex ue), G2 = he (axy ux + aey ue), same with v for F3, G3
            const double heb = F2 * fma(axx, ux, aex * ue) + G2 * fma(axy, ux, aey * ue) +
                               F3 * fma(axx, vx, aex * ve) + G3 * fma(axy, vx, aey * ve);
            a.Ga[gid] = fma(ep * rJ, heb, a.Ga[gid]);
            double uxb = he * fma(axx, F2, axy * G2), ueb = he * fma(aex, F2, aey * G2);
            double vxb = he * fma(axx, F3, axy * G3), veb = he * fma(aex, F3, aey * G3);
            sG[w][0][node] = uxb;
            sG[w][1][node] = ueb;
            sG[w][2][node] = vxb;
            sG[w][3][node] = veb;
            // the lifts (+-iw0 (U* - u))
            auto put = [&](int f, int p, double cu, double cv) {
                const long long sl = side + f * n + p;
                a.GUs[sl] = cu;
                a.GUs[KS + sl] = cv;
            };
            if (i == N) { put(1, j, iw0 * uxb, iw0 * vxb); ubar[r] -= iw0 * uxb; vbar[r] -= iw0 * vxb; }
            if (i == 0) { put(3, j, -iw0 * uxb, -iw0 * vxb); ubar[r] += iw0 * uxb; vbar[r] += iw0 * vxb; }
            if (j == N) { put(2, i, iw0 * ueb, iw0 * veb); ubar[r] -= iw0 * ueb; vbar[r] -= iw0 * veb; }
            if (j == 0) { put(0, i, -iw0 * ueb, -iw0 * veb); ubar[r] += iw0 * ueb; vbar[r] += iw0 * veb; }
        }
        __syncwarp();
        // u^(a, b) += sum_i D_{i a} ux^(i, b) + sum_j D_{j b} ue^(a, j)
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            if (node >= nn) continue;
            const int i = node % n, j = node / n;
            double su = ubar[r], sv = vbar[r];
#pragma unroll
            for (int q = 0; q < n; ++q) {
                const double di = sD[q * n + i], dj = sD[q * n + j];
                su = fma(di, sG[w][0][j * n + q], su);
                sv = fma(di, sG[w][2][j * n + q], sv);
                su = fma(dj, sG[w][1][q * n + i], su);
                sv = fma(dj, sG[w][3][q * n + i], sv);
            }
            const long long gid = base + node;
            a.Guv[gid] += su;
            a.Guv[KN + gid] += sv;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Interface flux in reverse. normal_flux_adj differentiates the flux of the
// forward kernel in the normal frame (same expression, same branches).
// ---------------------------------------------------------------------------
// sgn(x) y (zero for x = 0) by the sign bits: integer operations only.
__device__ __forceinline__ double sgn_times(double x, double y) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    if ((bx << 1) == 0ULL) return 0.0;
    return __longlong_as_double(__double_as_longlong(y) ^ (long long)(bx & 0x8000000000000000ULL));
}

template <bool ES>
__device__ __forceinline__ void normal_flux_adj(double g, double r2g, double hm, double hp, double utm, double utp,
                                                double vtm, double vtp, double bm, double bp, double F1b, double F2b,
                                                double F3b, double& hmb, double& hpb, double& utmb, double& utpb,
                                                double& vtmb, double& vtpb, double& bmb, double& bpb) {
    const double ha = 0.5 * (hm + hp), ua = 0.5 * (utm + utp), va = 0.5 * (vtm + vtp);
    double hab = 0.0, uab = 0.0, vab = 0.0, h2ab = 0.0;
    hmb = hpb = utmb = utpb = vtmb = vtpb = bmb = bpb = 0.0;
    if (ES) {
        const double cm = sqrt_pos(g * pos_part(hm)), cp = sqrt_pos(g * pos_part(hp));
        const double ca = 0.5 * (cm + cp);
        const double gH = g * ((hp + bp) - (hm + bm));
        const double dut = utp - utm, dvt = vtp - vtm;
        const double A1 = fabs(ua + ca) * r2g, B1 = fma(ca, dut, gH);
        const double A3 = fabs(ua - ca) * r2g, B3 = fma(-ca, dut, gH);
        const double s1 = A1 * B1, s3 = A3 * B3, d1 = s1 + s3;
        const double lam2 = fabs(ha * ua);
        // F1 -= d1/2;  F2 -= (ua d1 + ca (s1 - s3))/2;  F3 -= (va d1 + lam2 dvt)/2
        const double d1b = -0.5 * fma(va, F3b, fma(ua, F2b, F1b));
        uab -= 0.5 * d1 * F2b;
        double cab = -0.5 * (s1 - s3) * F2b;
        const double s1b = fma(-0.5 * ca, F2b, d1b), s3b = fma(0.5 * ca, F2b, d1b);
        vab -= 0.5 * d1 * F3b;
        const double lam2b = -0.5 * dvt * F3b;
        const double dvtb = -0.5 * lam2 * F3b;
        const double A1b = s1b * B1, B1b = s1b * A1, A3b = s3b * B3, B3b = s3b * A3;
        const double sp = sgn_times(ua + ca, r2g * A1b), sm = sgn_times(ua - ca, r2g * A3b);
        uab += sp + sm;
        cab += sp - sm;
        cab += (B1b - B3b) * dut;
        const double dutb = ca * (B1b - B3b);
        const double gHb = g * (B1b + B3b);
        const double sl = sgn_times(ha * ua, lam2b);
        hab += sl * ua;
        uab += sl * ha;
        hpb += gHb;
        bpb += gHb;
        hmb -= gHb;
        bmb -= gHb;
        utpb += dutb;
        utmb -= dutb;
        vtpb += dvtb;
        vtmb -= dvtb;
        // c = sqrt(g h): dc/dh = g/(2c) for h > 0
        const double qg = 0.25 * g * cab;
        if (hm > 0.0) hmb += qg * recip_pos(cm);
        if (hp > 0.0) hpb += qg * recip_pos(cp);
    }
    // EC part: F1 = ha ua, F2 = F1 ua + g h2a / 2, F3 = F1 va
    const double F1 = ha * ua;
    const double F1t = fma(va, F3b, fma(ua, F2b, F1b));
    uab = fma(F1, F2b, uab);
    vab = fma(F1, F3b, vab);
    h2ab += 0.5 * g * F2b;
    hab = fma(ua, F1t, hab);
    uab = fma(ha, F1t, uab);
    hmb += 0.5 * hab + hm * h2ab;
    hpb += 0.5 * hab + hp * h2ab;
    utmb += 0.5 * uab;
    utpb += 0.5 * uab;
    vtmb += 0.5 * vab;
    vtpb += 0.5 * vab;
}

// Slot cotangents: [4][KS] (h, u, v, b) of the node behind each side slot.
template <bool ES>
__global__ void k_surface_adj(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv,
                              const double* __restrict__ Gfo, const double* __restrict__ GUs, int av,
                              double* __restrict__ Gsl) {
    const long long total = (long long)m.nfaces * m.n;
    const long long S = m.KS;
    const double g = m.g;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long im = m.f_im[t], ip = m.f_ip[t], tm = m.f_tm[t], tp = m.f_tp[t];
        const double nx = m.f_nx[t], ny = m.f_ny[t], js = 8.0 * m.f_js8[t];
        const double hm = W[im], hp = W[ip];
        const double um = uv[im], vm = uv[m.KN + im], up = uv[ip], vp = uv[m.KN + ip];
        const double utm = fma(nx, um, ny * vm), vtm = fma(nx, vm, -ny * um);
        const double utp = fma(nx, up, ny * vp), vtp = fma(nx, vp, -ny * up);
        // Fout[tm] = G, Fout[tp] = -G; G = js (F1, nx F2 - ny F3, ny F2 + nx F3)
        const double G1b = Gfo[tm] - Gfo[tp], G2b = Gfo[S + tm] - Gfo[S + tp], G3b = Gfo[2 * S + tm] - Gfo[2 * S + tp];
        const double F1b = js * G1b, F2b = js * fma(nx, G2b, ny * G3b), F3b = js * fma(-ny, G2b, nx * G3b);
        double hmb, hpb, utmb, utpb, vtmb, vtpb, bmb, bpb;
        normal_flux_adj<ES>(g, m.r2g, hm, hp, utm, utp, vtm, vtp, m.f_bm[t], m.f_bp[t], F1b, F2b, F3b, hmb, hpb, utmb,
                            utpb, vtmb, vtpb, bmb, bpb);
        // rotation: ut = nx u + ny v, vt = nx v - ny u
        double umb = fma(nx, utmb, -ny * vtmb), vmb = fma(ny, utmb, nx * vtmb);
        double upb = fma(nx, utpb, -ny * vtpb), vpb = fma(ny, utpb, nx * vtpb);
        if (av) {
            // U* = ({u}, {v}) on both slots
            const double us = 0.5 * (GUs[tm] + GUs[tp]), vs = 0.5 * (GUs[S + tm] + GUs[S + tp]);
            umb += us;
            upb += us;
            vmb += vs;
            vpb += vs;
        }
        Gsl[tm] = hmb;
        Gsl[S + tm] = umb;
        Gsl[2 * S + tm] = vmb;
        Gsl[3 * S + tm] = bmb;
        Gsl[tp] = hpb;
        Gsl[S + tp] = upb;
        Gsl[2 * S + tp] = vpb;
        Gsl[3 * S + tp] = bpb;
    }
}

template <bool ES>
__global__ void k_wall_adj(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv,
                           const double* __restrict__ Gfo, const double* __restrict__ GUs, int av,
                           double* __restrict__ Gsl) {
    const long long total = (long long)m.nwall * m.n;
    const long long S = m.KS;
    const double g = m.g;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long im = m.w_im[t], tm = m.w_tm[t];
        const double nx = m.w_nx[t], ny = m.w_ny[t], js = m.w_js[t];
        const double hm = W[im], um = uv[im], vm = uv[m.KN + im], bm = m.bn[im];
        const double utm = fma(nx, um, ny * vm), vtm = fma(nx, vm, -ny * um);
        const double G1b = Gfo[tm], G2b = Gfo[S + tm], G3b = Gfo[2 * S + tm];
        const double F1b = js * G1b, F2b = js * fma(nx, G2b, ny * G3b), F3b = js * fma(-ny, G2b, nx * G3b);
        double hmb, hpb, utmb, utpb, vtmb, vtpb, bmb, bpb;
        normal_flux_adj<ES>(g, m.r2g, hm, hm, utm, -utm, vtm, vtm, bm, bm, F1b, F2b, F3b, hmb, hpb, utmb, utpb, vtmb,
                            vtpb, bmb, bpb);
        // mirror: hp = hm, utp = -utm, vtp = vtm, bp = bm
        const double hb = hmb + hpb, utb = utmb - utpb, vtb = vtmb + vtpb;
        double umb = fma(nx, utb, -ny * vtb), vmb = fma(ny, utb, nx * vtb);
        if (av) {
            umb += GUs[tm];  // U* = own u at a wall
            vmb += GUs[S + tm];
        }
        Gsl[tm] = hb;
        Gsl[S + tm] = umb;
        Gsl[2 * S + tm] = vmb;
        Gsl[3 * S + tm] = bmb + bpb;
    }
}

// ---------------------------------------------------------------------------
// Gather: slot cotangents onto nodes and u = hu/h in reverse; the slot
// cotangents of b (the interface fluxes' bathymetry jumps) go to bbar.
// One thread per node (a streaming kernel: full occupancy hides the
// latency of its dozen independent loads); accumulates into the caller's
// Wbar, bbar. The source coefficients' part of bbar is k_src_adj's.
// ---------------------------------------------------------------------------
constexpr int GA_TPB = 256;

struct GatherArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Ga;
    const double* Guv;
    const double* Gsl;
    double* Wbar;
    double* bbar;  // nullable
};

template <int N>
__global__ void __launch_bounds__(GA_TPB) k_gather_adj(GatherArgs a) {
    constexpr int n = N + 1, nn = n * n;
    const DeviceMesh& m = a.m;
    const long long KN = m.KN, KS = m.KS;
    const long long gid = (long long)blockIdx.x * GA_TPB + threadIdx.x;
    if (gid >= KN) return;
    const long long k = gid / nn;
    const int node = (int)(gid - k * nn), i = node % n, j = node / n;
    const long long side = k * 4 * n;
    double gh = a.Ga[gid], gu = a.Guv[gid], gv = a.Guv[KN + gid], gb = 0.0;
    auto take = [&](int f, int p) {
        const long long sl = side + f * n + p;
        gh += a.Gsl[sl];
        gu += a.Gsl[KS + sl];
        gv += a.Gsl[2 * KS + sl];
        gb += a.Gsl[3 * KS + sl];
    };
    const bool edge = j == 0 || i == N || j == N || i == 0;
    if (j == 0) take(0, i);
    if (i == N) take(1, j);
    if (j == N) take(2, i);
    if (i == 0) take(3, j);
    double ghu = a.Ga[KN + gid], ghv = a.Ga[2 * KN + gid];
    const double h = a.W[gid];
    if (h > 0.0) {
        const double rh = recip_pos(h);
        gh -= (a.uv[gid] * gu + a.uv[KN + gid] * gv) * rh;
        ghu = fma(gu, rh, ghu);
        ghv = fma(gv, rh, ghv);
    }
    a.Wbar[gid] += gh;
    a.Wbar[KN + gid] += ghu;
    a.Wbar[2 * KN + gid] += ghv;
    if (a.bbar && edge) a.bbar[gid] += gb;
}

// ---------------------------------------------------------------------------
// Source coefficients in reverse: bbar += (d src / d b)^T Gsrc, for one
// stage's cotangents or their sum over stages (the map is linear and depends
// on the geometry only). src_c = -(g/2) gamma_c / J (Eq. SourceDisc) with
//   gamma_x(i,j) = sum_q D_iq (axx_ij + axx_qj) b_qj + sum_q D_jq (aex_ij + aex_iq) b_iq
// and gamma_y likewise with axy, aey. For i < q on a line the entry
// D_iq (a_i + a_q) is 4/(w_i w_j) times the volume kernel's pair constant S
// of the pair, and the reversed entry D_qi (a_q + a_i) is -4/(w_q w_j) S
// (SBP: w_q D_qi = -w_i D_iq off the diagonal). With c = g fwJ2 Gsrc
// (= 4/(w_i w_j) times -(g/2) Gsrc / J) at every node, a pair costs four
// fused multiply-adds,
//   bbar_q += S_x c_x,i + S_y c_y,i,   bbar_i -= S_x c_x,q + S_y c_y,q,
// and the diagonal 2 D_ii a_i, nonzero at the two end nodes of a line only
// (LGL), adds D_ii (w_i w_j / 2) (a_x c_x + a_y c_y) there. One thread per
// line as in the volume kernels: the xi-line j = l, then the eta-line i = l
// continuing the node sums in shared memory.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void src_pairs_adj(const double* __restrict__ pmk, const double* cxl, const double* cyl,
                                              double* acc) {
    constexpr int n = N + 1;
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int q = i + 1; q < n; ++q) {
            const double2 c = __ldg(reinterpret_cast<const double2*>(pmk + 2 * pair_index_adj<N>(i, q) * n));
            acc[q] = fma(c.y, cyl[i], fma(c.x, cxl[i], acc[q]));
            acc[i] = fma(-c.y, cyl[q], fma(-c.x, cxl[q], acc[i]));
        }
}

template <int N>
__global__ void __launch_bounds__(adj_ne<N>() * (N + 1)) k_src_adj(DeviceMesh m, const double* __restrict__ Gsrc,
                                                                  double* __restrict__ bbar) {
    constexpr int n = N + 1, nn = n * n, NE = adj_ne<N>(), NT = NE * n, BLK = NE * nn;
    constexpr int NP = N * (N + 1) / 2;
    __shared__ double sc[2][BLK];
    __shared__ double sacc[BLK];
    const int t = threadIdx.x;
    const long long k0 = (long long)blockIdx.x * NE;
    const long long KN = m.KN;
    for (int idx = t; idx < BLK; idx += NT) {
        const int e = idx / nn;
        const long long k = k0 + e;
        double cx = 0.0, cy = 0.0;
        if (k < m.K) {
            const long long gid = k * nn + (idx - e * nn);
            const double f = m.g * m.fwJ2[gid];
            cx = f * Gsrc[gid];
            cy = f * Gsrc[KN + gid];
        }
        sc[0][idx] = cx;
        sc[1][idx] = cy;
    }
    __syncthreads();
    const int e = t / n, l = t - e * n;
    const long long k = k0 + e;
    const bool valid = k < m.K;
    const double* pmx = m.pm + ((size_t)(valid ? k : 0) * 2 * NP * n + l) * 2;
    const double* pme = pmx + (size_t)NP * n * 2;
    const double half_wl = 0.5 * wq<N>(l);
    const double c0 = Dm<N>(0, 0) * wq<N>(0) * half_wl, cN = Dm<N>(N, N) * wq<N>(N) * half_wl;
    const int eb = e * nn;
    double acc[n], cxl[n], cyl[n];
    // ---- xi-line j = l: nodes (p, l) ----------------------------------------
#pragma unroll
    for (int p = 0; p < n; ++p) {
        acc[p] = 0.0;
        cxl[p] = sc[0][eb + l * n + p];
        cyl[p] = sc[1][eb + l * n + p];
    }
    if (valid) {
        src_pairs_adj<N>(pmx, cxl, cyl, acc);
        const long long g0 = k * nn + l * n, gN = g0 + N;
        acc[0] = fma(c0, fma(m.axx[g0], cxl[0], m.axy[g0] * cyl[0]), acc[0]);
        acc[N] = fma(cN, fma(m.axx[gN], cxl[N], m.axy[gN] * cyl[N]), acc[N]);
    }
#pragma unroll
    for (int p = 0; p < n; ++p) sacc[eb + l * n + p] = acc[p];
    __syncthreads();
    if (!valid) return;
    // ---- eta-line i = l: nodes (l, p) ---------------------------------------
#pragma unroll
    for (int p = 0; p < n; ++p) {
        acc[p] = sacc[eb + p * n + l];
        cxl[p] = sc[0][eb + p * n + l];
        cyl[p] = sc[1][eb + p * n + l];
    }
    src_pairs_adj<N>(pme, cxl, cyl, acc);
    {
        const long long g0 = k * nn + l, gN = g0 + (long long)N * n;
        acc[0] = fma(c0, fma(m.aex[g0], cxl[0], m.aey[g0] * cyl[0]), acc[0]);
        acc[N] = fma(cN, fma(m.aex[gN], cxl[N], m.aey[gN] * cyl[N]), acc[N]);
    }
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const long long gid = k * nn + (long long)p * n + l;
        bbar[gid] += acc[p];
    }
}

// ---------------------------------------------------------------------------
// Stage update in reverse with the limiter's recorded plan.
//   Limiter (forward): Wl = theta (Y - mean) + mean on limited elements with
//   theta = m0/(m0 - Y0[amin]), then hu = hv = 0 on cut nodes.
//   MODE 1 (2N-storage, register K/dt): Y = W_in + (b dt) Kh, Kh = a Kh_prev + R.
//     Yb = limiter^T Wb; Khb += (b dt) Yb; Rb = Khb; Khb_prev = a Khb; Wb <- Yb.
//   MODE 2 (SSP): Y = a Wn + b (W_in + dt R).
//     Yb = limiter^T Wb; Wnb += a Yb; Wb <- b Yb; Rb = (b dt) Yb.
// ---------------------------------------------------------------------------
struct UpdAdjArgs {
    DeviceMesh m;
    double* Wb;            // in: cotangent of the stage output; out: of the stage input (direct part)
    const double* Y;       // pre-limit stage result
    const uint8_t* act;    // [K] limited element
    const int32_t* amin;   // [K] node of the minimum h
    const uint8_t* cut;    // [KN] h_tol cut
    double* Khb;           // MODE 1: register cotangent (in/out)
    double* Rb;            // out: cotangent of the stage's right-hand side
    double* Wnb;           // MODE 2: += cotangent of the step's start state
    double a, b, dt;
    int limiter;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int N, int MODE>
__global__ void __launch_bounds__(128) k_update_adj(UpdAdjArgs a) {
    constexpr int n = N + 1, nn = n * n, PER = (nn + 31) / 32;
    const DeviceMesh& m = a.m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long KN = m.KN;
    for (long long k = (long long)blockIdx.x * 4 + wid; k < m.K; k += (long long)gridDim.x * 4) {
        double yb[3][PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            yb[0][r] = yb[1][r] = yb[2][r] = 0.0;
            if (node >= nn) continue;
            const long long gid = k * nn + node;
            yb[0][r] = a.Wb[gid];
            yb[1][r] = a.Wb[KN + gid];
            yb[2][r] = a.Wb[2 * KN + gid];
            if (a.limiter && a.cut[gid]) yb[1][r] = yb[2][r] = 0.0;
        }
        if (a.limiter && a.act[k]) {
            // theta and the means of the pre-limit state
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int node = lane + 32 * r;
                if (node < nn) {
                    const long long gid = k * nn + node;
                    const double wj = m.wJ[gid];
                    s0 = fma(wj, a.Y[gid], s0);
                    s1 = fma(wj, a.Y[KN + gid], s1);
                    s2 = fma(wj, a.Y[2 * KN + gid], s2);
                }
            }
            const double rv = m.rvol[k];
            const double m0 = wsum(s0) * rv, m1 = wsum(s1) * rv, m2 = wsum(s2) * rv;
            const long long gmin = k * nn + a.amin[k];
            const double y = a.Y[gmin];
            const double den = m0 - y;
            const double theta = fmin(1.0, m0 / den);
            // sums of the output cotangents and theta's cotangent
            double S0 = 0.0, S1 = 0.0, S2 = 0.0, T = 0.0;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int node = lane + 32 * r;
                if (node < nn) {
                    const long long gid = k * nn + node;
                    S0 += yb[0][r];
                    S1 += yb[1][r];
                    S2 += yb[2][r];
                    T = fma(yb[0][r], a.Y[gid] - m0, T);
                    T = fma(yb[1][r], a.Y[KN + gid] - m1, T);
                    T = fma(yb[2][r], a.Y[2 * KN + gid] - m2, T);
                }
            }
            S0 = wsum(S0);
            S1 = wsum(S1);
            S2 = wsum(S2);
            T = wsum(T);
            const bool clamped = !(m0 / den < 1.0);
            const double dm0 = clamped ? 0.0 : -y / (den * den) * T;  // d theta / d m0
            const double dy = clamped ? 0.0 : m0 / (den * den) * T;   // d theta / d Y0[amin]
            const double om = 1.0 - theta;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int node = lane + 32 * r;
                if (node < nn) {
                    const long long gid = k * nn + node;
                    const double c = m.wJ[gid] * rv;
                    yb[0][r] = fma(theta, yb[0][r], c * fma(om, S0, dm0));
                    yb[1][r] = fma(theta, yb[1][r], c * om * S1);
                    yb[2][r] = fma(theta, yb[2][r], c * om * S2);
                    if (gid == gmin) yb[0][r] += dy;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            if (node >= nn) continue;
            const long long gid = k * nn + node;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long id = c * KN + gid;
                if (MODE == 1) {
                    const double kb = fma(a.b * a.dt, yb[c][r], a.Khb[id]);
                    a.Rb[id] = kb;
                    a.Khb[id] = a.a * kb;
                    a.Wb[id] = yb[c][r];
                } else {
                    a.Wnb[id] = fma(a.a, yb[c][r], a.Wnb[id]);
                    a.Wb[id] = a.b * yb[c][r];
                    a.Rb[id] = (a.b * a.dt) * yb[c][r];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Limiter with a recorded plan (the forward of the adjoint's recomputation):
// the same arithmetic as the fused stage update's limiter, applied to a
// state already updated, plus the plan and the velocities of the result.
// ---------------------------------------------------------------------------
struct LimRecArgs {
    DeviceMesh m;
    double* W;
    double* uv;
    uint8_t* act;
    int32_t* amin;
    uint8_t* cut;
    double h_tol;
    int* status;
};

__device__ __forceinline__ bool is_neg(double x) {
    return (unsigned long long)__double_as_longlong(x) > 0x8000000000000000ULL;
}

template <int N>
__global__ void __launch_bounds__(128) k_limit_rec(LimRecArgs a) {
    constexpr int n = N + 1, nn = n * n, PER = (nn + 31) / 32;
    const DeviceMesh& m = a.m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long KN = m.KN;
    for (long long k = (long long)blockIdx.x * 4 + wid; k < m.K; k += (long long)gridDim.x * 4) {
        double h[PER], hu[PER], hv[PER];
        bool neg = false;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            h[r] = hu[r] = hv[r] = 0.0;
            if (node < nn) {
                const long long gid = k * nn + node;
                h[r] = a.W[gid];
                hu[r] = a.W[KN + gid];
                hv[r] = a.W[2 * KN + gid];
                neg |= is_neg(h[r]);
            }
        }
        bool active = false;
        int arg = 0;
        if (__any_sync(0xffffffffu, neg)) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, mn = INFINITY;
            int an = nn;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int node = lane + 32 * r;
                if (node < nn) {
                    const double wj = m.wJ[k * nn + node];
                    s0 = fma(wj, h[r], s0);
                    s1 = fma(wj, hu[r], s1);
                    s2 = fma(wj, hv[r], s2);
                    if (h[r] < mn) { mn = h[r]; an = node; }
                }
            }
            const double rv = m.rvol[k];
            const double m0 = wsum(s0) * rv, m1 = wsum(s1) * rv, m2 = wsum(s2) * rv;
            // minimum and its first node
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double om = __shfl_xor_sync(0xffffffffu, mn, o);
                const int oa = __shfl_xor_sync(0xffffffffu, an, o);
                if (om < mn || (om == mn && oa < an)) { mn = om; an = oa; }
            }
            if (m0 < 0.0) {
                if (lane == 0) atomicOr(a.status, 1);
            } else if (m0 - mn > 0.0) {
                const double theta = fmin(1.0, m0 / (m0 - mn));
                active = true;
                arg = an;
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    h[r] = fma(theta, h[r] - m0, m0);
                    hu[r] = fma(theta, hu[r] - m1, m1);
                    hv[r] = fma(theta, hv[r] - m2, m2);
                }
            }
        }
        if (lane == 0) {
            a.act[k] = active ? 1 : 0;
            a.amin[k] = arg;
        }
        const long long tb = __double_as_longlong(a.h_tol);
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int node = lane + 32 * r;
            if (node >= nn) continue;
            const long long gid = k * nn + node;
            const bool c = (long long)__double_as_longlong(h[r]) < tb;
            if (c) hu[r] = hv[r] = 0.0;
            a.cut[gid] = c ? 1 : 0;
            a.W[gid] = h[r];
            a.W[KN + gid] = hu[r];
            a.W[2 * KN + gid] = hv[r];
            double u, v;
            velocities(h[r], hu[r], hv[r], u, v);
            a.uv[gid] = u;
            a.uv[KN + gid] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Gauge misfit: loss += sum_g (sum_nodes w_g h - target_g)^2 and, when Wb is
// given, Wb_h += 2 (h_g - target_g) w_g. One block; gauges in order, so two
// gauges in one element accumulate deterministically.
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_gauge(DeviceMesh m, const double* __restrict__ W, int ng, const int32_t* __restrict__ elem,
                        const double* __restrict__ wts, const double* __restrict__ target, double* values,
                        double* loss, double* Wb) {
    constexpr int n = N + 1, nn = n * n;
    __shared__ double part[128];
    __shared__ double acc;
    if (threadIdx.x == 0) acc = 0.0;
    __syncthreads();
    for (int gi = 0; gi < ng; ++gi) {
        const long long base = (long long)elem[gi] * nn;
        double s = 0.0;
        for (int node = threadIdx.x; node < nn; node += blockDim.x) s = fma(wts[(long long)gi * nn + node], W[base + node], s);
        part[threadIdx.x] = s;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
            __syncthreads();
        }
        const double r = part[0] - (target ? target[gi] : 0.0);
        if (threadIdx.x == 0) {
            acc = fma(r, r, acc);
            if (values) values[gi] = part[0];
        }
        if (Wb)
            for (int node = threadIdx.x; node < nn; node += blockDim.x)
                Wb[base + node] = fma(2.0 * r, wts[(long long)gi * nn + node], Wb[base + node]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss += acc;
}

__global__ void k_axpy(long long count, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

#define SWE_SWITCH_N_ADJ(N, CALL)                                                     \
    switch (N) {                                                                      \
        case 1: CALL(1); break; case 2: CALL(2); break; case 3: CALL(3); break;      \
        case 4: CALL(4); break; case 5: CALL(5); break; case 6: CALL(6); break;      \
        case 7: CALL(7); break; case 8: CALL(8); break; case 9: CALL(9); break;      \
        case 10: CALL(10); break; case 11: CALL(11); break; case 12: CALL(12); break; \
        default: break;                                                               \
    }

template <int N, bool AV>
void vol_adj_n(swe_ctx* c, const VolAdjArgs& a, cudaStream_t s) {
    constexpr size_t smem = adj_vol_smem<N>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_volume_adj<N, AV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    Timed tm(c, KC_ADJ_VOL, s);
    k_volume_adj<N, AV><<<grid_for(c->m.K, adj_ne<N>()), adj_ne<N>() * (N + 1), smem, s>>>(a);
}

}  // namespace

void init_tables_adjoint() { upload_tables(); }

void launch_rhs_adjoint(swe_ctx* c, const double* W, const double* Rb, double* Wbar, double* bbar, cudaStream_t s,
                        bool defer_src) {
    AdjWork& A = c->adj;
    const DeviceMesh& m = c->m;
    const bool av = c->p.av != 0;
    defer_src = defer_src && bbar != nullptr;
    VolAdjArgs va{m, W, c->w.uv, Rb, c->w.eps, A.Ga, A.Guv, A.Gfo, defer_src ? A.Gsrc_acc : A.Gsrc, A.Gfvt, A.Gfvo,
                  defer_src ? 1 : 0};
#define SWE_VA(NN) \
    if (av) vol_adj_n<NN, true>(c, va, s); else vol_adj_n<NN, false>(c, va, s)
    SWE_SWITCH_N_ADJ(m.N, SWE_VA)
#undef SWE_VA
    // The source coefficients onto b read only the volume kernel's Gsrc: on
    // large meshes they run on the second stream beside the viscous and
    // interface-flux reverse kernels, and the gather (the other writer of
    // bbar) waits for them.
    const bool src_now = bbar && !defer_src;
    const bool src_side = src_now && c->side;
    if (src_side) {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(c->s_av, c->ev_fork, 0);
        launch_src_adjoint(c, A.Gsrc, bbar, c->s_av);
        cudaEventRecord(c->ev_join, c->s_av);
    }
    if (av) {
        const long long total = (long long)m.nfaces * m.n;
        if (total > 0) {
            Timed tm(c, KC_ADJ, s);
            k_visc_face_adj<<<grid_for(total, 128), 128, 0, s>>>(m, A.Gfvo, A.Gfvtr);
        }
        AvAdjArgs aa{m, W, c->w.uv, c->w.Ustar, c->w.eps, A.Gfvt, A.Gfvtr, A.Ga, A.Guv, A.GUs,
                     c->w.vlist, c->w.vcount};
        cudaMemsetAsync(A.GUs, 0, sizeof(double) * 2 * (size_t)m.KS, s);
        // a fixed grid striding over the list: sixteen blocks per SM at most
        const int ablocks = grid_for(m.K, AVA_WPB) < 16 * c->sms ? grid_for(m.K, AVA_WPB) : 16 * c->sms;
#define SWE_AA(NN)                                                                         \
    {                                                                                      \
        Timed tm(c, KC_ADJ, s);                                                            \
        k_av_adj<NN><<<ablocks, 32 * AVA_WPB, 0, s>>>(aa);                                 \
    }
        SWE_SWITCH_N_ADJ(m.N, SWE_AA)
#undef SWE_AA
    }
    {
        const long long total = (long long)m.nfaces * m.n;
        if (total > 0) {
            Timed tm(c, KC_ADJ, s);
            if (c->p.flux)
                k_surface_adj<true><<<grid_for(total, 128), 128, 0, s>>>(m, W, c->w.uv, A.Gfo, A.GUs, av, A.Gsl);
            else
                k_surface_adj<false><<<grid_for(total, 128), 128, 0, s>>>(m, W, c->w.uv, A.Gfo, A.GUs, av, A.Gsl);
        }
        const long long walls = (long long)m.nwall * m.n;
        if (walls > 0) {
            Timed tm(c, KC_ADJ, s);
            if (c->p.flux)
                k_wall_adj<true><<<grid_for(walls, 128), 128, 0, s>>>(m, W, c->w.uv, A.Gfo, A.GUs, av, A.Gsl);
            else
                k_wall_adj<false><<<grid_for(walls, 128), 128, 0, s>>>(m, W, c->w.uv, A.Gfo, A.GUs, av, A.Gsl);
        }
    }
    if (src_side) cudaStreamWaitEvent(s, c->ev_join, 0);
    GatherArgs ga{m, W, c->w.uv, A.Ga, A.Guv, A.Gsl, Wbar, bbar};
#define SWE_GA(NN)                                                                          \
    {                                                                                       \
        Timed tm(c, KC_ADJ, s);                                                             \
        k_gather_adj<NN><<<grid_for(m.KN, GA_TPB), GA_TPB, 0, s>>>(ga);                     \
    }
    SWE_SWITCH_N_ADJ(m.N, SWE_GA)
#undef SWE_GA
    if (src_now && !src_side) launch_src_adjoint(c, A.Gsrc, bbar, s);
}

void launch_src_adjoint(swe_ctx* c, const double* Gsrc, double* bbar, cudaStream_t s) {
#define SWE_SA(NN)                                                                          \
    {                                                                                       \
        Timed tm(c, KC_ADJ, s);                                                             \
        k_src_adj<NN><<<grid_for(c->m.K, adj_ne<NN>()), adj_ne<NN>() * (NN + 1), 0, s>>>(c->m, Gsrc, bbar); \
    }
    SWE_SWITCH_N_ADJ(c->m.N, SWE_SA)
#undef SWE_SA
}

void launch_limit_record(swe_ctx* c, double* W, uint8_t* act, int32_t* amin, uint8_t* cut, cudaStream_t s) {
    LimRecArgs a{c->m, W, c->w.uv, act, amin, cut, c->h_tol, c->w.status};
#define SWE_LR(NN)                                                                          \
    {                                                                                       \
        Timed tm(c, KC_UPDATE, s);                                                          \
        k_limit_rec<NN><<<grid_for(c->m.K, 4), 128, 0, s>>>(a);                             \
    }
    SWE_SWITCH_N_ADJ(c->m.N, SWE_LR)
#undef SWE_LR
}

void launch_update_adjoint(swe_ctx* c, int mode, double* Wb, const double* Y, const uint8_t* act,
                           const int32_t* amin, const uint8_t* cut, double* Khb, double* Rb, double* Wnb, double a,
                           double b, double dt, cudaStream_t s) {
    UpdAdjArgs u{c->m, Wb, Y, act, amin, cut, Khb, Rb, Wnb, a, b, dt, c->p.limiter};
#define SWE_UA(NN)                                                                          \
    {                                                                                       \
        Timed tm(c, KC_ADJ, s);                                                             \
        if (mode == 1) k_update_adj<NN, 1><<<grid_for(c->m.K, 4), 128, 0, s>>>(u);          \
        else k_update_adj<NN, 2><<<grid_for(c->m.K, 4), 128, 0, s>>>(u);                    \
    }
    SWE_SWITCH_N_ADJ(c->m.N, SWE_UA)
#undef SWE_UA
}

void launch_gauge(swe_ctx* c, const double* W, int ng, const int32_t* elem, const double* wts,
                  const double* target, double* values, double* loss, double* Wb, cudaStream_t s) {
#define SWE_GG(NN)                                                                          \
    {                                                                                       \
        Timed tm(c, KC_ADJ, s);                                                             \
        k_gauge<NN><<<1, 128, 0, s>>>(c->m, W, ng, elem, wts, target, values, loss, Wb);    \
    }
    SWE_SWITCH_N_ADJ(c->m.N, SWE_GG)
#undef SWE_GG
}

void launch_axpy(swe_ctx* c, long long count, double a, const double* x, double* y, cudaStream_t s) {
    Timed tm(c, KC_ADJ, s);
    const int blocks = grid_for(count, 256) > 4096 ? 4096 : grid_for(count, 256);
    k_axpy<<<blocks, 256, 0, s>>>(count, a, x, y);
}

}  // namespace swe
