// Volume kernel: split-form flux differencing (Eq. fluxDiffFormF with the
// curvilinear two-point fluxes of Eq. Fmij and Eq. volumeFluxes), the
// interface-flux lift of Eq. fluxDiffFormF, the BR1 viscous divergence of
// Eq. ViscTermsDisc, the well-balanced source of Eq. SourceDisc, and the
// scaling R = -(L - S - L^v)/J of Eq. CurvilinearECDGSEMviscous.
//
// Design (FP64-ALU bound on GB300): the two-point flux is symmetric, so each
// node pair (i,m) of a line is evaluated once and scattered to both ends with
// D~_im and D~_mi = 2 D_mi (the diagonal of D~ = 2D + S vanishes for LGL
// nodes). One thread owns one xi-line or one eta-line of an element and keeps
// that line's accumulators in registers; the loops are fully unrolled, so the
// derivative-matrix entries are compile-time constant-bank operands. With the
// contravariant vector a = (y_eta, -x_eta) on xi-lines and (-y_xi, x_xi) on
// eta-lines, and sums instead of averages, one pair costs
//   A = a_i + a_m,  Q = (hu_i+hu_m) A_x + (hv_i+hv_m) A_y,  P = 2 g h_i h_m,
//   X2 = (u_i+u_m) Q + P A_x,  X3 = (v_i+v_m) Q + P A_y
// with the flux components Q/4, X2/8, X3/8; the accumulators hold 2 L_1,
// 4 L_2, 4 L_3 and are rescaled once per node.
#include "kcommon.cuh"

namespace swe {
namespace {

enum {
    F_H, F_HU, F_HV, F_U, F_V, F_P, F_AX, F_AY, F_EX, F_EY, F_A1, F_A2, F_A3,
    F_BASE_COUNT,
    F_FT2 = F_BASE_COUNT, F_FT3, F_GT2, F_GT3,
    F_AV_COUNT
};

struct VolArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Fout;
    const double* Fvt;
    const double* Fvout;
    const double* eps;
    double* R;
    const int* stop;
};

template <int N>
constexpr int vol_ne() {
    return (128 / (2 * (N + 1))) > 0 ? 128 / (2 * (N + 1)) : 1;
}

template <int N, bool AV>
constexpr size_t vol_smem() {
    return sizeof(double) * ((size_t)(AV ? F_AV_COUNT : F_BASE_COUNT) * vol_ne<N>() * (N + 1) * (N + 1) +
                             (AV ? (N + 1) * (N + 1) : 0));
}

template <int N, bool AV>
__global__ void __launch_bounds__(vol_ne<N>() * 2 * (N + 1)) k_volume(VolArgs a) {
    constexpr int n = N + 1, nn = n * n, NE = vol_ne<N>(), TPE = 2 * n, NT = NE * TPE;
    constexpr int BLK = NE * nn;
    constexpr double iw0 = N * (N + 1) / 2.0;  // 1/omega_0
    extern __shared__ double sm[];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    const int t = threadIdx.x;
    const long long k0 = (long long)blockIdx.x * NE;
    double* s = sm;
    auto S = [&](int f) { return s + f * BLK; };
    double* sD = sm + (AV ? F_AV_COUNT : F_BASE_COUNT) * BLK;

    // ---- stage the block's elements in shared memory --------------------
    for (int idx = t; idx < BLK; idx += NT) {
        const int e = idx / nn;
        const long long k = k0 + e;
        double h = 0, hu = 0, hv = 0, u = 0, v = 0, ax = 0, ay = 0, ex = 0, ey = 0;
        if (k < m.K) {
            const long long gid = k * nn + (idx - e * nn);
            h = a.W[gid];
            hu = a.W[m.KN + gid];
            hv = a.W[2 * m.KN + gid];
            u = a.uv[gid];
            v = a.uv[m.KN + gid];
            ax = m.axx[gid];
            ay = m.axy[gid];
            ex = m.aex[gid];
            ey = m.aey[gid];
            if (AV && a.eps[k] > 0.0) {
                S(F_FT2)[idx] = a.Fvt[gid];
                S(F_FT3)[idx] = a.Fvt[m.KN + gid];
                S(F_GT2)[idx] = a.Fvt[2 * m.KN + gid];
                S(F_GT3)[idx] = a.Fvt[3 * m.KN + gid];
            }
        }
        S(F_H)[idx] = h;
        S(F_HU)[idx] = hu;
        S(F_HV)[idx] = hv;
        S(F_U)[idx] = u;
        S(F_V)[idx] = v;
        S(F_P)[idx] = 2.0 * m.g * h;
        S(F_AX)[idx] = ax;
        S(F_AY)[idx] = ay;
        S(F_EX)[idx] = ex;
        S(F_EY)[idx] = ey;
    }
    if (AV)
        for (int idx = t; idx < nn; idx += NT) sD[idx] = Dm<N>(idx / n, idx % n);
    __syncthreads();

    // ---- symmetric pair loop, one line per thread -----------------------
    const int e = t / TPE, l = t - e * TPE;
    const bool xi = l < n;
    const int line = xi ? l : l - n;
    const int base = e * nn + (xi ? line * n : line);
    const int stride = xi ? 1 : n;
    const double* sAx = xi ? S(F_AX) : S(F_EX);
    const double* sAy = xi ? S(F_AY) : S(F_EY);
    const double* sH = S(F_H);
    const double* sHU = S(F_HU);
    const double* sHV = S(F_HV);
    const double* sU = S(F_U);
    const double* sV = S(F_V);
    const double* sP = S(F_P);
    double A1[n], A2[n], A3[n];
#pragma unroll
    for (int p = 0; p < n; ++p) A1[p] = A2[p] = A3[p] = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int ni = base + i * stride;
        const double hu_i = sHU[ni], hv_i = sHV[ni], u_i = sU[ni], v_i = sV[ni], p_i = sP[ni];
        const double ax_i = sAx[ni], ay_i = sAy[ni];
#pragma unroll
        for (int q = i + 1; q < n; ++q) {
            const int nq = base + q * stride;
            const double cx = ax_i + sAx[nq];
            const double cy = ay_i + sAy[nq];
            const double Q = fma(hu_i + sHU[nq], cx, (hv_i + sHV[nq]) * cy);
            const double P = p_i * sH[nq];
            const double X2 = fma(u_i + sU[nq], Q, P * cx);
            const double X3 = fma(v_i + sV[nq], Q, P * cy);
            const double dij = Dm<N>(i, q), dji = Dm<N>(q, i);
            A1[i] = fma(dij, Q, A1[i]);
            A1[q] = fma(dji, Q, A1[q]);
            A2[i] = fma(dij, X2, A2[i]);
            A2[q] = fma(dji, X2, A2[q]);
            A3[i] = fma(dij, X3, A3[i]);
            A3[q] = fma(dji, X3, A3[q]);
        }
    }
    double* sA1 = S(F_A1);
    double* sA2 = S(F_A2);
    double* sA3 = S(F_A3);
    if (xi) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sA1[base + p * stride] = A1[p];
            sA2[base + p * stride] = A2[p];
            sA3[base + p * stride] = A3[p];
        }
    }
    __syncthreads();
    if (!xi) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
            sA1[base + p * stride] += A1[p];
            sA2[base + p * stride] += A2[p];
            sA3[base + p * stride] += A3[p];
        }
    }
    __syncthreads();

    // ---- per node: lifts, viscous divergence, source, scaling -----------
    for (int idx = t; idx < BLK; idx += NT) {
        const int ee = idx / nn, node = idx - ee * nn;
        const long long k = k0 + ee;
        if (k >= m.K) continue;
        const int i = node % n, j = node / n;
        const long long gid = k * nn + node;
        double a1 = sA1[idx], a2 = sA2[idx], a3 = sA3[idx];
        // interface flux: + (1/omega_0) F_out on every face through the node
        auto lift = [&](int f, int pnode) {
            const long long sl = (k * 4 + f) * n + pnode;
            a1 = fma(2.0 * iw0, a.Fout[sl], a1);
            a2 = fma(4.0 * iw0, a.Fout[m.KS + sl], a2);
            a3 = fma(4.0 * iw0, a.Fout[2 * m.KS + sl], a3);
        };
        if (j == 0) lift(0, i);
        if (i == N) lift(1, j);
        if (j == N) lift(2, i);
        if (i == 0) lift(3, j);
        if (AV) {
            double L2 = 0.0, L3 = 0.0;
            const bool visc = a.eps[k] > 0.0;
            const int eb = ee * nn;
            if (visc) {
                for (int q = 0; q < n; ++q) {
                    const double di = sD[i * n + q], dj = sD[j * n + q];
                    L2 = fma(di, S(F_FT2)[eb + j * n + q], L2);
                    L3 = fma(di, S(F_FT3)[eb + j * n + q], L3);
                    L2 = fma(dj, S(F_GT2)[eb + q * n + i], L2);
                    L3 = fma(dj, S(F_GT3)[eb + q * n + i], L3);
                }
            }
            const double ft2 = visc ? S(F_FT2)[idx] : 0.0, ft3 = visc ? S(F_FT3)[idx] : 0.0;
            const double gt2 = visc ? S(F_GT2)[idx] : 0.0, gt3 = visc ? S(F_GT3)[idx] : 0.0;
            auto vlift = [&](int f, int pnode, double own2, double own3) {
                const long long sl = (k * 4 + f) * n + pnode;
                L2 += iw0 * (a.Fvout[sl] - own2);
                L3 += iw0 * (a.Fvout[m.KS + sl] - own3);
            };
            if (j == 0) vlift(0, i, -gt2, -gt3);
            if (i == N) vlift(1, j, ft2, ft3);
            if (j == N) vlift(2, i, gt2, gt3);
            if (i == 0) vlift(3, j, -ft2, -ft3);
            a2 = fma(-4.0, L2, a2);
            a3 = fma(-4.0, L3, a3);
        }
        const double rJ = m.rJ[gid];
        const double h = S(F_H)[idx];
        a.R[gid] = -0.5 * rJ * a1;
        a.R[m.KN + gid] = fma(h, m.srcx[gid], -0.25 * rJ * a2);
        a.R[2 * m.KN + gid] = fma(h, m.srcy[gid], -0.25 * rJ * a3);
    }
}

template <int N, bool AV>
void launch_n(swe_ctx* c, const VolArgs& a, cudaStream_t s) {
    constexpr int NE = vol_ne<N>();
    constexpr size_t smem = vol_smem<N, AV>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_volume<N, AV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int blocks = grid_for(c->m.K, NE);
    Timed tm(c, KC_VOLUME, s);
    k_volume<N, AV><<<blocks, NE * 2 * (N + 1), smem, s>>>(a);
}

}  // namespace

void init_tables_volume() { upload_tables(); }

void launch_volume(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop) {
    VolArgs a{c->m, W, c->w.uv, c->w.Fout, c->w.Fvt, c->w.Fvout, c->w.eps, R, stop};
    const bool av = c->p.av != 0;
#define SWE_VOL_CASE(NN)                                         \
    case NN:                                                     \
        if (av) launch_n<NN, true>(c, a, s);                     \
        else launch_n<NN, false>(c, a, s);                       \
        break;
    switch (c->m.N) {
        SWE_VOL_CASE(1) SWE_VOL_CASE(2) SWE_VOL_CASE(3) SWE_VOL_CASE(4)
        SWE_VOL_CASE(5) SWE_VOL_CASE(6) SWE_VOL_CASE(7) SWE_VOL_CASE(8)
        SWE_VOL_CASE(9) SWE_VOL_CASE(10) SWE_VOL_CASE(11) SWE_VOL_CASE(12)
        default: break;
    }
#undef SWE_VOL_CASE
}

}  // namespace swe
