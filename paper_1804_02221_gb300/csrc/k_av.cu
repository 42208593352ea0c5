// Artificial viscosity, per element: the modal smoothness indicator and the
// viscosity epsilon_k (App. A), then, only where epsilon_k > 0, the BR1
// gradients of u and v (Eq. BR1, strong form with the (U* - u) lift on the
// outward normal) and the viscous fluxes F^v = h eps (U1, V1),
// G^v = h eps (U2, V2) (Thm. 1) with their contravariant forms for the volume
// kernel and their values at the element's side nodes for the interface
// average.
#include <math.h>

#include "kcommon.cuh"

namespace swe {
namespace {

struct AvArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Ustar;
    double* Fvt;
    double* Fvtr;
    double* eps;
    double eps0, smin, smax;
    const int* stop;
};

template <int N>
constexpr int av_ne() {
    return (128 / ((N + 1) * (N + 1))) > 0 ? 128 / ((N + 1) * (N + 1)) : 1;
}

template <int N>
__global__ void k_av(AvArgs a) {
    constexpr int n = N + 1, nn = n * n, NE = av_ne<N>(), BLK = NE * nn;
    constexpr double iw0 = N * (N + 1) / 2.0;
    __shared__ double sh_h[BLK], sh_u[BLK], sh_v[BLK], sh_T[BLK];
    __shared__ double sh_q[4][BLK];
    __shared__ double sh_D[nn], sh_Vi[nn];
    __shared__ double sh_eps[NE];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    const int t = threadIdx.x;
    const int e = t / nn, node = t - e * nn;
    const long long k = (long long)blockIdx.x * NE + e;
    const bool valid = t < BLK && k < m.K;
    const long long gid = k * nn + node;
    if (t < nn) {
        sh_D[t] = Dm<N>(t / n, t % n);
        sh_Vi[t] = c_Vinv[mat_offset(N) + t];
    }
    if (t < BLK) {
        sh_h[t] = valid ? a.W[gid] : 0.0;
        sh_u[t] = valid ? a.uv[gid] : 0.0;
        sh_v[t] = valid ? a.uv[m.KN + gid] : 0.0;
    }
    __syncthreads();
    const int i = node % n, j = node / n;
    const int eb = e * nn;
    // modal coefficients Qhat = Vinv Q Vinv^T (Eq. TransformationToModal),
    // Q[i][j] = h at (xi_i, eta_j): first T[a][j] = sum_i Vinv[a][i] Q[i][j]
    if (t < BLK) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s = fma(sh_Vi[i * n + q], sh_h[eb + j * n + q], s);
        sh_T[t] = s;  // T[a = i][j]
    }
    __syncthreads();
    if (t < BLK) {
        // Qhat[a = i][c = j] = sum_q T[a][q] Vinv[c][q]
        double s = 0.0;
        for (int q = 0; q < n; ++q) s = fma(sh_T[eb + q * n + i], sh_Vi[j * n + q], s);
        const double q2 = s * s;
        const bool top = (i == N) || (j == N);
        const bool low = (i < N) && (j < N);
        const bool sub = low && ((i == N - 1) || (j == N - 1));
        sh_q[0][t] = q2;                 // all modes
        sh_q[1][t] = top ? q2 : 0.0;     // a mode of degree N in some direction
        sh_q[2][t] = low ? q2 : 0.0;     // degree <= N-1 in both
        sh_q[3][t] = sub ? q2 : 0.0;     // degree N-1 in some direction, <= N-1 in both
    }
    __syncthreads();
    // energy sums of Eq. sigmadof in a fixed order, then epsilon (App. A)
    if (t < NE * 4) {
        const int ee = t / 4, which = t - ee * 4;
        double s = 0.0;
        for (int q = 0; q < nn; ++q) s += sh_q[which][ee * nn + q];
        sh_T[ee * nn + which] = s;  // T is free again
    }
    __syncthreads();
    if (t < NE) {
        const double den1 = sh_T[t * nn + 0], num1 = sh_T[t * nn + 1];
        const double den2 = sh_T[t * nn + 2], num2 = sh_T[t * nn + 3];
        double r = den1 > 0.0 ? num1 / den1 : 0.0;
        if (N >= 2) {
            const double r2 = den2 > 0.0 ? num2 / den2 : 0.0;
            r = fmax(r, r2);
        }
        double ep = 0.0;
        if (a.eps0 != 0.0 && r > 0.0) {
            const double sig = log10(r);
            if (sig >= a.smax) ep = a.eps0;
            else if (sig > a.smin)
                ep = 0.5 * a.eps0 * (1.0 + sin(3.14159265358979323846 * (sig - 0.5 * (a.smax + a.smin)) /
                                                (a.smax - a.smin)));
        }
        sh_eps[t] = ep;
        if ((long long)blockIdx.x * NE + t < m.K) a.eps[(long long)blockIdx.x * NE + t] = ep;
    }
    __syncthreads();
    if (!valid) return;
    const double ep = sh_eps[e];
    const bool bnd = (i == 0) || (i == N) || (j == 0) || (j == N);
    const long long KS = m.KS;
    auto side = [&](int f, int p) { return (k * 4 + f) * n + p; };
    if (!(ep > 0.0)) {
        if (bnd) {
            auto zero = [&](int f, int p) {
                const long long sl = side(f, p);
                a.Fvtr[sl] = 0.0;
                a.Fvtr[KS + sl] = 0.0;
                a.Fvtr[2 * KS + sl] = 0.0;
                a.Fvtr[3 * KS + sl] = 0.0;
            };
            if (j == 0) zero(0, i);
            if (i == N) zero(1, j);
            if (j == N) zero(2, i);
            if (i == 0) zero(3, j);
        }
        return;
    }
    // BR1 gradient: D applied along xi and eta plus the interface lift
    double ux = 0.0, ue = 0.0, vx = 0.0, ve = 0.0;
    for (int q = 0; q < n; ++q) {
        const double di = sh_D[i * n + q], dj = sh_D[j * n + q];
        ux = fma(di, sh_u[eb + j * n + q], ux);
        vx = fma(di, sh_v[eb + j * n + q], vx);
        ue = fma(dj, sh_u[eb + q * n + i], ue);
        ve = fma(dj, sh_v[eb + q * n + i], ve);
    }
    const double u = sh_u[t], v = sh_v[t];
    if (i == N) { const long long sl = side(1, j); ux += iw0 * (a.Ustar[sl] - u); vx += iw0 * (a.Ustar[KS + sl] - v); }
    if (i == 0) { const long long sl = side(3, j); ux -= iw0 * (a.Ustar[sl] - u); vx -= iw0 * (a.Ustar[KS + sl] - v); }
    if (j == N) { const long long sl = side(2, i); ue += iw0 * (a.Ustar[sl] - u); ve += iw0 * (a.Ustar[KS + sl] - v); }
    if (j == 0) { const long long sl = side(0, i); ue -= iw0 * (a.Ustar[sl] - u); ve -= iw0 * (a.Ustar[KS + sl] - v); }
    const double axx = m.axx[gid], axy = m.axy[gid], aex = m.aex[gid], aey = m.aey[gid];
    // J grad u = a_xi du/dxi + a_eta du/deta; F^v = h eps grad(.)
    const double he = sh_h[t] * ep * m.rJ[gid];
    const double F2 = he * fma(axx, ux, aex * ue);  // h eps U1
    const double G2 = he * fma(axy, ux, aey * ue);  // h eps U2
    const double F3 = he * fma(axx, vx, aex * ve);  // h eps V1
    const double G3 = he * fma(axy, vx, aey * ve);  // h eps V2
    const long long KN = m.KN;
    a.Fvt[gid] = fma(axx, F2, axy * G2);
    a.Fvt[KN + gid] = fma(axx, F3, axy * G3);
    a.Fvt[2 * KN + gid] = fma(aex, F2, aey * G2);
    a.Fvt[3 * KN + gid] = fma(aex, F3, aey * G3);
    if (bnd) {
        auto put = [&](int f, int p) {
            const long long sl = side(f, p);
            a.Fvtr[sl] = F2;
            a.Fvtr[KS + sl] = F3;
            a.Fvtr[2 * KS + sl] = G2;
            a.Fvtr[3 * KS + sl] = G3;
        };
        if (j == 0) put(0, i);
        if (i == N) put(1, j);
        if (j == N) put(2, i);
        if (i == 0) put(3, j);
    }
}

template <int N>
void av_n(swe_ctx* c, const AvArgs& a, cudaStream_t s) {
    constexpr int NE = av_ne<N>();
    const int threads = ((NE * (N + 1) * (N + 1) + 31) / 32) * 32;
    Timed tm(c, KC_AV, s);
    k_av<N><<<grid_for(c->m.K, NE), threads, 0, s>>>(a);
}

}  // namespace

void init_tables_av() { upload_tables(); }

void launch_av(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    AvArgs a{c->m, W, c->w.uv, c->w.Ustar, c->w.Fvt, c->w.Fvtr, c->w.eps, c->p.eps0, c->sigma_min,
             c->sigma_max, stop};
    switch (c->m.N) {
        case 1: av_n<1>(c, a, s); break;
        case 2: av_n<2>(c, a, s); break;
        case 3: av_n<3>(c, a, s); break;
        case 4: av_n<4>(c, a, s); break;
        case 5: av_n<5>(c, a, s); break;
        case 6: av_n<6>(c, a, s); break;
        case 7: av_n<7>(c, a, s); break;
        case 8: av_n<8>(c, a, s); break;
        case 9: av_n<9>(c, a, s); break;
        case 10: av_n<10>(c, a, s); break;
        case 11: av_n<11>(c, a, s); break;
        case 12: av_n<12>(c, a, s); break;
        default: break;
    }
}

}  // namespace swe
