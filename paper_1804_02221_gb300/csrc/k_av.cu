// Artificial viscosity: the element smoothness indicator and viscosity
// epsilon_k (App. A), then, only where epsilon_k > 0, the BR1 gradients of u
// and v (Eq. BR1, strong form with the (U* - u) lift on the outward normal)
// and the viscous fluxes F^v = h eps (U1, V1), G^v = h eps (U2, V2)
// (Thm. 1), with their contravariant forms F~v, G~v, their values at the
// element's side nodes for the interface average, and the volume part of the
// viscous divergence of Eq. ViscTermsDisc, L^v = sum_q D_iq F~v_(q,j) +
// D_jq G~v_(i,q), which the volume kernel adds (weighted by -w_i w_j) to the
// viscous elements' nodes: computed here by the warp that owns the element,
// so that the volume kernel's blocks stay balanced whether or not they hold
// viscous elements.
//
// Indicator without the full modal transform. With Qhat = Vinv Q Vinv^T the
// three energies of Eq. sigmadof are
//   E_all = sum Qhat^2,  E_top = sum over modes of degree N in some direction,
//   E_sub = sum over modes of degree N-1 in some direction and <= N-1 in both.
// LGL quadrature (N+1 nodes) integrates f^2 of a degree-N polynomial f up to
// one term: int f^2 = sum_i w_i f_i^2 - k f_N^2, k = (N+1)/N, f_N its top
// normalised Legendre coefficient (the rule is exact to degree 2N-1, and its
// error on degree 2N depends only on the leading coefficient). Applied along
// each direction, with the projections
//   y_xi[j] = sum_i Vinv[N][i] Q[i][j],   y_eta[i] = sum_j Vinv[N][j] Q[i][j],
//   z_xi[j] = sum_i Vinv[N-1][i] Q[i][j], z_eta[i] = sum_j Vinv[N-1][j] Q[i][j],
//   B0 = Qhat[N][N], C0 = Qhat[N][N-1], B2 = Qhat[N-1][N], C2 = Qhat[N-1][N-1],
// and S_y = sum w y^2 etc.:
//   E_all = sum_ij w_i w_j Q_ij^2 - k (S_yxi + S_yeta) + k^2 B0^2
//   E_top = S_yxi + S_yeta - (2k+1) B0^2
//   E_sub = S_zxi - (k+1) B2^2 + S_zeta - (k+1) C0^2 - C2^2
// which costs O(N^2) per element instead of the O(N^3) transform. One warp
// evaluates several elements at a time (8 to 32, av_epw), so the per-element
// sums are short butterflies over 32/av_epw lanes and the scalar work runs on
// av_epw lanes at once.
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
    double* Lv;
    double* eps;
    int* vlist;   // [K] the viscous elements of the state (indicator kernel), in no fixed order
    int* vcount;  // their number
    EpsParams ep;
    const int* stop;
};

constexpr int AV_WPB = 2;  // warps per block

// Elements per warp. Wide: 32 up to N = 4, 16 for N = 5..8, 8 above
// (measured on the dam break at 4.2M nodes: 32 instead of 16 at N = 2, 3 and
// of 8 at N = 4 took 12-17% off the kernel, 16 instead of 8 at N = 5 and 7
// took 4-5%): more elements per warp spread the per-element scalar work (the
// eight sums, epsilon) over more lanes and keep more loads in flight. Narrow:
// 32 at N = 1, 16 at N = 2, 3, 8 above, for meshes too small to give the wide
// mapping enough warps (64 x 64 quads at N = 4: 64 blocks for 152 SMs, the
// kernel 1.8x slower than narrow).
template <int N, bool WIDE>
constexpr int av_epw() {
    if (WIDE) return N <= 4 ? 32 : (N <= 8 ? 16 : 8);
    return N == 1 ? 32 : (N <= 3 ? 16 : 8);
}

// epsilon from the nine sums of one element (S_yxi, S_yeta, S_zxi, S_zeta,
// B0, C0, B2, C2, sum w w Q^2).
template <int N>
__device__ __forceinline__ double epsilon_from_sums(const double* S, const EpsParams& ep) {
    constexpr double k1 = (N + 1.0) / N;
    const double B0 = S[4], C0 = S[5], B2 = S[6], C2 = S[7];
    const double e_all = S[8] - k1 * (S[0] + S[1]) + k1 * k1 * B0 * B0;
    const double e_top = S[0] + S[1] - (2.0 * k1 + 1.0) * B0 * B0;
    const double e_sub = S[2] - (k1 + 1.0) * B2 * B2 + S[3] - (k1 + 1.0) * C0 * C0 - C2 * C2;
    const double den2 = e_all - e_top;
    // both ratios at most 10^sigma_min (epsilon = 0, the common case for
    // smooth elements) is decided without a division
    const bool flat = !(e_top > ep.rmin * e_all) && (N < 2 || !(e_sub > ep.rmin * den2));
    if (flat || ep.eps0 == 0.0) return 0.0;
    double r = e_all > 0.0 ? e_top / e_all : 0.0;
    if (N >= 2 && den2 > 0.0) r = fmax(r, e_sub / den2);
    if (!(r > ep.rmin)) return 0.0;
    if (r >= ep.rmax) return ep.eps0;
    // epsilon is continuous in sigma = log10(r), so the comparisons with
    // 10^sigma_min and 10^sigma_max above decide the two flat branches
    const double sig = log10(r);
    if (sig >= ep.smax) return ep.eps0;
    if (!(sig > ep.smin)) return 0.0;
    return 0.5 * ep.eps0 *
           (1.0 + sin(3.14159265358979323846 * (sig - 0.5 * (ep.smax + ep.smin)) / (ep.smax - ep.smin)));
}

// The smoothness indicator and epsilon of every element; the viscous
// elements are appended to a list (in no fixed order: every element's fluxes
// are computed independently, so the results do not depend on it) for the
// viscous-flux kernel.
template <int N, bool WIDE>
__global__ void __launch_bounds__(32 * AV_WPB) k_av(AvArgs a) {
    constexpr int AV_EPW = av_epw<N, WIDE>();
    constexpr int LPE = 32 / AV_EPW;  // lanes per element for the sums (4, 2 or 1)
    constexpr int SPL = 8 / LPE;      // projection sums per lane (2, 4 or 8)
    constexpr int n = N + 1, nn = n * n, P4 = 4 * n;
    __shared__ double sVi[nn], sWW[nn];
    __shared__ double sQ[AV_WPB][AV_EPW][nn];
    __shared__ double sP[AV_WPB][AV_EPW][P4];
    __shared__ double sS[AV_WPB][AV_EPW][9];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        sVi[t] = c_Vinv[mat_offset(N) + t];
        sWW[t] = c_w[vec_offset(N) + t % n] * c_w[vec_offset(N) + t / n];
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long k0 = ((long long)blockIdx.x * AV_WPB + w) * AV_EPW;
    if (k0 >= m.K) return;  // whole warps leave together; no block barrier follows
    const int ne = (int)((m.K - k0) < AV_EPW ? (m.K - k0) : AV_EPW);
    double(*Q)[nn] = sQ[w];
    // ---- water heights of the warp's elements (contiguous in memory) --
    // a compile-time trip count, unrolled: the loads of all iterations
    // are in flight together
    constexpr int LQ = (AV_EPW * nn + 31) / 32;
#pragma unroll
    for (int r = 0; r < LQ; ++r) {
        const int idx = lane + 32 * r;
        if (idx < AV_EPW * nn) {
            const int e = idx / nn;
            Q[e][idx - e * nn] = e < ne ? a.W[k0 * nn + idx] : 0.0;
        }
    }
    __syncwarp();
    // ---- the four projections of every element ------------------------
    // AV_EPW n / 8 tasks per lane, unrolled: the lane's
    // independent dot products interleave, instead of one dependent chain
    // of fused multiply-adds at a time
    static_assert((AV_EPW * P4) % 32 == 0, "projection tasks fill whole warps");
#pragma unroll
    for (int r = 0; r < AV_EPW * P4 / 32; ++r) {
        const int s = lane + 32 * r;
        const int e = s / P4, L = s - e * P4, t = L / n, p = L - t * n;
        const double* vr = sVi + (t < 2 ? N : N - 1) * n;
        // t even: sum over i at j = p; t odd: sum over j at i = p. One
        // code path with an index stride, so that the lanes of a warp do
        // not split into two half-empty FP64 instruction streams.
        const int b0 = (t & 1) ? p : p * n, st = (t & 1) ? n : 1;
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < n; ++q) v = fma(vr[q], Q[e][b0 + q * st], v);
        sP[w][e][L] = v;
    }
    // ---- sum w w Q^2: LPE lanes per element ----------------------------
    const int e4 = lane / LPE, sub = lane % LPE;
    double swq = 0.0;
#pragma unroll
    for (int r = 0; r < (nn + LPE - 1) / LPE; ++r) {
        const int node = sub + LPE * r;
        const double q = node < nn ? Q[e4][node] : 0.0;
        swq = fma(sWW[node < nn ? node : 0] * q, q, swq);
    }
#pragma unroll
    for (int o = 1; o < LPE; o <<= 1) swq += __shfl_xor_sync(0xffffffffu, swq, o);
    __syncwarp();
    // ---- the eight projection sums: SPL per lane -----------------------
    // sum index m: 0..3 weighted squares of y_xi, y_eta, z_xi, z_eta;
    // 4: B0 = Vinv[N].y_xi, 5: C0 = Vinv[N-1].y_xi, 6: B2 = Vinv[N].z_xi,
    // 7: C2 = Vinv[N-1].z_xi; each written as sum_p (c_p x_p) y_p
#pragma unroll
    for (int h2 = 0; h2 < SPL; ++h2) {
        const int mi = SPL * sub + h2;
        const bool sq = mi < 4;
        const double* x = sP[w][e4] + (sq ? mi : (mi < 6 ? 0 : 2)) * n;
        const double* c = sVi + ((mi & 1) == 0 ? N : N - 1) * n;
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            const double cp = sq ? c_w[vec_offset(N) + p] : c[p];
            const double yp = sq ? x[p] : 1.0;
            s = fma(cp * x[p], yp, s);
        }
        sS[w][e4][mi] = s;
    }
    if (sub == 0) sS[w][e4][8] = swq;
    __syncwarp();
    // ---- epsilon, one lane per element --------------------------------
    if (lane < AV_EPW) {
        const double ep = epsilon_from_sums<N>(sS[w][lane], a.ep);
        if (lane < ne) {
            a.eps[k0 + lane] = ep;
            if (ep > 0.0) a.vlist[atomicAdd(a.vcount, 1)] = (int)(k0 + lane);
        }
    }
}

// The list of viscous elements from the viscosities already in the work
// buffer (the adjoint sweeps set them from the forward pass's records).
__global__ void k_visc_list(long long K, const double* __restrict__ eps, int* __restrict__ vlist,
                            int* __restrict__ vcount) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K;
         k += (long long)gridDim.x * blockDim.x)
        if (eps[k] > 0.0) vlist[atomicAdd(vcount, 1)] = (int)k;
}

// Elements per block of the viscous-flux kernel (one thread per node, whole
// elements, about 128 threads) and its block size in whole warps.
template <int N>
constexpr int vf_eb() {
    return (N + 1) * (N + 1) >= 128 ? 1 : 128 / ((N + 1) * (N + 1));
}
template <int N>
constexpr int vf_threads() {
    return (vf_eb<N>() * (N + 1) * (N + 1) + 31) / 32 * 32;
}

// Viscous elements only, from the list: the BR1 gradients (strong form with
// the (U* - u) lift on the outward normal), the viscous fluxes F^v = h eps
// grad(u), G^v = h eps grad(v), their contravariant forms F~v, G~v, their
// values at the side nodes for the interface average, and the volume part of
// the viscous divergence sum_q D_iq F~v_(q,j) + D_jq G~v_(i,q). One thread per
// node, EB elements per block, the blocks striding over the list; every
// element's nodes run in parallel, so many viscous elements cost what few do
// per element (earlier, one warp took its viscous elements one at a time).
template <int N>
__global__ void __launch_bounds__(vf_threads<N>()) k_visc_flux(AvArgs a) {
    constexpr int n = N + 1, nn = n * n, EB = vf_eb<N>();
    constexpr double iw0 = N * (N + 1) / 2.0;
    __shared__ double sD[nn];
    __shared__ double sU[EB][nn], sV[EB][nn];
    __shared__ double sF[4][EB][nn];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) sD[t] = Dm<N>(t / n, t % n);
    const int t = threadIdx.x, e = t / nn, node = t - e * nn;
    const int i = node % n, j = node / n;
    const long long KS = m.KS, KN = m.KN;
    const int count = *a.vcount;  // the same for every thread: the loop below is uniform
    const int groups = (count + EB - 1) / EB;
    for (int gq = blockIdx.x; gq < groups; gq += gridDim.x) {
        const int li = gq * EB + e;
        const bool live = e < EB && li < count;
        const long long k = live ? a.vlist[li] : 0;
        const long long base = k * nn, side = k * 4 * n, gid = base + node;
        const double ep = live ? a.eps[k] : 0.0;
        if (live) {
            sU[e][node] = a.uv[gid];
            sV[e][node] = a.uv[KN + gid];
        }
        __syncthreads();  // also: sD, and the previous group's reads of sF done
        if (live) {
            const double* U = sU[e];
            const double* V = sV[e];
            // BR1 gradient: D along xi and eta plus the interface lift
            double ux = 0.0, ue = 0.0, vx = 0.0, ve = 0.0;
#pragma unroll
            for (int q = 0; q < n; ++q) {
                const double di = sD[i * n + q], dj = sD[j * n + q];
                ux = fma(di, U[j * n + q], ux);
                vx = fma(di, V[j * n + q], vx);
                ue = fma(dj, U[q * n + i], ue);
                ve = fma(dj, V[q * n + i], ve);
            }
            const double u = U[node], v = V[node];
            if (i == N) { const long long sl = side + 1 * n + j; ux += iw0 * (a.Ustar[sl] - u); vx += iw0 * (a.Ustar[KS + sl] - v); }
            if (i == 0) { const long long sl = side + 3 * n + j; ux -= iw0 * (a.Ustar[sl] - u); vx -= iw0 * (a.Ustar[KS + sl] - v); }
            if (j == N) { const long long sl = side + 2 * n + i; ue += iw0 * (a.Ustar[sl] - u); ve += iw0 * (a.Ustar[KS + sl] - v); }
            if (j == 0) { const long long sl = side + 0 * n + i; ue -= iw0 * (a.Ustar[sl] - u); ve -= iw0 * (a.Ustar[KS + sl] - v); }
            const double axx = m.axx[gid], axy = m.axy[gid], aex = m.aex[gid], aey = m.aey[gid];
            // J grad u = a_xi du/dxi + a_eta du/deta; F^v = h eps grad(.)
            const double he = a.W[gid] * ep * m.rJ[gid];
            const double F2 = he * fma(axx, ux, aex * ue);  // h eps U1
            const double G2 = he * fma(axy, ux, aey * ue);  // h eps U2
            const double F3 = he * fma(axx, vx, aex * ve);  // h eps V1
            const double G3 = he * fma(axy, vx, aey * ve);  // h eps V2
            const double ft2 = fma(axx, F2, axy * G2), ft3 = fma(axx, F3, axy * G3);
            const double gt2 = fma(aex, F2, aey * G2), gt3 = fma(aex, F3, aey * G3);
            a.Fvt[gid] = ft2;
            a.Fvt[KN + gid] = ft3;
            a.Fvt[2 * KN + gid] = gt2;
            a.Fvt[3 * KN + gid] = gt3;
            sF[0][e][node] = ft2;
            sF[1][e][node] = ft3;
            sF[2][e][node] = gt2;
            sF[3][e][node] = gt3;
            auto put = [&](int f, int p) {
                const long long sl = side + f * n + p;
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
        __syncthreads();
        if (live) {
            double L2 = 0.0, L3 = 0.0;
#pragma unroll
            for (int q = 0; q < n; ++q) {
                const double di = sD[i * n + q], dj = sD[j * n + q];
                L2 = fma(di, sF[0][e][j * n + q], L2);
                L3 = fma(di, sF[1][e][j * n + q], L3);
                L2 = fma(dj, sF[2][e][q * n + i], L2);
                L3 = fma(dj, sF[3][e][q * n + i], L3);
            }
            a.Lv[gid] = L2;
            a.Lv[KN + gid] = L3;
        }
        __syncthreads();  // sU, sV and sF are rewritten by the next group
    }
}

template <int N>
void indicator_n(swe_ctx* c, const AvArgs& a, cudaStream_t s) {
    cudaMemsetAsync(a.vcount, 0, sizeof(int), s);
    // the wide mapping when it still gives at least 8 warps per SM
    const bool wide = c->m.K >= (long long)av_epw<N, true>() * 8 * c->sms;
    const int blocks = grid_for(c->m.K, AV_WPB * (wide ? av_epw<N, true>() : av_epw<N, false>()));
    Timed tm(c, KC_AV, s);
    if (wide) k_av<N, true><<<blocks, 32 * AV_WPB, 0, s>>>(a);
    else k_av<N, false><<<blocks, 32 * AV_WPB, 0, s>>>(a);
}

template <int N>
void visc_flux_n(swe_ctx* c, const AvArgs& a, cudaStream_t s) {
    // blocks striding over the list of viscous elements: at most one group of
    // EB elements per block per pass, eight blocks per SM
    const int groups = grid_for(c->m.K, vf_eb<N>());
    const int blocks = groups < 8 * c->sms ? groups : 8 * c->sms;
    Timed tm(c, KC_AV, s);
    k_visc_flux<N><<<blocks, vf_threads<N>(), 0, s>>>(a);
}

}  // namespace

void init_tables_av() { upload_tables(); }

void launch_visc_list(swe_ctx* c, cudaStream_t s) {
    cudaMemsetAsync(c->w.vcount, 0, sizeof(int), s);
    const int blocks = grid_for(c->m.K, 256) < 8 * c->sms ? grid_for(c->m.K, 256) : 8 * c->sms;
    Timed tm(c, KC_AV, s);
    k_visc_list<<<blocks, 256, 0, s>>>(c->m.K, c->w.eps, c->w.vlist, c->w.vcount);
}

EpsParams eps_params(const swe_ctx* c) {
    return EpsParams{c->p.eps0, c->sigma_min, c->sigma_max, pow(10.0, c->sigma_min), pow(10.0, c->sigma_max)};
}

void launch_indicator(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    AvArgs a{c->m, W, c->w.uv, c->w.Ustar, c->w.Fvt, c->w.Fvtr, c->w.Lv, c->w.eps, c->w.vlist, c->w.vcount,
             eps_params(c), stop};
    switch (c->m.N) {
        case 1: indicator_n<1>(c, a, s); break;
        case 2: indicator_n<2>(c, a, s); break;
        case 3: indicator_n<3>(c, a, s); break;
        case 4: indicator_n<4>(c, a, s); break;
        case 5: indicator_n<5>(c, a, s); break;
        case 6: indicator_n<6>(c, a, s); break;
        case 7: indicator_n<7>(c, a, s); break;
        case 8: indicator_n<8>(c, a, s); break;
        case 9: indicator_n<9>(c, a, s); break;
        case 10: indicator_n<10>(c, a, s); break;
        case 11: indicator_n<11>(c, a, s); break;
        case 12: indicator_n<12>(c, a, s); break;
        default: break;
    }
}

void launch_visc_flux(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    AvArgs a{c->m, W, c->w.uv, c->w.Ustar, c->w.Fvt, c->w.Fvtr, c->w.Lv, c->w.eps, c->w.vlist, c->w.vcount,
             eps_params(c), stop};
    switch (c->m.N) {
        case 1: visc_flux_n<1>(c, a, s); break;
        case 2: visc_flux_n<2>(c, a, s); break;
        case 3: visc_flux_n<3>(c, a, s); break;
        case 4: visc_flux_n<4>(c, a, s); break;
        case 5: visc_flux_n<5>(c, a, s); break;
        case 6: visc_flux_n<6>(c, a, s); break;
        case 7: visc_flux_n<7>(c, a, s); break;
        case 8: visc_flux_n<8>(c, a, s); break;
        case 9: visc_flux_n<9>(c, a, s); break;
        case 10: visc_flux_n<10>(c, a, s); break;
        case 11: visc_flux_n<11>(c, a, s); break;
        case 12: visc_flux_n<12>(c, a, s); break;
        default: break;
    }
}

void launch_av(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    launch_indicator(c, W, s, stop);
    launch_visc_flux(c, W, s, stop);
}

}  // namespace swe
