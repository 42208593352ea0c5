// Volume kernel, the template of all launch shapes: split-form flux
// differencing (Eq. fluxDiffFormF with the curvilinear two-point fluxes of
// Eq. Fmij and Eq. volumeFluxes), the
// interface-flux lift of Eq. fluxDiffFormF, the BR1 viscous divergence of
// Eq. ViscTermsDisc, the well-balanced source of Eq. SourceDisc, and the
// scaling R = -(L - S - L^v)/J of Eq. CurvilinearECDGSEMviscous.
//
// Design (FP64-ALU bound on GB300):
//  * The two-point flux is symmetric, so each node pair (i, q) of a line is
//    evaluated once. The accumulators hold w_i w_j L (the quadrature weight
//    of the node times L); by the SBP property w_q D_qi = -w_i D_iq, so the
//    partner node receives exactly the negative of the node's contribution,
//    and the diagonal of D~ = 2D + S vanishes for LGL nodes.
//  * The static per-pair factor w_i w_j D_iq / 4 (a_i + a_q) (a the
//    contravariant vector of the line direction: (y_eta, -x_eta) along xi,
//    (-y_xi, x_xi) along eta) is precomputed on the host and read as one
//    16-byte (Sx, Sy) load. The pair's fluxes are
//      Q  = (hu_i+hu_q) Sx + (hv_i+hv_q) Sy,   P = 2g h_i h_q,
//      X2 = (u_i+u_q) Q + P Sx,                X3 = (v_i+v_q) Q + P Sy,
//    with contributions (2Q, X2, X3) to node i and their negatives to node
//    q. The own-velocity parts u_i Q (node i) and u_q Q (node q) are not
//    formed per pair: each node accumulates A1 = sum of +-Q and, per pair,
//    only the partner's velocity term, u_q Q + P Sx at node i and
//    -(u_i Q + P Sx) at node q; after both lines the node adds u A1 (and
//    v A1), and the mass row 2 A1 is scaled by 2f = -2/(w_i w_j J) instead
//    of doubling A1. One pair is then 15 FP64 instructions (4 for Q,
//    1 for P, 2 for the mass sums, 8 fused multiply-adds for the momenta).
//    From N = 3 up the pressure parts P Sx = p_i (h_q Sx) are summed per
//    node as h_q Sx (B2, B3) and scaled by the node's p = 2g h once per line
//    (once per node with the shuffle hand-over): 14 per pair. The sums start
//    from w_i w_j gamma / 4 (the split bathymetry source, sum_q b_q Sx over
//    both lines), so the scaling also forms the source term h srcx and the
//    end takes one product less per momentum component.
//  * One thread per element line: it runs its xi-line, hands the results
//    over (through shared memory, or at N = 3 and 7 by a transpose across
//    the element's lanes with warp shuffles, at N = 7 pressure sums
//    included), then
//    runs the eta-line with the same index starting from them, and finishes
//    the nodes of that column (interface lifts, viscous terms, source,
//    scaling by -1/(w_i w_j J)) in registers.
//  * The volume part of the viscous divergence (sum_q D_iq F~v + D_jq G~v)
//    of the few viscous elements comes from the AV kernel (Lv); here it is
//    weighted by -w_i w_j and added, with the viscous interface lifts. A
//    block holding a viscous element then costs what the others cost, and
//    the AV variant stages nothing more than the inviscid one.
//    The loops are fully unrolled: all pair indices are compile-time.
//  * Launch shapes: blocks of TPB/(N+1) elements (TPB = 64, 128, 256), one
//    translation unit per shape; every shape computes every element with the
//    same instructions in the same order, so the results are bitwise equal
//    and the shape is a pure performance choice (swe_autotune).
#pragma once
#include "kcommon.cuh"

namespace swe {
namespace {

// Shared-memory planes of the staged elements.
enum { F_H, F_HU, F_HV, F_U, F_V, F_P, F_A1, F_A2, F_A3, F_COUNT };

struct VolArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* Fout;
    const double* Fvt;
    const double* Fvout;
    const double* Lv;
    const double* eps;
    const uint32_t* touch;  // bit f: a viscous flux crosses side f (viscous face kernel)
    double* R;
    const int* stop;
};

// Elements per block of the launch shape with (about) TPB threads.
template <int N, int TPB>
constexpr int vol_ne() {
    return (TPB / (N + 1)) > 0 ? TPB / (N + 1) : 1;
}

// Pressure parts of the pair fluxes summed per node (14 FP64 instructions
// per pair and 2 or 4 per node instead of 15 per pair), the sums started from
// the source (2 per node fewer at the end): a gain from N = 3 up (measured:
// N = 3 -5%, N = 4 -3%, N = 5, 6, 8 -3%; without the source in the sums the
// per-node products cost what the pairs save at N = 3).
template <int N>
constexpr bool vol_pressure_sums() {
    return pressure_sums_degree(N);
}

// The xi -> eta hand-over through warp shuffles. Where n = N + 1 is a power
// of two (N = 3 and 7 of the line kernel's degrees), every element's n lines
// are n consecutive lanes of one warp, and the hand-over is an n x n
// transpose of each accumulator across those lanes: the block needs no
// hand-over planes and no second barrier. With the pressure sums (N = 7)
// the sums travel with the other accumulators unscaled and are scaled by
// 2g h once per node, after the eta-line (2 FP64 instructions per node
// fewer), and the block stages only the five state planes.
template <int N>
constexpr bool vol_shfl() {
    return ((N + 1) & N) == 0 && N + 1 <= 32;
}

// The pressure sums handed over unscaled through two more shared-memory
// planes (the 2g h plane's slot, F_B2, and one after the hand-over planes,
// F_B3) and scaled once per node after the eta-line (2 FP64 instructions per
// node fewer), where that staging admits as many 128-thread blocks per SM as
// the one with 2g h, or at least three (12 warps, the N = 7 kernel's), and
// the 256-thread shape still fits the 227 KB a block may use: N = 2, 4, 5, 6,
// 8, 9, 10 (measured: -0.7 to -2.6% of the kernel, also where a block per SM
// is lost: N = 4 and 5 gain from the registers the lower count allows).
// Decided per degree, not per launch shape, so that every shape computes the
// same bits.
enum { F_B2 = F_P, F_B3 = F_COUNT };
template <int N>
constexpr bool vol_bhand() {
    if constexpr (!vol_pressure_sums<N>() || vol_shfl<N>()) {
        return false;
    } else {
        constexpr size_t plane = sizeof(double) * (size_t)vol_ne<N, 128>() * (N + 1) * (N + 1);
        constexpr size_t wide = sizeof(double) * (size_t)vol_ne<N, 256>() * (N + 1) * (N + 1);
        constexpr size_t blocks = (228 * 1024) / ((F_COUNT + 1) * plane + 1024);
        return (blocks == (228 * 1024) / (F_COUNT * plane + 1024) || blocks >= 3) &&
               (F_COUNT + 1) * wide <= 227 * 1024;
    }
}

// The pressure sums run through both lines unscaled (started from the
// source in the xi-line) and are scaled by 2g h once per node.
template <int N>
constexpr bool vol_unscaled() {
    return vol_pressure_sums<N>() && (vol_shfl<N>() || vol_bhand<N>());
}

// The 2g h plane: where the pairs form the pressure, or where the sums are
// scaled once per line.
template <int N>
constexpr bool vol_has_p() {
    return !vol_pressure_sums<N>() || !vol_unscaled<N>();
}

// Shared-memory planes: the staged state, 2g h (vol_has_p), and the
// hand-over planes where the hand-over goes through shared memory (with
// the two pressure-sum planes for vol_bhand).
template <int N>
constexpr int vol_planes() {
    return vol_shfl<N>() ? (vol_has_p<N>() ? (int)F_P + 1 : (int)F_P)
                         : (vol_bhand<N>() ? (int)F_COUNT + 1 : (int)F_COUNT);
}

template <int N, bool AV, int TPB>
constexpr size_t vol_smem() {
    return sizeof(double) * ((size_t)vol_planes<N>() * vol_ne<N, TPB>() * (N + 1) * (N + 1));
}

// Shapes whose staging exceeds the 227 KB of shared memory a block may use
// are not built (the 128-thread shape fits every degree).
template <int N, bool AV, int TPB>
constexpr bool vol_fits() {
    return vol_smem<N, AV, TPB>() <= 227 * 1024;
}

// Blocks per SM passed to __launch_bounds__: the count that the staging of
// the shared-memory hand-over (all F_COUNT planes, one more with vol_bhand;
// 228 KB per SM, 1 KB reserved per block) admits, so that the register
// allocation does not lower the occupancy below it. The shuffle variants
// stage fewer planes but keep this bound and with it the registers of the
// pair loops (168 a thread at N = 7; capping them to the blocks the smaller
// staging admits spills).
template <int N, bool AV, int TPB>
constexpr int vol_min_blocks() {
    constexpr int threads = vol_ne<N, TPB>() * (N + 1);
    constexpr int warps = (threads + 31) / 32;
    constexpr size_t full =
        sizeof(double) * ((size_t)(vol_bhand<N>() ? F_COUNT + 1 : F_COUNT) * vol_ne<N, TPB>() * (N + 1) * (N + 1));
    constexpr int by_smem = (int)((228 * 1024) / (full + 1024));
    constexpr int by_warps = 64 / warps;
    constexpr int b = by_smem < by_warps ? by_smem : by_warps;
    return b > 0 ? b : 1;
}

// In-place transpose across the n lanes l = 0..n-1 of an element (n a power
// of two, the lanes consecutive and aligned within the warp): lane l holds
// row l of an n x n array on entry and column l on return. For each bit M of
// the lane index, lanes l and l^M exchange the entries whose index differs
// from the lane's in bit M; after all bits, entry p of lane l came from
// entry l of lane p. Every lane of the warp must take part.
template <int n>
__device__ __forceinline__ void lane_transpose(double (&x)[n], int l) {
#pragma unroll
    for (int M = n / 2; M >= 1; M /= 2) {
        const bool hi = (l & M) != 0;
#pragma unroll
        for (int p = 0; p < n; ++p) {
            if (p & M) continue;
            const double send = hi ? x[p] : x[p | M];
            const double r = __shfl_xor_sync(0xffffffffu, send, M);
            if (hi) x[p] = r;
            else x[p | M] = r;
        }
    }
}

template <int N>
__host__ __device__ constexpr int pair_index(int i, int q) {
    return i * (N + 1) - i * (i + 1) / 2 + (q - i - 1);
}

// All pairs of one line: nodes base + p*stride, p = 0..N; the (Sx, Sy) pair
// constants of the thread's line at pmk[2 * pair * (N+1)] (16-byte aligned).
// Accumulates A1 += +-Q and the partner-velocity parts of the momenta (the
// own-velocity parts u A1, v A1 are added once per node by the caller).
template <int N, int BLK>
__device__ __forceinline__ void pair_loop(const double* __restrict__ s, int base, int stride,
                                          const double* __restrict__ pmk, double* A1, double* A2,
                                          double* A3, double* B2, double* B3) {
    constexpr int n = N + 1;
    const double* sH = s + F_H * BLK;
    const double* sHU = s + F_HU * BLK;
    const double* sHV = s + F_HV * BLK;
    const double* sU = s + F_U * BLK;
    const double* sV = s + F_V * BLK;
    const double* sP = s + F_P * BLK;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const int ni = base + i * stride;
        const double hu_i = sHU[ni], hv_i = sHV[ni], u_i = sU[ni], v_i = sV[ni];
        const double h_i = sH[ni];
        // 2g h_i for the per-pair pressure (degrees without the pressure
        // sums; with them the plane may be absent, as at N = 7)
        double p_i = 0.0;
        if constexpr (!vol_pressure_sums<N>()) p_i = sP[ni];
#pragma unroll
        for (int q = i + 1; q < n; ++q) {
            const int nq = base + q * stride;
            const int pr = pair_index<N>(i, q);
            const double2 c = __ldg(reinterpret_cast<const double2*>(pmk + 2 * pr * n));
            const double Q = fma(hu_i + sHU[nq], c.x, (hv_i + sHV[nq]) * c.y);
            A1[i] += Q;
            A1[q] -= Q;
            if constexpr (vol_pressure_sums<N>()) {
                // P Sx = p_i (h_q Sx) at node i and p_q (-h_i Sx) at node q:
                // the sums of h Sx, h Sy are scaled by the node's p = 2g h
                // once per line (B2, B3), one product per pair fewer
                const double h_q = sH[nq];
                A2[i] = fma(sU[nq], Q, A2[i]);
                A2[q] = fma(-u_i, Q, A2[q]);
                A3[i] = fma(sV[nq], Q, A3[i]);
                A3[q] = fma(-v_i, Q, A3[q]);
                B2[i] = fma(h_q, c.x, B2[i]);
                B2[q] = fma(-h_i, c.x, B2[q]);
                B3[i] = fma(h_q, c.y, B3[i]);
                B3[q] = fma(-h_i, c.y, B3[q]);
            } else {
                const double P = p_i * sH[nq];
                A2[i] = fma(P, c.x, fma(sU[nq], Q, A2[i]));
                A2[q] = fma(-P, c.x, fma(-u_i, Q, A2[q]));
                A3[i] = fma(P, c.y, fma(sV[nq], Q, A3[i]));
                A3[q] = fma(-P, c.y, fma(-v_i, Q, A3[q]));
            }
        }
    }
}

template <int N, bool AV, int TPB>
__global__ void __launch_bounds__(vol_ne<N, TPB>() * (N + 1), (vol_min_blocks<N, AV, TPB>()))
    k_volume(VolArgs a) {
    constexpr int n = N + 1, nn = n * n, NE = vol_ne<N, TPB>(), NT = NE * n, BLK = NE * nn;
    constexpr int NP = N * (N + 1) / 2;
    extern __shared__ double sm[];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    const int t = threadIdx.x;
    const long long k0 = (long long)blockIdx.x * NE;
    auto S = [&](int f) { return sm + f * BLK; };

    // ---- stage the block's elements ---------------------------------------
    const double g2 = 2.0 * m.g;
    for (int idx = t; idx < BLK; idx += NT) {
        const int e = idx / nn;
        const long long k = k0 + e;
        double h = 0, hu = 0, hv = 0, u = 0, v = 0;
        if (k < m.K) {
            const long long gid = k * nn + (idx - e * nn);
            h = a.W[gid];
            hu = a.W[m.KN + gid];
            hv = a.W[2 * m.KN + gid];
            u = a.uv[gid];
            v = a.uv[m.KN + gid];
        }
        S(F_H)[idx] = h;
        S(F_HU)[idx] = hu;
        S(F_HV)[idx] = hv;
        S(F_U)[idx] = u;
        S(F_V)[idx] = v;
        if constexpr (vol_has_p<N>()) S(F_P)[idx] = g2 * h;
    }
    __syncthreads();

    const int e = t / n, l = t - e * n;
    const long long k = k0 + e;
    const bool valid = k < m.K;
    const double* pmx = m.pm + ((size_t)(valid ? k : 0) * 2 * NP * n + l) * 2;
    const double* pme = pmx + (size_t)NP * n * 2;
    const long long KS = m.KS;
    const long long side = (valid ? k : 0) * 4 * n;
    const double ek = (AV && valid) ? a.eps[k] : 0.0;
    const bool visc = ek > 0.0;
    // a viscous interface flux crosses side f only where the element or its
    // face-f neighbour is viscous (bit f of the mask); elsewhere the viscous
    // lift is exactly zero and is skipped without reading the slot
    const unsigned tmask = (AV && valid) ? a.touch[k] : 0u;
    const bool touch = tmask != 0u;
    double A1[n], A2[n], A3[n], B2[n], B3[n];

    // ---- xi-line j = l ----------------------------------------------------
#pragma unroll
    for (int p = 0; p < n; ++p) A1[p] = A2[p] = A3[p] = B2[p] = B3[p] = 0.0;
    if (valid) {
        if constexpr (vol_unscaled<N>()) {
            // the pressure sums start from the source (see the eta-line)
            // and run through both lines before they are scaled
#pragma unroll
            for (int p = 0; p < n; ++p) {
                B2[p] = m.ssx[k * nn + l * n + p];
                B3[p] = m.ssy[k * nn + l * n + p];
            }
        }
        pair_loop<N, BLK>(sm, e * nn + l * n, 1, pmx, A1, A2, A3, B2, B3);
        if constexpr (vol_pressure_sums<N>() && !vol_unscaled<N>()) {
            // the pressure parts P Sx = 2g h_i h_q Sx: the node's 2g h times its sums
#pragma unroll
            for (int p = 0; p < n; ++p) {
                const double pp = S(F_P)[e * nn + l * n + p];
                A2[p] = fma(pp, B2[p], A2[p]);
                A3[p] = fma(pp, B3[p], A3[p]);
                B2[p] = B3[p] = 0.0;
            }
        }
        // Lifts at the row's end nodes i = N (side 1) and i = 0 (side 3),
        // weighted by the tangential LGL weight w_l: done here, where every
        // lane holds one of them, rather than in the column phase where only
        // two lanes of eight would. A1 still holds sum Q there (doubled and
        // multiplied by u, v later), so it gets half the mass lift and the
        // momenta get -u, -v times that half in advance.
        const double wl = wq<N>(l), wlh = 0.5 * wl;
        const long long gid0 = k * nn + l * n;
#pragma unroll
        for (int end = 0; end < 2; ++end) {
            const int p = end == 0 ? N : 0, f = end == 0 ? 1 : 3;
            const long long sl = side + f * n + l;
            const int nd = e * nn + l * n + p;
            const double t1 = wlh * a.Fout[sl];
            A1[p] += t1;
            A2[p] = fma(-S(F_U)[nd], t1, fma(wl, a.Fout[KS + sl], A2[p]));
            A3[p] = fma(-S(F_V)[nd], t1, fma(wl, a.Fout[2 * KS + sl], A3[p]));
            if (AV && ((tmask >> f) & 1u)) {
                // viscous lift -w_l (F^v*_out - own outward flux) where a
                // viscous flux crosses the side
                const double fv2 = a.Fvout[sl], fv3 = a.Fvout[KS + sl];
                const double sg = end == 0 ? 1.0 : -1.0;
                const double own2 = visc ? sg * a.Fvt[gid0 + p] : 0.0;
                const double own3 = visc ? sg * a.Fvt[m.KN + gid0 + p] : 0.0;
                A2[p] = fma(-wl, fv2 - own2, A2[p]);
                A3[p] = fma(-wl, fv3 - own3, A3[p]);
            }
        }
    }
    if constexpr (vol_shfl<N>()) {
        // row l -> column l of the element, on every lane of the warp
        lane_transpose<n>(A1, l);
        lane_transpose<n>(A2, l);
        lane_transpose<n>(A3, l);
        if constexpr (vol_pressure_sums<N>()) {
            lane_transpose<n>(B2, l);
            lane_transpose<n>(B3, l);
        }
    } else {
#pragma unroll
        for (int p = 0; p < n; ++p) {
            S(F_A1)[e * nn + l * n + p] = A1[p];
            S(F_A2)[e * nn + l * n + p] = A2[p];
            S(F_A3)[e * nn + l * n + p] = A3[p];
            if constexpr (vol_bhand<N>()) {
                S(F_B2)[e * nn + l * n + p] = B2[p];
                S(F_B3)[e * nn + l * n + p] = B3[p];
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < n; ++p) {
            A1[p] = S(F_A1)[e * nn + p * n + l];
            A2[p] = S(F_A2)[e * nn + p * n + l];
            A3[p] = S(F_A3)[e * nn + p * n + l];
            if constexpr (vol_bhand<N>()) {
                B2[p] = S(F_B2)[e * nn + p * n + l];
                B3[p] = S(F_B3)[e * nn + p * n + l];
            }
        }
    }

    // ---- eta-line i = l, starting from the xi results ----------------------
    if (valid) {
        if constexpr (vol_pressure_sums<N>() && !vol_unscaled<N>()) {
            // the eta-line pressure sums start from the source: 2g h ssx
            // scaled by f is the source term h srcx of the node
#pragma unroll
            for (int p = 0; p < n; ++p) {
                B2[p] = m.ssx[k * nn + p * n + l];
                B3[p] = m.ssy[k * nn + p * n + l];
            }
        }
        pair_loop<N, BLK>(sm, e * nn + l, n, pme, A1, A2, A3, B2, B3);
        if constexpr (vol_pressure_sums<N>()) {
#pragma unroll
            for (int p = 0; p < n; ++p) {
                double pp;  // 2g h of the node
                if constexpr (vol_has_p<N>()) pp = S(F_P)[e * nn + p * n + l];
                else pp = g2 * S(F_H)[e * nn + p * n + l];
                A2[p] = fma(pp, B2[p], A2[p]);
                A3[p] = fma(pp, B3[p], A3[p]);
            }
        }
    }
    // own-velocity parts of the momentum fluxes; A1 keeps sum Q (half the
    // mass flux difference): the mass row is scaled by 2f = -2/(w_i w_j J) at
    // the end and its remaining lifts take half weights, which gives f (2 A1 +
    // w F) bit for bit without forming 2 A1
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const int nd = e * nn + p * n + l;
        A2[p] = fma(S(F_U)[nd], A1[p], A2[p]);
        A3[p] = fma(S(F_V)[nd], A1[p], A3[p]);
    }

    if (!valid) return;

    // ---- nodes (i = l, j = p): lifts, viscous terms, source, scaling --------
    const int i = l;
    const double wi = wq<N>(i), wih = 0.5 * wi;
#pragma unroll
    for (int p = 0; p < n; ++p) {
        const int j = p;
        const long long gid = k * nn + j * n + i;
        double a1 = A1[p], a2 = A2[p], a3 = A3[p];
        // interface flux: w_i w_j (1/w_0) F_out = (tangential weight) F_out
        // (half of it in the mass row, which is scaled by 2f)
        auto lift = [&](int f, int pn) {
            const long long sl = side + f * n + pn;
            a1 = fma(wih, a.Fout[sl], a1);
            a2 = fma(wi, a.Fout[KS + sl], a2);
            a3 = fma(wi, a.Fout[2 * KS + sl], a3);
        };
        if (j == 0) lift(0, i);
        if (j == N) lift(2, i);
        if (AV && touch) {
            if (visc) {
                // the volume part of the viscous divergence (AV kernel)
                const double wij = wi * wq<N>(j);
                a2 = fma(-wij, a.Lv[gid], a2);
                a3 = fma(-wij, a.Lv[m.KN + gid], a3);
            }
            // viscous lift at sides 0 and 2: -(tangential weight) (F^v*_out -
            // own outward flux), where a viscous flux crosses the side
            auto vlift = [&](int f, double sg) {
                const long long sl = side + f * n + i;
                if ((tmask >> f) & 1u) {
                    const double fv2 = a.Fvout[sl], fv3 = a.Fvout[KS + sl];
                    const double own2 = visc ? sg * a.Fvt[2 * m.KN + gid] : 0.0;
                    const double own3 = visc ? sg * a.Fvt[3 * m.KN + gid] : 0.0;
                    a2 = fma(-wi, fv2 - own2, a2);
                    a3 = fma(-wi, fv3 - own3, a3);
                }
            };
            if (j == 0) vlift(0, -1.0);
            if (j == N) vlift(2, 1.0);
        }
        const double f = m.fwJ[gid];
        a.R[gid] = m.fwJ2[gid] * a1;
        if constexpr (vol_pressure_sums<N>()) {
            // the source is in the pressure sums
            a.R[m.KN + gid] = f * a2;
            a.R[2 * m.KN + gid] = f * a3;
        } else {
            const double h = S(F_H)[e * nn + j * n + i];
            a.R[m.KN + gid] = fma(h, m.srcx[gid], f * a2);
            a.R[2 * m.KN + gid] = fma(h, m.srcy[gid], f * a3);
        }
    }
}

// N = 1: one thread per element. With 4 nodes an element's line holds one
// pair, too little work between the line kernel's staging and hand-over
// barriers to keep the FP64 pipe busy (measured: 7% faster than the line
// kernel at N = 1; at N = 2, with three pairs a line and 166 registers, 5%
// slower, so N >= 2 keeps the line kernel). Here a
// thread holds its whole element in registers (state, velocities, the three
// accumulators), runs the pairs of all its xi- and eta-lines back to back,
// then adds the own-velocity parts, the interface lifts (tangential weight
// times F_out, every side), the viscous terms and the source, and scales by
// -1/(w_i w_j J): no shared memory and no barriers. The arithmetic of a pair
// is the line kernel's with pressure sums (14 FP64 instructions; the sums of
// both lines start from the source and are scaled by 2g h once per node, the
// mass row by the stored 2f); the block size (TPB elements) is the launch
// shape, with the same instructions for every shape.
template <int N>
constexpr bool vol_ept() {
    return N <= 1;
}

template <int N>
__device__ __forceinline__ int side_node(int f, int p) {
    return f == 0 ? p : (f == 1 ? p * (N + 1) + N : (f == 2 ? N * (N + 1) + p : p * (N + 1)));
}

template <int N, bool AV, int TPB>
__global__ void __launch_bounds__(TPB) k_volume_ept(VolArgs a) {
    static_assert(pressure_sums_degree(N), "the element-per-thread kernel starts its pressure sums from ssx");
    constexpr int n = N + 1, nn = n * n, NP = N * (N + 1) / 2;
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    const long long k = (long long)blockIdx.x * TPB + threadIdx.x;
    if (k >= m.K) return;
    const long long g0 = k * nn;
    const double g2 = 2.0 * m.g;
    // B2, B3: the pressure sums sum_q h_q Sx, h_q Sy of both lines of a node,
    // started from the bathymetry source w_i w_j gamma / 4 and scaled by the
    // node's 2g h once, after all pairs (the line kernel's pressure sums)
    double h[nn], hu[nn], hv[nn], u[nn], v[nn], A1[nn], A2[nn], A3[nn], B2[nn], B3[nn];
#pragma unroll
    for (int d = 0; d < nn; ++d) {
        h[d] = a.W[g0 + d];
        hu[d] = a.W[m.KN + g0 + d];
        hv[d] = a.W[2 * m.KN + g0 + d];
        u[d] = a.uv[g0 + d];
        v[d] = a.uv[m.KN + g0 + d];
        A1[d] = A2[d] = A3[d] = 0.0;
        B2[d] = m.ssx[g0 + d];
        B3[d] = m.ssy[g0 + d];
    }
    // pair constants of the element: [direction][pair][line][2]
    const double* pm = m.pm + (size_t)k * 4 * NP * n;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
            for (int i = 0; i < n; ++i) {
#pragma unroll
                for (int q = i + 1; q < n; ++q) {
                    const int ni = dir == 0 ? l * n + i : i * n + l;
                    const int nq = dir == 0 ? l * n + q : q * n + l;
                    const int pr = pair_index<N>(i, q);
                    const double2 c =
                        __ldg(reinterpret_cast<const double2*>(pm + 2 * ((dir * NP + pr) * n + l)));
                    const double Q = fma(hu[ni] + hu[nq], c.x, (hv[ni] + hv[nq]) * c.y);
                    A1[ni] += Q;
                    A1[nq] -= Q;
                    A2[ni] = fma(u[nq], Q, A2[ni]);
                    A2[nq] = fma(-u[ni], Q, A2[nq]);
                    A3[ni] = fma(v[nq], Q, A3[ni]);
                    A3[nq] = fma(-v[ni], Q, A3[nq]);
                    B2[ni] = fma(h[nq], c.x, B2[ni]);
                    B2[nq] = fma(-h[ni], c.x, B2[nq]);
                    B3[ni] = fma(h[nq], c.y, B3[ni]);
                    B3[nq] = fma(-h[ni], c.y, B3[nq]);
                }
            }
        }
    }
    // pressure parts (with the source) and own-velocity parts of the momentum
    // fluxes; A1 keeps sum Q (half the mass flux difference): the mass row is
    // scaled by 2f and its lifts take half weights (bit for bit f (2 A1 + w F))
#pragma unroll
    for (int d = 0; d < nn; ++d) {
        const double pp = g2 * h[d];
        A2[d] = fma(pp, B2[d], A2[d]);
        A3[d] = fma(pp, B3[d], A3[d]);
        A2[d] = fma(u[d], A1[d], A2[d]);
        A3[d] = fma(v[d], A1[d], A3[d]);
    }
    // interface flux: w_i w_j (1/w_0) F_out = (tangential weight) F_out
    const long long side = k * 4 * n;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int p = 0; p < n; ++p) {
            const int d = side_node<N>(f, p);
            const long long sl = side + f * n + p;
            const double wt = wq<N>(p);
            A1[d] = fma(0.5 * wt, a.Fout[sl], A1[d]);
            A2[d] = fma(wt, a.Fout[m.KS + sl], A2[d]);
            A3[d] = fma(wt, a.Fout[2 * m.KS + sl], A3[d]);
        }
    }
    const bool visc = AV && a.eps[k] > 0.0;
    const unsigned tmask = AV ? a.touch[k] : 0u;
    if (AV && tmask != 0u) {
        if (visc) {
            // the volume part of the viscous divergence (AV kernel)
#pragma unroll
            for (int j = 0; j < n; ++j) {
#pragma unroll
                for (int i = 0; i < n; ++i) {
                    const double wij = wq<N>(i) * wq<N>(j);
                    A2[j * n + i] = fma(-wij, a.Lv[g0 + j * n + i], A2[j * n + i]);
                    A3[j * n + i] = fma(-wij, a.Lv[m.KN + g0 + j * n + i], A3[j * n + i]);
                }
            }
        }
        // viscous lifts -(tangential weight) (F^v*_out - own outward flux)
        // where a viscous flux crosses the side
#pragma unroll
        for (int f = 0; f < 4; ++f) {
#pragma unroll
            for (int p = 0; p < n; ++p) {
                const int d = side_node<N>(f, p);
                const long long sl = side + f * n + p;
                if ((tmask >> f) & 1u) {
                    const double fv2 = a.Fvout[sl], fv3 = a.Fvout[m.KS + sl];
                    const double sg = (f == 1 || f == 2) ? 1.0 : -1.0;
                    const long long pl = (f == 1 || f == 3) ? 0 : 2 * m.KN;  // F~v on xi sides, G~v on eta sides
                    const double own2 = visc ? sg * a.Fvt[pl + g0 + d] : 0.0;
                    const double own3 = visc ? sg * a.Fvt[pl + m.KN + g0 + d] : 0.0;
                    const double wt = wq<N>(p);
                    A2[d] = fma(-wt, fv2 - own2, A2[d]);
                    A3[d] = fma(-wt, fv3 - own3, A3[d]);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < nn; ++d) {
        const long long gid = g0 + d;
        const double f = m.fwJ[gid];
        a.R[gid] = m.fwJ2[gid] * A1[d];
        a.R[m.KN + gid] = f * A2[d];
        a.R[2 * m.KN + gid] = f * A3[d];
    }
}

// Opt in to the kernel's shared memory once per process (before any stream
// capture: contexts call it at creation).
template <int N, bool AV, int TPB>
void set_attr() {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_volume<N, AV, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)vol_smem<N, AV, TPB>());
        attr = true;
    }
}

template <int N, bool AV, int TPB>
bool launch_n(swe_ctx* c, const VolArgs& a, cudaStream_t s) {
    if constexpr (vol_ept<N>()) {
        Timed tm(c, KC_VOLUME, s);
        k_volume_ept<N, AV, TPB><<<grid_for(c->m.K, TPB), TPB, 0, s>>>(a);
        return true;
    } else if constexpr (!vol_fits<N, AV, TPB>()) {
        return false;
    } else {
        constexpr int NE = vol_ne<N, TPB>();
        set_attr<N, AV, TPB>();
        const int blocks = grid_for(c->m.K, NE);
        Timed tm(c, KC_VOLUME, s);
        k_volume<N, AV, TPB><<<blocks, NE * (N + 1), vol_smem<N, AV, TPB>(), s>>>(a);
        return true;
    }
}

template <int N, int TPB>
bool prepare_n() {
    if constexpr (vol_ept<N>()) return true;
    if constexpr (vol_fits<N, true, TPB>()) set_attr<N, true, TPB>();
    if constexpr (vol_fits<N, false, TPB>()) set_attr<N, false, TPB>();
    return vol_fits<N, true, TPB>() && vol_fits<N, false, TPB>();
}

template <int TPB>
bool prepare_shape(int N) {
    switch (N) {
        case 1: return prepare_n<1, TPB>(); case 2: return prepare_n<2, TPB>();
        case 3: return prepare_n<3, TPB>(); case 4: return prepare_n<4, TPB>();
        case 5: return prepare_n<5, TPB>(); case 6: return prepare_n<6, TPB>();
        case 7: return prepare_n<7, TPB>(); case 8: return prepare_n<8, TPB>();
        case 9: return prepare_n<9, TPB>(); case 10: return prepare_n<10, TPB>();
        case 11: return prepare_n<11, TPB>(); case 12: return prepare_n<12, TPB>();
        default: return false;
    }
}

template <int TPB>
bool launch_shape(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop) {
    VolArgs a{c->m, W, c->w.uv, c->w.Fout, c->w.Fvt, c->w.Fvout, c->w.Lv, c->w.eps, c->w.touch, R, stop};
    const bool av = c->p.av != 0;
#define SWE_VOL_CASE(NN) \
    case NN: return av ? launch_n<NN, true, TPB>(c, a, s) : launch_n<NN, false, TPB>(c, a, s);
    switch (c->m.N) {
        SWE_VOL_CASE(1) SWE_VOL_CASE(2) SWE_VOL_CASE(3) SWE_VOL_CASE(4)
        SWE_VOL_CASE(5) SWE_VOL_CASE(6) SWE_VOL_CASE(7) SWE_VOL_CASE(8)
        SWE_VOL_CASE(9) SWE_VOL_CASE(10) SWE_VOL_CASE(11) SWE_VOL_CASE(12)
        default: return false;
    }
#undef SWE_VOL_CASE
}

}  // namespace
}  // namespace swe

// Exported entry points of the translation unit of one launch shape.
#define SWE_VOLUME_SHAPE(TPB)                                                                        \
    namespace swe {                                                                                  \
    void volume_init_##TPB() { upload_tables(); }                                                    \
    bool volume_prepare_##TPB(int N) { return prepare_shape<TPB>(N); }                                 \
    bool volume_launch_##TPB(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop) { \
        return launch_shape<TPB>(c, W, R, s, stop);                                                  \
    }                                                                                                \
    }
