// Standard (non-split) volume kernel: the volume integral of Eq. VolInt
// (second line) in strong form, sum_q D_iq F~_qj + sum_q D_jq G~_iq with the
// nodal contravariant fluxes F~ = y_eta f - x_eta g, G~ = -y_xi f + x_xi g of
// the physical fluxes, the interface lift (F* - F~_own) at face nodes, the
// BR1 viscous divergence of Eq. ViscTermsDisc, the non-split source
// -g h J grad b and the scaling by 1/J. This is the scheme the paper
// compares the split form against; it is neither entropy stable nor well
// balanced.
//
// Design: blocks of 128 threads own NE = 512/(N+1)^2 elements and loop over
// their nodes, so that every warp is full whatever (N+1)^2 is (an FP64 warp
// instruction costs the same with any number of active lanes). The block
// stages the contravariant fluxes of its elements in shared memory (6
// planes, 4 more for the viscous fluxes), then every node applies its row of
// D along both lines: 6(N+1) fused multiply-adds per node against the N pair
// evaluations of the split form.
// With Q = a.(hu, hv) and p = g h^2/2 the contravariant fluxes are
// (Q, u Q + a_x p, v Q + a_y p) for the direction vector a, 14 FP64
// instructions for both directions. The own-flux part of the lift,
// -F~_own/w at the face nodes, is folded into the diagonal of the staged
// matrix (D_00 + 1/w_0, D_NN - 1/w_N), so a face node only adds
// F_out/w_0, and the result is -(L - L^v)/J + h (source coefficient).
#include "kcommon.cuh"

namespace swe {
namespace {

struct StdArgs {
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

enum { P_F1, P_F2, P_F3, P_G1, P_G2, P_G3, P_FLUX, P_VF2 = P_FLUX, P_VF3, P_VG2, P_VG3, P_ALL };

constexpr int STD_THREADS = 128;

template <int N>
constexpr int std_ne() {
    return (N + 1) * (N + 1) >= 512 ? 1 : 512 / ((N + 1) * (N + 1));
}

// Staging planes, then D' (and the plain D for the viscous divergence).
template <int N, bool AV>
constexpr size_t std_smem() {
    return sizeof(double) *
           ((size_t)(AV ? P_ALL : P_FLUX) * std_ne<N>() * (N + 1) * (N + 1) + (AV ? 2 : 1) * (N + 1) * (N + 1));
}

template <int N, bool AV>
__global__ void __launch_bounds__(STD_THREADS) k_volume_std(StdArgs a) {
    constexpr int n = N + 1, nn = n * n, NE = std_ne<N>(), BLK = NE * nn;
    extern __shared__ double sm[];
    if (stopped(a.stop)) return;
    const DeviceMesh& m = a.m;
    const long long k0 = (long long)blockIdx.x * NE;
    auto P = [&](int f) { return sm + f * BLK; };
    double* sD = sm + (AV ? P_ALL : P_FLUX) * BLK;
    double* sDv = sD + nn;  // plain D (AV only)
    constexpr double rw0 = N * (N + 1) / 2.0;  // 1/w_0 = 1/w_N, the LGL end weight
    for (int idx = threadIdx.x; idx < nn; idx += STD_THREADS) {
        const int row = idx / n, col = idx % n;
        const double d = Dm<N>(row, col);
        if (AV) sDv[idx] = d;
        sD[idx] = (row == col && row == 0) ? d + rw0 : (row == col && row == N) ? d - rw0 : d;
    }
    // ---- contravariant fluxes of the block's nodes ----------------------------
    for (int t = threadIdx.x; t < BLK; t += STD_THREADS) {
        const int e = t / nn, r = t - e * nn;
        const long long k = k0 + e;
        double Ft[3] = {0.0, 0.0, 0.0}, Gt[3] = {0.0, 0.0, 0.0};
        if (k < m.K) {
            const long long gid = k * nn + r;
            const double h = a.W[gid], hu = a.W[m.KN + gid], hv = a.W[2 * m.KN + gid];
            const double u = a.uv[gid], v = a.uv[m.KN + gid];
            const double p = (0.5 * m.g * h) * h;
            const double axx = m.axx[gid], axy = m.axy[gid], aex = m.aex[gid], aey = m.aey[gid];
            const double Q = fma(axx, hu, axy * hv), Qe = fma(aex, hu, aey * hv);
            Ft[0] = Q;
            Ft[1] = fma(u, Q, axx * p);
            Ft[2] = fma(v, Q, axy * p);
            Gt[0] = Qe;
            Gt[1] = fma(u, Qe, aex * p);
            Gt[2] = fma(v, Qe, aey * p);
            if (AV && a.eps[k] > 0.0) {
                P(P_VF2)[t] = a.Fvt[gid];
                P(P_VF3)[t] = a.Fvt[m.KN + gid];
                P(P_VG2)[t] = a.Fvt[2 * m.KN + gid];
                P(P_VG3)[t] = a.Fvt[3 * m.KN + gid];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P(P_F1 + c)[t] = Ft[c];
            P(P_G1 + c)[t] = Gt[c];
        }
    }
    __syncthreads();

    // ---- D' along the xi-line and the eta-line of every node -----------------
    const long long KS = m.KS;
    for (int t = threadIdx.x; t < BLK; t += STD_THREADS) {
        const int e = t / nn, r = t - e * nn, i = r % n, j = r / n;
        const long long k = k0 + e;
        if (k >= m.K) break;  // the remaining nodes of the block are past the mesh too
        const long long gid = k * nn + r;
        const int eb = e * nn;
        double L[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < n; ++q) {
            const double di = sD[i * n + q], dj = sD[j * n + q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                L[c] = fma(di, P(P_F1 + c)[eb + j * n + q], L[c]);
                L[c] = fma(dj, P(P_G1 + c)[eb + q * n + i], L[c]);
            }
        }
        // interface flux: + F_out / w_0 at the face nodes
        const long long side = k * 4 * n;
        auto lift = [&](int f, int pn) {
            const long long sl = side + f * n + pn;
#pragma unroll
            for (int c = 0; c < 3; ++c) L[c] = fma(rw0, a.Fout[c * KS + sl], L[c]);
        };
        if (j == 0) lift(0, i);
        if (j == N) lift(2, i);
        if (i == N) lift(1, j);
        if (i == 0) lift(3, j);
        if (AV && a.eps[k] > 0.0) {
            double L2 = 0.0, L3 = 0.0;
#pragma unroll
            for (int q = 0; q < n; ++q) {
                const double di = sDv[i * n + q], dj = sDv[j * n + q];
                L2 = fma(di, P(P_VF2)[eb + j * n + q], L2);
                L3 = fma(di, P(P_VF3)[eb + j * n + q], L3);
                L2 = fma(dj, P(P_VG2)[eb + q * n + i], L2);
                L3 = fma(dj, P(P_VG3)[eb + q * n + i], L3);
            }
            L[1] -= L2;
            L[2] -= L3;
            const double ft2 = P(P_VF2)[t], ft3 = P(P_VF3)[t], gt2 = P(P_VG2)[t], gt3 = P(P_VG3)[t];
            // viscous lift: -(1/w_0) (F^v*_out - own outward viscous flux)
            auto vlift = [&](int f, int pn, double own2, double own3) {
                const long long sl = side + f * n + pn;
                L[1] = fma(-rw0, a.Fvout[sl] - own2, L[1]);
                L[2] = fma(-rw0, a.Fvout[KS + sl] - own3, L[2]);
            };
            if (j == 0) vlift(0, i, -gt2, -gt3);
            if (j == N) vlift(2, i, gt2, gt3);
            if (i == N) vlift(1, j, ft2, ft3);
            if (i == 0) vlift(3, j, -ft2, -ft3);
        }
        const double h = a.W[gid];
        const double mrJ = -m.rJ[gid];
        a.R[gid] = mrJ * L[0];
        a.R[m.KN + gid] = fma(h, m.srcx[gid], mrJ * L[1]);
        a.R[2 * m.KN + gid] = fma(h, m.srcy[gid], mrJ * L[2]);
    }
}

template <int N, bool AV>
void launch_n(swe_ctx* c, const StdArgs& a, cudaStream_t s) {
    constexpr int NE = std_ne<N>();
    static_assert(std_smem<N, AV>() <= 48 * 1024, "standard volume staging fits the default shared memory");
    Timed tm(c, KC_VOLUME, s);
    k_volume_std<N, AV><<<grid_for(c->m.K, NE), STD_THREADS, std_smem<N, AV>(), s>>>(a);
}

}  // namespace

void init_tables_volume_std() { upload_tables(); }

void launch_volume_std(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop) {
    StdArgs a{c->m, W, c->w.uv, c->w.Fout, c->w.Fvt, c->w.Fvout, c->w.eps, R, stop};
    const bool av = c->p.av != 0;
#define SWE_STD_CASE(NN)                         \
    case NN:                                     \
        if (av) launch_n<NN, true>(c, a, s);     \
        else launch_n<NN, false>(c, a, s);       \
        break;
    switch (c->m.N) {
        SWE_STD_CASE(1) SWE_STD_CASE(2) SWE_STD_CASE(3) SWE_STD_CASE(4)
        SWE_STD_CASE(5) SWE_STD_CASE(6) SWE_STD_CASE(7) SWE_STD_CASE(8)
        SWE_STD_CASE(9) SWE_STD_CASE(10) SWE_STD_CASE(11) SWE_STD_CASE(12)
        default: break;
    }
#undef SWE_STD_CASE
}

}  // namespace swe
