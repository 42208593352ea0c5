// Node-, face- and element-wise kernels other than the volume term:
// primitives, the entropy-stable interface flux, the BR1 viscous interface
// average, the fused Runge-Kutta stage update with the positivity limiter,
// the time-step reduction and the diagnostic integrals.
#include <math.h>

#include "kcommon.cuh"

namespace swe {
namespace {

// ---------------------------------------------------------------------------
// Primitive velocities u = hu/h, v = hv/h (zero where h <= 0): one reciprocal
// per node, reused by every later kernel of the stage.
// ---------------------------------------------------------------------------
__global__ void k_prim(long long KN, const double* __restrict__ W, double* __restrict__ uv,
                       const int* stop) {
    if (stopped(stop)) return;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < KN;
         id += (long long)gridDim.x * blockDim.x) {
        double u, v;
        velocities(W[id], W[KN + id], W[2 * KN + id], u, v);
        uv[id] = u;
        uv[KN + id] = v;
    }
}

// ---------------------------------------------------------------------------
// Interface flux through the owner's outward normal at every unique face
// node (Eq. NumericalSurfaceFlux evaluated in the normal frame, App. B):
// rotate the velocities (Eq. rotatingVelocities), EC flux of Eq.
// surfaceFluxes, minus 1/2 R~|Lambda~|R~^T [[q~]] (Eqs. fesandges,
// RightEigenvectors2DCurved, ScalingMatrix2DCurved), rotate back (Eq.
// surfaceFlux2DRotated), times the surface Jacobian. With [[a^2]] = 2{a}[[a]]
// the projection R~^T [[q~]] is (g[[h+b]] + {c}[[u~]], [[v~]],
// g[[h+b]] - {c}[[u~]]). Writes +F to the owner's side slot and -F to the
// neighbour's, and the BR1 interface values {u}, {v} to both.
// ---------------------------------------------------------------------------
// Eight times the flux in the normal frame, from sums and differences of the
// two sides: H = h- + h+, U = u~- + u~+, V = v~- + v~+ (twice the averages),
// du = [[u~]], dv = [[v~]], C = c- + c+ with c = sqrt(g max(h, 0)) (twice
// {c}) and f = H U (four times the EC mass flux {h}{u~}). With the
// dissipation's projections scaled by four,
//   S1 = |U + C| (C/(2g) du + [[h+b]]),   S3 = |U - C| (-C/(2g) du + [[h+b]]),
// D = S1 + S3 and r2g = 1/(2g), g2 = 2g:
//   8 F1 = 2f - D,
//   8 F2 = f U + g2 (h-^2 + h+^2) - (U D + C (S1 - S3))/2,
//   8 F3 = f V - V D/2 - |f| dv,
// the EC flux of Eq. surfaceFluxes minus 1/2 R~|Lambda~|R~^T [[q~]] with the
// averages written as half sums; the factor 8 is in the rotation back
// (the face planes hold the normals and surface Jacobians divided by 8, an
// exact scaling).
template <bool ES>
__device__ __forceinline__ void normal_flux8(double g, double g2, double r2g, double hm, double hp, double U,
                                             double V, double du, double dv, double bm, double bp, double& F1,
                                             double& F2, double& F3) {
    const double f = (hm + hp) * U;
    F2 = fma(f, U, g2 * fma(hm, hm, hp * hp));
    F3 = f * V;
    if (ES) {
        const double C = sqrt_pos(g * pos_part(hm)) + sqrt_pos(g * pos_part(hp));
        const double jH = (hp + bp) - (hm + bm);
        const double Cr = C * r2g;
        const double S1 = fabs(U + C) * fma(Cr, du, jH);
        const double S3 = fabs(U - C) * fma(-Cr, du, jH);
        const double D = S1 + S3;
        F1 = fma(2.0, f, -D);
        F2 = fma(-0.5, fma(U, D, C * (S1 - S3)), F2);
        F3 = fma(-fabs(f), dv, fma(-0.5 * V, D, F3));
    } else {
        F1 = 2.0 * f;
    }
}

// Interface flux through the owner's outward normal at every unique face
// node (Eq. NumericalSurfaceFlux evaluated in the normal frame, App. B):
// the velocity sums and jumps rotated into the frame (Eq.
// rotatingVelocities), the flux of normal_flux8, rotated back (Eq.
// surfaceFlux2DRotated) with the unscaled normal over 8, whose length is the
// surface Jacobian over 8. Writes +F to the owner's side slot and -F to the
// neighbour's, and the BR1 interface values {u}, {v} to both.
template <bool ES>
__global__ void k_surface(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv,
                          double* __restrict__ Fout, double* __restrict__ Ustar, const int* stop) {
    if (stopped(stop)) return;
    const long long total = (long long)m.nfaces * m.n;
    const double g = m.g, g2 = 2.0 * m.g;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long im = m.f_im[t], ip = m.f_ip[t], tm = m.f_tm[t], tp = m.f_tp[t];
        const double nx = m.f_nx[t], ny = m.f_ny[t];
        const double hm = W[im], hp = W[ip];
        const double um = uv[im], vm = uv[m.KN + im], up = uv[ip], vp = uv[m.KN + ip];
        const double su = um + up, sv = vm + vp, ju = up - um, jv = vp - vm;
        const double U = fma(nx, su, ny * sv), V = fma(nx, sv, -ny * su);
        const double du = fma(nx, ju, ny * jv), dv = fma(nx, jv, -ny * ju);
        double F1, F2, F3;
        normal_flux8<ES>(g, g2, m.r2g, hm, hp, U, V, du, dv, m.f_bm[t], m.f_bp[t], F1, F2, F3);
        const double sx = m.f_sx8[t], sy = m.f_sy8[t];
        const double G1 = m.f_js8[t] * F1;
        const double G2 = fma(sx, F2, -sy * F3);
        const double G3 = fma(sy, F2, sx * F3);
        Fout[tm] = G1;
        Fout[m.KS + tm] = G2;
        Fout[2 * m.KS + tm] = G3;
        Fout[tp] = negated(G1);
        Fout[m.KS + tp] = negated(G2);
        Fout[2 * m.KS + tp] = negated(G3);
        const double us = 0.5 * su, vs = 0.5 * sv;
        Ustar[tm] = us;
        Ustar[m.KS + tm] = vs;
        Ustar[tp] = us;
        Ustar[m.KS + tp] = vs;
    }
}

// Solid walls: the flux against the mirror state (same h and b, normal
// velocity reversed) to the own side slot only; BR1 takes the own velocity
// as U* (no gradient lift). The viscous interface flux of a wall slot is
// zero and is never written after creation.
template <bool ES>
__global__ void k_wall(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv,
                       double* __restrict__ Fout, double* __restrict__ Ustar, const int* stop) {
    if (stopped(stop)) return;
    const long long total = (long long)m.nwall * m.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long im = m.w_im[t], tm = m.w_tm[t];
        const double nx = m.w_nx[t], ny = m.w_ny[t], js = m.w_js[t];
        const double hm = W[im], um = uv[im], vm = uv[m.KN + im], bm = m.bn[im];
        const double utm = fma(nx, um, ny * vm), vtm = fma(nx, vm, -ny * um);
        // mirror state: U = 0, V = 2 v~, du = -2 u~, dv = 0
        double F1, F2, F3;
        normal_flux8<ES>(m.g, 2.0 * m.g, m.r2g, hm, hm, 0.0, 2.0 * vtm, -2.0 * utm, 0.0, bm, bm, F1, F2, F3);
        const double js8 = 0.125 * js;
        Fout[tm] = js8 * F1;
        Fout[m.KS + tm] = js8 * fma(nx, F2, -ny * F3);
        Fout[2 * m.KS + tm] = js8 * fma(ny, F2, nx * F3);
        Ustar[tm] = um;
        Ustar[m.KS + tm] = vm;
    }
}

// BR1 interface values alone (U* = {u}, V* = {v} on both sides of every
// face; the own value at solid walls), for callers that need them without
// the interface flux (the adjoint's recomputation of the forward quantities).
__global__ void k_ustar(DeviceMesh m, const double* __restrict__ uv, double* __restrict__ Ustar) {
    const long long total = (long long)m.nfaces * m.n, walls = (long long)m.nwall * m.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total + walls;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < total) {
            const long long im = m.f_im[t], ip = m.f_ip[t], tm = m.f_tm[t], tp = m.f_tp[t];
            const double us = 0.5 * (uv[im] + uv[ip]), vs = 0.5 * (uv[m.KN + im] + uv[m.KN + ip]);
            Ustar[tm] = us;
            Ustar[m.KS + tm] = vs;
            Ustar[tp] = us;
            Ustar[m.KS + tp] = vs;
        } else {
            const long long w = t - total, im = m.w_im[w], tm = m.w_tm[w];
            Ustar[tm] = uv[im];
            Ustar[m.KS + tm] = uv[m.KN + im];
        }
    }
}

// ---------------------------------------------------------------------------
// BR1 viscous interface flux {F^v . n} (Thm. 1) with the owner's unscaled
// outward normal; +avg to the owner's slot, -avg to the neighbour's. Only
// viscous elements (eps_k > 0) carry side-node viscous fluxes: the other
// side's traces count as zero and are not read.
// ---------------------------------------------------------------------------
//
// Only the faces of the viscous elements are visited (the list of the AV
// indicator kernel, one thread per side slot): every other face carries no
// viscous flux, and its slots (which may hold the values of an earlier
// state) are not read (below). A face between two viscous elements is
// evaluated by its owner's visit only.
//
// The same launch writes the side masks of the volume kernel, one pass over
// the elements: bit f of touch[k] is set where a viscous flux crosses side f
// of element k (k viscous, walls included, or its face-f neighbour viscous);
// the volume kernel reads the viscous interface flux of exactly those sides.
__global__ void k_visc_face(DeviceMesh m, const double* __restrict__ Fvtr, const double* __restrict__ eps,
                            const int* __restrict__ vlist, const int* __restrict__ vcount,
                            double* __restrict__ Fvout, uint32_t* __restrict__ touch, const int* stop) {
    if (stopped(stop)) return;
    const long long S = m.KS, sps = 4LL * m.n;  // side slots per element
    const long long nn = (long long)m.n * m.n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m.K;
         k += (long long)gridDim.x * blockDim.x) {
        const bool vk = nonzero(eps[k]);
        unsigned mask = 0u;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const long long nb = m.s_nb[k * sps + f * m.n];
            if (vk || (nb >= 0 && nonzero(eps[nb / nn]))) mask |= 1u << f;
        }
        touch[k] = mask;
    }
    const long long work = (long long)*vcount * sps;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < work;
         w += (long long)gridDim.x * blockDim.x) {
        const long long k = vlist[w / sps];
        const long long sl = k * sps + w % sps;
        const int t = m.s_face[sl];
        if (t < 0) continue;  // solid wall: no viscous flux, the slot stays zero
        const long long tm = m.f_tm[t], tp = m.f_tp[t];
        const bool vm = nonzero(eps[tm / sps]), vp = nonzero(eps[tp / sps]);
        if (sl == tp && vm) continue;  // the owner, viscous too, evaluates the face
        const double F2 = (vm ? Fvtr[tm] : 0.0) + (vp ? Fvtr[tp] : 0.0);
        const double F3 = (vm ? Fvtr[S + tm] : 0.0) + (vp ? Fvtr[S + tp] : 0.0);
        const double G2 = (vm ? Fvtr[2 * S + tm] : 0.0) + (vp ? Fvtr[2 * S + tp] : 0.0);
        const double G3 = (vm ? Fvtr[3 * S + tm] : 0.0) + (vp ? Fvtr[3 * S + tp] : 0.0);
        // (the unscaled normal over 8: 4 times it is half the normal, exactly)
        const double nx = m.f_sx8[t], ny = m.f_sy8[t];
        const double a2 = 4.0 * fma(nx, F2, ny * G2);
        const double a3 = 4.0 * fma(nx, F3, ny * G3);
        Fvout[tm] = a2;
        Fvout[S + tm] = a3;
        Fvout[tp] = negated(a2);
        Fvout[S + tp] = negated(a3);
    }
}

// ---------------------------------------------------------------------------
// Runge-Kutta stage update fused with the positivity limiter (Eq. PosPres),
// the h_tol momentum cut and the primitives of the next stage; one warp per
// element, deterministic butterfly reductions.
//   MODE 0: limiter only.
//   MODE 1: 2N-storage stage with the register kept divided by dt:
//           Kh = a Kh + R (Kh = R when a = 0), W = W + (b dt) Kh.
//   MODE 2: SSP stage W = a Wn + b (W + dt R).
// The tests that decide whether an element needs limiting (a node with
// h < 0), the h_tol cut (h < h_tol) and the non-finite check use the bit
// patterns of the values (integer comparisons; IEEE doubles other than NaN
// order like their bit patterns read as sign-magnitude integers), so an
// element that needs no limiting costs no FP64 instruction beyond the update.
// ---------------------------------------------------------------------------
struct UpdArgs {
    DeviceMesh m;
    double* W;
    const double* R;
    double* Kreg;
    int wreg;  // write the register (0 at a scheme's last stage: nothing reads it there)
    const double* Wn;
    double a, b, dt_host;
    const double* dt_dev;
    int limiter;
    double h_tol;
    double* uv;  // nullable: write u = hu/h, v = hv/h of the new state
    int* status;
    const int* stop;
};

constexpr int UPD_MAX_WPB = 8;  // warps (elements) per block: 2, 4 (default) or 8 (swe_autotune)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Lanes per element of the per-element kernels: the smallest power of two
// that holds the element's nodes, at most a warp. Small degrees put several
// elements on one warp (N=1: 8, N=2 and 3: 2), so that the lanes are not idle.
template <int N>
constexpr int elem_lanes() {
    constexpr int nn = (N + 1) * (N + 1);
    return nn <= 4 ? 4 : (nn <= 8 ? 8 : (nn <= 16 ? 16 : 32));
}

// Butterfly sum / min over aligned groups of G lanes. For G < 32 the result
// equals the full-warp butterfly of the same values with zeros (+inf) in the
// other lanes, bit for bit: those steps only add exact zeros.
template <int G>
__device__ __forceinline__ double seg_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ double seg_max(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int G>
__device__ __forceinline__ double seg_min(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Any lane of this lane's group of G.
template <int G>
__device__ __forceinline__ bool seg_any(bool pred, int lane) {
    const unsigned b = __ballot_sync(0xffffffffu, pred);
    if (G == 32) return b != 0u;
    const unsigned gm = ((1u << G) - 1u) << (lane & ~(G - 1));
    return (b & gm) != 0u;
}

// x < 0 (not -0.0) from the bit pattern.
__device__ __forceinline__ bool is_negative(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b > 0x8000000000000000ULL;
}

// Inf or NaN from the bit pattern.
__device__ __forceinline__ bool non_finite(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ULL) == 0x7ff0000000000000ULL;
}

// x < t for t > 0 and x not NaN, from the bit patterns.
__device__ __forceinline__ bool below(double x, long long tbits) {
    return (long long)__double_as_longlong(x) < tbits;
}

// One element on G lanes (sub = the lane's index in its group). Every lane
// of the warp takes part in the group reductions, also the lanes of a group
// whose element is past the end (valid false: no loads or stores).
template <int N, int MODE, int G>
__device__ __forceinline__ void update_element(const UpdArgs& a, long long k, bool valid, int sub, int lane) {
    constexpr int n = N + 1, nn = n * n, PER = (nn + G - 1) / G;
    const DeviceMesh& m = a.m;
    const long long KN = m.KN;
    const double dt = !valid ? 0.0 : (a.dt_dev ? a.dt_dev[m.inst ? m.inst[k] : 0] : a.dt_host);
    const double bdt = a.b * dt;
    double h[PER], hu[PER], hv[PER];
    bool neg = false, bad = false;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int node = sub + G * r;
        h[r] = hu[r] = hv[r] = 0.0;
        if (valid && node < nn) {
            const long long gid = k * nn + node;
            double w0 = a.W[gid], w1 = a.W[KN + gid], w2 = a.W[2 * KN + gid];
            if (MODE == 1) {
                double k0v = a.R[gid], k1v = a.R[KN + gid], k2v = a.R[2 * KN + gid];
                if (a.a != 0.0) {
                    k0v = fma(a.a, a.Kreg[gid], k0v);
                    k1v = fma(a.a, a.Kreg[KN + gid], k1v);
                    k2v = fma(a.a, a.Kreg[2 * KN + gid], k2v);
                }
                if (a.wreg) {
                    a.Kreg[gid] = k0v;
                    a.Kreg[KN + gid] = k1v;
                    a.Kreg[2 * KN + gid] = k2v;
                }
                w0 = fma(bdt, k0v, w0);
                w1 = fma(bdt, k1v, w1);
                w2 = fma(bdt, k2v, w2);
            } else if (MODE == 2) {
                const double s0 = fma(dt, a.R[gid], w0), s1 = fma(dt, a.R[KN + gid], w1),
                             s2 = fma(dt, a.R[2 * KN + gid], w2);
                w0 = fma(a.a, a.Wn[gid], a.b * s0);
                w1 = fma(a.a, a.Wn[KN + gid], a.b * s1);
                w2 = fma(a.a, a.Wn[2 * KN + gid], a.b * s2);
            }
            h[r] = w0;
            hu[r] = w1;
            hv[r] = w2;
            neg |= is_negative(w0);
            bad |= non_finite(w0) || non_finite(w1) || non_finite(w2);
        }
    }
    // group decisions; the shuffles below run on all 32 lanes (warp-uniform
    // branches only), the per-group results are applied under the group's own
    // flags
    bad = seg_any<G>(bad, lane);
    const bool anyneg = seg_any<G>(neg, lane);
    if (bad && (a.limiter || MODE != 0) && sub == 0) atomicOr(a.status, 2);
    if (a.limiter) {
        const bool here = !bad;  // the limiter acts on finite elements
        const bool need = here && anyneg;
        bool ok = true;
        if (__any_sync(0xffffffffu, need)) {
            // an element of this warp needs limiting: J-weighted means and minimum
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, mn = INFINITY;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int node = sub + G * r;
                if (valid && node < nn) {
                    const double wj = m.wJ[k * nn + node];
                    s0 = fma(wj, h[r], s0);
                    s1 = fma(wj, hu[r], s1);
                    s2 = fma(wj, hv[r], s2);
                    mn = fmin(mn, h[r]);
                }
            }
            const double rv = valid ? m.rvol[k] : 0.0;
            const double m0 = seg_sum<G>(s0) * rv, m1 = seg_sum<G>(s1) * rv, m2 = seg_sum<G>(s2) * rv;
            mn = seg_min<G>(mn);
            if (need) {
                if (m0 < 0.0) {
                    if (sub == 0) atomicOr(a.status, 1);
                    ok = false;
                } else if (m0 - mn > 0.0) {
                    const double theta = fmin(1.0, m0 / (m0 - mn));
#pragma unroll
                    for (int r = 0; r < PER; ++r) {
                        h[r] = fma(theta, h[r] - m0, m0);
                        hu[r] = fma(theta, hu[r] - m1, m1);
                        hv[r] = fma(theta, hv[r] - m2, m2);
                    }
                }
            }
        }
        if (ok && here) {
            const long long tb = __double_as_longlong(a.h_tol);
#pragma unroll
            for (int r = 0; r < PER; ++r)
                if (below(h[r], tb)) hu[r] = hv[r] = 0.0;
        }
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int node = sub + G * r;
        if (valid && node < nn) {
            const long long gid = k * nn + node;
            a.W[gid] = h[r];
            a.W[KN + gid] = hu[r];
            a.W[2 * KN + gid] = hv[r];
            if (a.uv) {
                double u, v;
                velocities(h[r], hu[r], hv[r], u, v);
                a.uv[gid] = u;
                a.uv[KN + gid] = v;
            }
        }
    }
}

// One element per group of G lanes (32/G elements per warp), blocks of
// blockDim.x/32 warps looping over the elements.
template <int N, int MODE>
__global__ void __launch_bounds__(32 * UPD_MAX_WPB) k_update(UpdArgs a) {
    if (stopped(a.stop)) return;
    constexpr int G = elem_lanes<N>(), EPW = 32 / G;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int sub = lane & (G - 1), grp = lane / G;
    for (long long kb = ((long long)blockIdx.x * wpb + wid) * EPW; kb < a.m.K;
         kb += (long long)gridDim.x * wpb * EPW) {
        const long long k = kb + grp;
        update_element<N, MODE, G>(a, k, k < a.m.K, sub, lane);
    }
}

// ---------------------------------------------------------------------------
// Time step: max over nodes of (lambda_xi + lambda_eta)/J and max over element
// side nodes of the inverse positivity restrictions of Eq. CFLConstraints
// (Lemma PosPres), reduced with integer atomics on the bit patterns of
// non-negative doubles; one warp per element.
// ---------------------------------------------------------------------------
struct DtArgs {
    DeviceMesh m;
    const double* W;
    const double* uv;
    const double* cfl_n;
    int pos;
    unsigned long long* bits;
    const double* eps;  // element viscosities of W (read when kv > 0)
    double kv;          // viscous restriction factor; 0: the paper's rule
    const int* stop;
};

// Non-negative doubles order like their bit patterns: max by an integer
// comparison (no FP64 instruction).
__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b > a ? b : a;
}

constexpr int DT_WPB = 4;  // warps (elements) per block of the time-step kernel

// One element on a group of G lanes (several elements per warp for small
// degrees; lanes of a group past the last element only join the
// shuffles). The celerities c = sqrt(g max(h, 0)) of the CFL part are kept in
// shared memory (sc, the group's n*n slots) for the own side of the
// positivity part. The maxima of non-negative values and the sign tests are
// integer operations on the bit patterns.
template <int N, int G, bool VISC>
__device__ __forceinline__ void dt_element(const DtArgs& a, long long k, bool valid, int sub, double* sc) {
    constexpr int n = N + 1, nn = n * n;
    const DeviceMesh& m = a.m;
    const double g = m.g, g2 = 2.0 * m.g;
    unsigned long long lamb = 0;
    // viscous restriction (VISC, kv > 0): the node's rate gains eps_k kv a^2
    const double ekv = (VISC && valid) ? a.eps[k] * a.kv : 0.0;
    for (int node = sub; node < nn && valid; node += G) {
        const long long id = k * nn + node;
        const double h = a.W[id], u = a.uv[id], v = a.uv[m.KN + id];
        const double c = sqrt_pos(g * pos_part(h));
        sc[node] = c;
        const double vel = fabs(fma(m.axx[id], u, m.axy[id] * v)) + fabs(fma(m.aex[id], u, m.aey[id] * v));
        const double an = a.cfl_n[id];
        double lam = fma(c, an, m.rJ[id] * vel);
        if (VISC) lam = fma(ekv * an, an, lam);
        lamb = max_bits(lamb, lam);
    }
    const double lam = seg_max<G>(__longlong_as_double((long long)lamb));
    unsigned long long* bits = a.bits + 2 * (valid && m.inst ? m.inst[k] : 0);
    if (valid && sub == 0 && lam > 0.0) atomic_max_pos(&bits[0], lam);
    if (a.pos) {  // uniform: the flag is a kernel argument
        __syncwarp();
        unsigned long long invb = 0;
        for (int sn = sub; sn < 4 * n && valid; sn += G) {
            const int f = sn / n, p = sn - f * n;
            const int i = (f == 0 || f == 2) ? p : (f == 1 ? N : 0);
            const int j = (f == 1 || f == 3) ? p : (f == 2 ? N : 0);
            const int ownl = j * n + i;
            const long long own = k * nn + ownl;
            const long long slot = k * 4 * n + sn;
            const long long sb = m.s_nb[slot];
            const bool wall = sb < 0;  // solid wall: the mirror state
            const long long nb = wall ? own : sb;
            const double nx = m.s_nx[slot], ny = m.s_ny[slot], rwa = m.s_rwa[slot];
            const double hm = a.W[own], hp = a.W[nb];
            const double utm = fma(nx, a.uv[own], ny * a.uv[m.KN + own]);
            const double utp = wall ? -utm : fma(nx, a.uv[nb], ny * a.uv[m.KN + nb]);
            const double cm = sc[ownl], cp = wall ? cm : sqrt_pos(g * pos_part(hp));
            // with s_u = 2 u~_a and s_c = 2 c_a (both sums, no halving):
            // A = |u~_a + c_a| + |u~_a - c_a| = max(|s_u|, s_c) and
            // B = |u~_a + c_a| - |u~_a - c_a| = sgn(s_u) min(|s_u|, s_c), the
            // maximum, minimum and sign taken on the bit patterns
            const double su = utm + utp, scs = cm + cp;
            const unsigned long long bau = (unsigned long long)__double_as_longlong(fabs(su)),
                                     bsc = (unsigned long long)__double_as_longlong(scs);
            const double A = __longlong_as_double((long long)(bau > bsc ? bau : bsc));
            const unsigned long long bB =
                (bau < bsc ? bau : bsc) | ((unsigned long long)__double_as_longlong(su) & 0x8000000000000000ULL);
            const double B = __longlong_as_double((long long)bB);
            const double i1 = (su + A) * rwa;
            if ((long long)__double_as_longlong(i1) > 0) invb = max_bits(invb, i1);
            const double jump = utp - utm;
            // h- > 0 and B [[u~]] < 0 (nonzero factors of opposite signs);
            // c_a |B [[u~]]| / (g h-) with c_a = s_c / 2
            const unsigned long long bJ = (unsigned long long)__double_as_longlong(jump);
            if ((long long)__double_as_longlong(hm) > 0 && ((bB ^ bJ) >> 63) && nonzero(B) && nonzero(jump))
                invb = max_bits(invb, fabs(scs * B * jump) * rwa * recip_pos(g2 * hm));
        }
        const double inv = seg_max<G>(__longlong_as_double((long long)invb));
        if (valid && sub == 0 && inv > 0.0) atomic_max_pos(&bits[1], inv);
    }
    __syncwarp();  // the next element reuses sc
}

template <int N, bool VISC>
__global__ void __launch_bounds__(32 * DT_WPB) k_dt(DtArgs a) {
    constexpr int G = elem_lanes<N>(), EPW = 32 / G, nn = (N + 1) * (N + 1);
    __shared__ double sc[DT_WPB][EPW * nn];
    if (stopped(a.stop)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int sub = lane & (G - 1), grp = lane / G;
    for (long long kb = ((long long)blockIdx.x * wpb + w) * EPW; kb < a.m.K; kb += (long long)gridDim.x * wpb * EPW) {
        const long long k = kb + grp;
        dt_element<N, G, VISC>(a, k, k < a.m.K, sub, sc[w] + grp * nn);
    }
}

// One thread per instance: dt[i] in use, dt[ninst + i] CFL, dt[2 ninst + i] positivity.
__global__ void k_dt_final(const unsigned long long* bits, double* dt, int ninst, double cfl, int N,
                           double dt_fixed, const int* stop) {
    if (stopped(stop)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const double lam = __longlong_as_double((long long)bits[2 * i]);
    const double inv = __longlong_as_double((long long)bits[2 * i + 1]);
    const double dtc = lam > 0.0 ? cfl * 2.0 / (N + 1.0) / lam : INFINITY;
    const double dtp = inv > 0.0 ? 1.0 / inv : INFINITY;
    dt[ninst + i] = dtc;
    dt[2 * ninst + i] = dtp;
    dt[i] = dt_fixed > 0.0 ? dt_fixed : fmin(dtc, dtp);
}

__global__ void k_copy(long long count, const double* __restrict__ src, double* __restrict__ dst,
                       const int* stop) {
    if (stopped(stop)) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Device-side rollback of an asynchronous step: where the status word is set,
// dst gets back src (the state at the start of the failing step).
// After a failed step (status set): the start state back into W, and the
// velocities of it (the integrals that follow read them).
__global__ void k_restore(long long KN, const double* __restrict__ src, double* __restrict__ dst,
                          double* __restrict__ uv, const int* status) {
    if (*(volatile const int*)status == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < KN;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = src[i], hu = src[KN + i], hv = src[2 * KN + i];
        dst[i] = h;
        dst[KN + i] = hu;
        dst[2 * KN + i] = hv;
        double u, v;
        velocities(h, hu, hv, u, v);
        uv[i] = u;
        uv[KN + i] = v;
    }
}

// ---------------------------------------------------------------------------
// Diagnostics: sum J w w W (what = 0, three sums), sum J w w e(W) (what = 1,
// Eq. entropyFunction), or all four (what = 2). Fixed grid, per-block tree
// sums, then one warp per component adds the partials in a fixed order: the
// result does not depend on scheduling. The kinetic part of e is
// (hu u + hv v)/2 with the velocities u, v of W (written by the primitives
// kernel or the stage update that produced W): no reciprocal here, and zero
// where h <= 0, where u = v = 0.
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__global__ void k_reduce_part(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv, int what,
                              double* __restrict__ part) {
    __shared__ double sh[4][RED_THREADS];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const double g = m.g;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < m.KN;
         id += (long long)gridDim.x * blockDim.x) {
        const double wj = m.wJ[id], h = W[id], hu = W[m.KN + id], hv = W[2 * m.KN + id];
        if (what != 1) {
            s0 = fma(wj, h, s0);
            s1 = fma(wj, hu, s1);
            s2 = fma(wj, hv, s2);
        }
        if (what != 0) {
            const double kin = 0.5 * fma(hu, uv[id], hv * uv[m.KN + id]);
            const double e = kin + g * h * fma(0.5, h, m.bn[id]);
            s3 = fma(wj, e, s3);
        }
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = s3;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) part[c * RED_BLOCKS + blockIdx.x] = sh[c][0];
}

// Discrete entropy rate: per-block partial sums of J w_i w_j q(W) . R with
// the entropy variables q = (g(h+b) - (u^2+v^2)/2, u, v) of Eq.
// entropyVariables (component 0), and of J w_i w_j sum_c |q_c R_c| (component
// 1, the scale of the cancellation); components 2 and 3 are zero.
__global__ void k_rate_part(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ R,
                            double* __restrict__ part) {
    __shared__ double sh[2][RED_THREADS];
    double s0 = 0.0, s1 = 0.0;
    const double g = m.g;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < m.KN;
         id += (long long)gridDim.x * blockDim.x) {
        const double wj = m.wJ[id], h = W[id];
        double u, v;
        velocities(h, W[m.KN + id], W[2 * m.KN + id], u, v);
        const double q1 = fma(g, h + m.bn[id], -0.5 * fma(u, u, v * v));
        const double t1 = q1 * R[id], t2 = u * R[m.KN + id], t3 = v * R[2 * m.KN + id];
        s0 = fma(wj, t1 + t2 + t3, s0);
        s1 = fma(wj, fabs(t1) + fabs(t2) + fabs(t3), s1);
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 2; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sh[0][0];
        part[RED_BLOCKS + blockIdx.x] = sh[1][0];
        part[2 * RED_BLOCKS + blockIdx.x] = 0.0;
        part[3 * RED_BLOCKS + blockIdx.x] = 0.0;
    }
}

// One warp per component: lane sums of a fixed stride, then a fixed butterfly.
// With status (nullable) also out[4] = dt[0], out[5] = the status word, so
// that a step's results come back in one device-to-host copy.
__global__ void k_reduce_final(const double* __restrict__ part, double* __restrict__ out,
                               const double* __restrict__ dt = nullptr, const int* __restrict__ status = nullptr) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < RED_BLOCKS; b += 32) s += part[c * RED_BLOCKS + b];
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
    if (threadIdx.x == 0 && status) {
        out[4] = dt[0];
        out[5] = (double)*(volatile const int*)status;
    }
}

// Per-instance integrals of an ensemble group: block i sums the nodes of
// elements [ebeg[i], ebeg[i+1]) into out[4 i .. 4 i + 3] (mass, momenta,
// entropy), in a fixed order.
__global__ void k_reduce_inst(DeviceMesh m, const double* __restrict__ W, const double* __restrict__ uv,
                              const long long* __restrict__ ebeg, double* __restrict__ out) {
    __shared__ double sh[4][RED_THREADS];
    const long long nn = (long long)m.n * m.n;
    const long long lo = ebeg[blockIdx.x] * nn, hi = ebeg[blockIdx.x + 1] * nn;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const double g = m.g;
    for (long long id = lo + threadIdx.x; id < hi; id += blockDim.x) {
        const double wj = m.wJ[id], h = W[id], hu = W[m.KN + id], hv = W[2 * m.KN + id];
        s0 = fma(wj, h, s0);
        s1 = fma(wj, hu, s1);
        s2 = fma(wj, hv, s2);
        const double kin = 0.5 * fma(hu, uv[id], hv * uv[m.KN + id]);
        s3 = fma(wj, kin + g * h * fma(0.5, h, m.bn[id]), s3);
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = s3;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

template <int N>
void update_n(swe_ctx* c, int mode, const UpdArgs& a, cudaStream_t s) {
    const int wpb = c->upd_wpb;
    const int blocks = persistent_grid(c, wpb * (32 / elem_lanes<N>()));
    Timed tm(c, KC_UPDATE, s);
    if (mode == 0) k_update<N, 0><<<blocks, 32 * wpb, 0, s>>>(a);
    else if (mode == 1) k_update<N, 1><<<blocks, 32 * wpb, 0, s>>>(a);
    else k_update<N, 2><<<blocks, 32 * wpb, 0, s>>>(a);
}

template <int N>
void dt_n(swe_ctx* c, const DtArgs& a, cudaStream_t s) {
    Timed tm(c, KC_DT, s);
    const int grid = persistent_grid(c, DT_WPB * (32 / elem_lanes<N>()));
    if (a.kv > 0.0) k_dt<N, true><<<grid, 32 * DT_WPB, 0, s>>>(a);
    else k_dt<N, false><<<grid, 32 * DT_WPB, 0, s>>>(a);
}

#define SWE_SWITCH_N(N, CALL)                                                         \
    switch (N) {                                                                      \
        case 1: CALL(1); break; case 2: CALL(2); break; case 3: CALL(3); break;      \
        case 4: CALL(4); break; case 5: CALL(5); break; case 6: CALL(6); break;      \
        case 7: CALL(7); break; case 8: CALL(8); break; case 9: CALL(9); break;      \
        case 10: CALL(10); break; case 11: CALL(11); break; case 12: CALL(12); break; \
        default: break;                                                               \
    }

}  // namespace

void init_tables_face() { upload_tables(); }

void launch_prim(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    Timed tm(c, KC_PRIM, s);
    k_prim<<<grid_for(c->m.KN, 256), 256, 0, s>>>(c->m.KN, W, c->w.uv, stop);
}

void launch_surface(swe_ctx* c, const double* W, cudaStream_t s, const int* stop) {
    const long long total = (long long)c->m.nfaces * c->m.n;
    if (total > 0) {
        Timed tm(c, KC_FACE, s);
        if (c->p.flux)
            k_surface<true><<<grid_for(total, 128), 128, 0, s>>>(c->m, W, c->w.uv, c->w.Fout, c->w.Ustar, stop);
        else
            k_surface<false><<<grid_for(total, 128), 128, 0, s>>>(c->m, W, c->w.uv, c->w.Fout, c->w.Ustar, stop);
    }
    const long long walls = (long long)c->m.nwall * c->m.n;
    if (walls > 0) {
        Timed tm(c, KC_FACE, s);
        if (c->p.flux)
            k_wall<true><<<grid_for(walls, 128), 128, 0, s>>>(c->m, W, c->w.uv, c->w.Fout, c->w.Ustar, stop);
        else
            k_wall<false><<<grid_for(walls, 128), 128, 0, s>>>(c->m, W, c->w.uv, c->w.Fout, c->w.Ustar, stop);
    }
}

void launch_ustar(swe_ctx* c, cudaStream_t s) {
    const long long total = ((long long)c->m.nfaces + c->m.nwall) * c->m.n;
    if (total == 0) return;
    Timed tm(c, KC_FACE, s);
    k_ustar<<<grid_for(total, 128), 128, 0, s>>>(c->m, c->w.uv, c->w.Ustar);
}

void launch_visc_face(swe_ctx* c, cudaStream_t s, const int* stop) {
    // a fixed grid striding over the elements and over the viscous elements'
    // side slots (their number is known on the device only): sixteen blocks
    // per SM at most
    const long long most = (long long)c->m.K * 4 * c->m.n;
    const int blocks = grid_for(most, 128) < 16 * c->sms ? grid_for(most, 128) : 16 * c->sms;
    Timed tm(c, KC_VFACE, s);
    k_visc_face<<<blocks, 128, 0, s>>>(c->m, c->w.Fvtr, c->w.eps, c->w.vlist, c->w.vcount, c->w.Fvout, c->w.touch,
                                       stop);
}

void launch_update(swe_ctx* c, int mode, double* W, double a, double b, double dt_host,
                   const double* dt_dev, cudaStream_t s, const int* stop, bool write_uv, bool write_reg) {
    UpdArgs u{c->m, W, c->w.R, c->w.Kreg, write_reg ? 1 : 0, c->w.Wn, a, b, dt_host, dt_dev, c->p.limiter,
              c->h_tol, write_uv ? c->w.uv : nullptr, c->w.status, stop};
#define SWE_UPD(NN) update_n<NN>(c, mode, u, s)
    SWE_SWITCH_N(c->m.N, SWE_UPD)
#undef SWE_UPD
}

void launch_dt(swe_ctx* c, const double* W, double dt_fixed, cudaStream_t s, const int* stop) {
    cudaMemsetAsync(c->w.dtbits, 0, 2 * sizeof(unsigned long long) * c->m.ninst, s);
    DtArgs a{c->m, W, c->w.uv, c->m.nax, (c->p.limiter && c->p.flux) ? 1 : 0, c->w.dtbits, c->w.eps, c->kv, stop};
#define SWE_DT(NN) dt_n<NN>(c, a, s)
    SWE_SWITCH_N(c->m.N, SWE_DT)
#undef SWE_DT
    Timed tm(c, KC_DT, s);
    k_dt_final<<<(c->m.ninst + 127) / 128, 128, 0, s>>>(c->w.dtbits, c->w.dt, c->m.ninst, c->p.cfl, c->m.N,
                                                          dt_fixed, stop);
}

void launch_copy(swe_ctx* c, const double* src, double* dst, long long count, cudaStream_t s,
                 const int* stop) {
    Timed tm(c, KC_UPDATE, s);
    k_copy<<<grid_for(count, 256) > 4096 ? 4096 : grid_for(count, 256), 256, 0, s>>>(count, src, dst, stop);
}

void launch_reduce(swe_ctx* c, const double* W, int what, double* host_out, cudaStream_t s) {
    launch_reduce_dev(c, W, what, false, s);
    cudaMemcpyAsync(host_out, c->w.part + 4 * RED_BLOCKS, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

void launch_reduce_dev(swe_ctx* c, const double* W, int what, bool pack, cudaStream_t s, double* dst) {
    {
        Timed tm(c, KC_REDUCE, s);
        k_reduce_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(c->m, W, c->w.uv, what, c->w.part);
    }
    Timed tm(c, KC_REDUCE, s);
    double* out = dst ? dst : c->w.part + 4 * RED_BLOCKS;
    if (pack)
        k_reduce_final<<<1, 128, 0, s>>>(c->w.part, out, c->w.dt, c->w.status);
    else
        k_reduce_final<<<1, 128, 0, s>>>(c->w.part, out);
}

void launch_restore(swe_ctx* c, double* W, cudaStream_t s) {
    const long long KN = c->m.KN;
    Timed tm(c, KC_UPDATE, s);
    k_restore<<<grid_for(KN, 256) > 4096 ? 4096 : grid_for(KN, 256), 256, 0, s>>>(KN, c->w.Wn, W, c->w.uv,
                                                                                   c->w.status);
}

void launch_rate(swe_ctx* c, const double* W, const double* R, double* host_out, cudaStream_t s) {
    {
        Timed tm(c, KC_REDUCE, s);
        k_rate_part<<<RED_BLOCKS, RED_THREADS, 0, s>>>(c->m, W, R, c->w.part);
    }
    {
        Timed tm(c, KC_REDUCE, s);
        k_reduce_final<<<1, 128, 0, s>>>(c->w.part, c->w.part + 4 * RED_BLOCKS);
    }
    cudaMemcpyAsync(host_out, c->w.part + 4 * RED_BLOCKS, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

void launch_reduce_inst(swe_ctx* c, const double* W, const long long* ebeg, double* out, cudaStream_t s) {
    Timed tm(c, KC_REDUCE, s);
    k_reduce_inst<<<c->m.ninst, RED_THREADS, 0, s>>>(c->m, W, c->w.uv, ebeg, out);
}

}  // namespace swe
