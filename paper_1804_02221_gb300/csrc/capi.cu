// C ABI of the swedg library: context construction (host geometry, face
// lists, device upload), the right-hand-side and time-step orchestration,
// diagnostics and timing.
#include <math.h>
#include <string.h>

#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "swe_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(SWE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme.
const double kLsrkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsrkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                          1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                          2277821191437.0 / 14882151754819.0};

constexpr int kEventPairs = 8192;

void init_device_tables(int device) {
    static std::mutex mu;
    static std::set<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(device)) return;
    swe::init_tables_volume();
    swe::init_tables_volume_std();
    swe::init_tables_adjoint();
    swe::init_tables_face();
    swe::init_tables_av();
    done.insert(device);
}

// Volume node (i, j) of face node p on face f.
inline void face_node(int N, int f, int p, int& i, int& j) {
    switch (f) {
        case 0: i = p; j = 0; break;
        case 1: i = N; j = p; break;
        case 2: i = p; j = N; break;
        default: i = 0; j = p; break;
    }
}

template <typename T>
T* dev_upload(swe_ctx* c, const std::vector<T>& h, cudaError_t& err) {
    void* p = nullptr;
    size_t bytes = h.size() * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) return nullptr;
    c->allocations.push_back(p);
    if (!h.empty()) err = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return static_cast<T*>(p);
}

double* dev_alloc(swe_ctx* c, size_t count, cudaError_t& err) {
    void* p = nullptr;
    err = cudaMalloc(&p, (count ? count : 1) * sizeof(double));
    if (err != cudaSuccess) return nullptr;
    c->allocations.push_back(p);
    return static_cast<double*>(p);
}

void free_all(swe_ctx* c) {
    for (void* p : c->allocations) cudaFree(p);
    c->allocations.clear();
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_first) cudaEventDestroy(c->ev_first);
    if (c->s_av) cudaStreamDestroy(c->s_av);
    c->ev_fork = c->ev_join = c->ev_first = nullptr;
    c->s_av = nullptr;
}

}  // namespace

namespace swe {

int set_last_error(int code, const std::string& msg) { return fail(code, msg); }

Timed::Timed(swe_ctx* c_, int cls, cudaStream_t s_) : c(c_), s(s_) {
    c->launches++;
    if (c->timing && ((c->timing_mask >> cls) & 1u) && c->ev_used < (int)c->ev_class.size()) {
        idx = c->ev_used++;
        c->ev_class[idx] = cls;
        cudaEventRecord(c->ev[2 * idx], s);
    }
}

Timed::~Timed() {
    if (idx >= 0) cudaEventRecord(c->ev[2 * idx + 1], s);
}

}  // namespace swe

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

namespace swe {

// Context construction shared by swe_create and the ensembles: inst (host,
// nullable) gives the instance index of every element (ninst instances);
// shared_status (device, nullable) replaces the context's own status word.
int create_ctx(int N, int K, const double* x, const double* y, const int32_t* EToE, const int32_t* EToF,
               const int32_t* flip, const double* b, double g, const swe_params* p, const int32_t* inst,
               int ninst, int* shared_status, swe_ctx** out) {
    if (!out) return fail(SWE_ERR_ARG, "swe_create: out is NULL");
    *out = nullptr;
    if (!x || !y || !EToE || !EToF || !flip || !b || !p)
        return fail(SWE_ERR_ARG, "swe_create: NULL input");
    if (N < 1 || N > NMAX) return fail(SWE_ERR_ARG, "swe_create: N must be in 1..12");
    if (K < 1) return fail(SWE_ERR_ARG, "swe_create: K must be >= 1");
    if (!(g > 0.0) || !isfinite(g)) return fail(SWE_ERR_ARG, "swe_create: g must be positive");
    if (p->flux != 0 && p->flux != 1) return fail(SWE_ERR_ARG, "swe_create: flux must be 0 or 1");
    if (p->rk != 0 && p->rk != 1) return fail(SWE_ERR_ARG, "swe_create: rk must be 0 or 1");
    if (p->volume != 0 && p->volume != 1) return fail(SWE_ERR_ARG, "swe_create: volume must be 0 or 1");
    if (p->av && !(p->eps0 >= 0.0)) return fail(SWE_ERR_ARG, "swe_create: eps0 must be >= 0");
    if (!isnan(p->h_tol) && !(p->h_tol >= 0.0)) return fail(SWE_ERR_ARG, "swe_create: h_tol must be >= 0");
    if (!(p->cfl_visc >= 0.0) || isinf(p->cfl_visc))
        return fail(SWE_ERR_ARG, "swe_create: cfl_visc must be finite and >= 0");
    const int n = N + 1, nn = n * n;
    const long long KN = (long long)K * nn, KS = (long long)K * 4 * n;
    if (KN * 3 > 2147483647LL) return fail(SWE_ERR_ARG, "swe_create: mesh too large for 32-bit node ids");
    // connectivity (EToE = -1: solid wall)
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < 4; ++f) {
            const int kk = EToE[4 * k + f], ff = EToF[4 * k + f];
            if (kk == -1) continue;
            if (kk < 0 || kk >= K || ff < 0 || ff > 3)
                return fail(SWE_ERR_ARG, "swe_create: EToE/EToF out of range at element " + std::to_string(k));
            if ((kk == k && ff == f) || EToE[4 * kk + ff] != k || EToF[4 * kk + ff] != f ||
                flip[4 * kk + ff] != flip[4 * k + f] || (flip[4 * k + f] != 0 && flip[4 * k + f] != 1))
                return fail(SWE_ERR_ARG, "swe_create: connectivity not reciprocal at element " + std::to_string(k));
        }
    const Tables& T = tables();
    const double* D = T.D + mat_offset(N);
    const double* w = T.w + vec_offset(N);

    // ---- host geometry (Sec. 2.1) ----
    std::vector<double> axx(KN), axy(KN), aex(KN), aey(KN), rJ(KN), wJ(KN), srcx(KN), srcy(KN), bn(KN),
        cfln(KN), rvol(K), Jv(KN);
    // the source as the start of the split volume kernel's pressure sums
    // (degrees with pressure sums only; empty otherwise)
    const bool psums = p->volume == 0 && swe::pressure_sums_degree(N);
    std::vector<double> ssx(psums ? KN : 0), ssy(psums ? KN : 0);
    std::vector<double> tmp(4 * nn);
    for (int k = 0; k < K; ++k) {
        const double* X = x + (size_t)k * nn;
        const double* Y = y + (size_t)k * nn;
        const double* Bk = b + (size_t)k * nn;
        double vol = 0.0;
        // metric terms from coordinates relative to the element's first node
        // (D annihilates constants): the sums then do not carry the
        // coordinates' magnitude, which on fine meshes exceeds the element
        // size by orders of magnitude and would cost digits of the metrics
        const double X0 = X[0], Y0 = Y[0];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double x_xi = 0, x_eta = 0, y_xi = 0, y_eta = 0;
                for (int q = 0; q < n; ++q) {
                    x_xi += D[i * n + q] * (X[j * n + q] - X0);
                    y_xi += D[i * n + q] * (Y[j * n + q] - Y0);
                    x_eta += D[j * n + q] * (X[q * n + i] - X0);
                    y_eta += D[j * n + q] * (Y[q * n + i] - Y0);
                }
                const double J = x_xi * y_eta - x_eta * y_xi;
                const long long id = (long long)k * nn + j * n + i;
                if (!(J > 0.0) || !isfinite(J))
                    return fail(SWE_ERR_GEOM, "swe_create: non-positive Jacobian in element " + std::to_string(k));
                axx[id] = y_eta;
                axy[id] = -x_eta;
                aex[id] = -y_xi;
                aey[id] = x_xi;
                Jv[id] = J;
                rJ[id] = 1.0 / J;
                wJ[id] = w[i] * w[j] * J;
                vol += wJ[id];
                bn[id] = Bk[j * n + i];
                cfln[id] = (sqrt(y_eta * y_eta + x_eta * x_eta) + sqrt(y_xi * y_xi + x_xi * x_xi)) / J;
            }
        rvol[k] = 1.0 / vol;
        // split-form bathymetry derivatives (Eq. SourceDisc, plain D):
        // gamma_c = a_xi,c D_xi b + D_xi(a_xi,c b) + a_eta,c D_eta b + D_eta(a_eta,c b)
        const long long o = (long long)k * nn;
        for (int a = 0; a < nn; ++a) {
            tmp[a] = axx[o + a] * bn[o + a];
            tmp[nn + a] = aex[o + a] * bn[o + a];
            tmp[2 * nn + a] = axy[o + a] * bn[o + a];
            tmp[3 * nn + a] = aey[o + a] * bn[o + a];
        }
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double bx = 0, be = 0, d0 = 0, d1 = 0, d2 = 0, d3 = 0;
                for (int q = 0; q < n; ++q) {
                    bx += D[i * n + q] * bn[o + j * n + q];
                    be += D[j * n + q] * bn[o + q * n + i];
                    d0 += D[i * n + q] * tmp[j * n + q];
                    d1 += D[j * n + q] * tmp[nn + q * n + i];
                    d2 += D[i * n + q] * tmp[2 * nn + j * n + q];
                    d3 += D[j * n + q] * tmp[3 * nn + q * n + i];
                }
                const long long id = o + j * n + i;
                if (p->volume == 1) {
                    // standard form: -g J grad b / J with J b_x = y_eta b_xi - y_xi b_eta,
                    // J b_y = -x_eta b_xi + x_xi b_eta
                    srcx[id] = -g * (axx[id] * bx + aex[id] * be) * rJ[id];
                    srcy[id] = -g * (axy[id] * bx + aey[id] * be) * rJ[id];
                    continue;
                }
                const double gx = axx[id] * bx + d0 + aex[id] * be + d1;
                const double gy = axy[id] * bx + d2 + aey[id] * be + d3;
                srcx[id] = -0.5 * g * gx * rJ[id];
                srcy[id] = -0.5 * g * gy * rJ[id];
                // h srcx = f (2g h) ssx with f = -1/(w_i w_j J): the source
                // joins the node's pressure sums sum_q h_q Sx before they
                // are scaled by 2g h (w_i w_j gamma / 4 = sum_q b_q Sx over
                // both lines of the node, with the pair constants' Sx)
                if (psums) {
                    ssx[id] = 0.25 * w[i] * w[j] * gx;
                    ssy[id] = 0.25 * w[i] * w[j] * gy;
                }
            }
    }

    // ---- pair constants of the volume kernel ----
    // For line l in direction d (0: xi-line j = l, 1: eta-line i = l) and the
    // pair (i, q), i < q, of positions along it: the contravariant vector a of
    // the direction summed over the two nodes, times w_i w_j D_iq / 4 with
    // (w_i w_j) the quadrature weight of the pair's first node. The volume
    // kernel accumulates w_i w_j L with these, so that the partner node takes
    // the negative (w_q D_qi = -w_i D_iq, the SBP property).
    const int NP = N * (N + 1) / 2;
    // (the standard volume form has no pairs)
    std::vector<double> pm(p->volume == 1 ? 0 : (size_t)K * 2 * NP * 2 * n), fwJ(KN);
    for (long long a = 0; a < KN; ++a) fwJ[a] = -1.0 / wJ[a];
    std::vector<double> fwJ2(p->volume == 1 ? 0 : KN);
    for (size_t a = 0; a < fwJ2.size(); ++a) fwJ2[a] = 2.0 * fwJ[a];  // exact
    for (int k = 0; k < K && p->volume == 0; ++k)
        for (int d = 0; d < 2; ++d) {
            const double* vx = d == 0 ? axx.data() : aex.data();
            const double* vy = d == 0 ? axy.data() : aey.data();
            for (int l = 0; l < n; ++l) {
                int pr = 0;
                for (int i = 0; i < n; ++i)
                    for (int q = i + 1; q < n; ++q, ++pr) {
                        const long long na = (long long)k * nn + (d == 0 ? l * n + i : i * n + l);
                        const long long nb = (long long)k * nn + (d == 0 ? l * n + q : q * n + l);
                        const int ii = d == 0 ? i : l, jj = d == 0 ? l : i;
                        const double s = w[ii] * w[jj] * D[i * n + q] * 0.25;
                        const size_t base = ((((size_t)k * 2 + d) * NP + pr) * n + l) * 2;
                        pm[base] = s * (vx[na] + vx[nb]);
                        pm[base + 1] = s * (vy[na] + vy[nb]);
                    }
            }
        }

    // ---- unique faces and element sides ----
    std::vector<int32_t> f_im, f_ip, f_tm, f_tp, s_nb(KS), s_face(KS, -1), w_im, w_tm;
    std::vector<double> f_nx, f_ny, f_js, f_sx, f_sy, f_bm, f_bp, s_nx(KS), s_ny(KS), s_rwa(KS), w_nx, w_ny, w_js;
    const double w0 = w[0];
    auto outward = [&](int k, int f, int i, int j, double& nx, double& ny) {
        const long long id = (long long)k * nn + j * n + i;
        switch (f) {
            case 0: nx = -aex[id]; ny = -aey[id]; break;
            case 1: nx = axx[id]; ny = axy[id]; break;
            case 2: nx = aex[id]; ny = aey[id]; break;
            default: nx = -axx[id]; ny = -axy[id]; break;
        }
    };
    int nfaces = 0, nwall = 0;
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < 4; ++f) {
            const int kk = EToE[4 * k + f], ff = EToF[4 * k + f], fl = flip[4 * k + f];
            if (kk < 0) {
                for (int pn = 0; pn < n; ++pn) {
                    int i, j;
                    face_node(N, f, pn, i, j);
                    const long long own = (long long)k * nn + j * n + i;
                    double nx, ny;
                    outward(k, f, i, j, nx, ny);
                    const double js = sqrt(nx * nx + ny * ny);
                    const long long slot = ((long long)k * 4 + f) * n + pn;
                    s_nb[slot] = -1;
                    s_nx[slot] = nx / js;
                    s_ny[slot] = ny / js;
                    s_rwa[slot] = js / (w0 * Jv[own]);
                    w_im.push_back((int32_t)own);
                    w_tm.push_back((int32_t)slot);
                    w_nx.push_back(nx / js);
                    w_ny.push_back(ny / js);
                    w_js.push_back(js);
                }
                ++nwall;
                continue;
            }
            for (int pn = 0; pn < n; ++pn) {
                const int q = fl ? N - pn : pn;
                int i, j, ii, jj;
                face_node(N, f, pn, i, j);
                face_node(N, ff, q, ii, jj);
                const long long own = (long long)k * nn + j * n + i;
                const long long nb = (long long)kk * nn + jj * n + ii;
                double nx, ny;
                outward(k, f, i, j, nx, ny);
                const double js = sqrt(nx * nx + ny * ny);
                const long long slot = ((long long)k * 4 + f) * n + pn;
                s_nb[slot] = (int32_t)nb;
                s_nx[slot] = nx / js;
                s_ny[slot] = ny / js;
                s_rwa[slot] = js / (w0 * Jv[own]);
                if (kk > k || (kk == k && ff > f)) {
                    s_face[slot] = (int32_t)f_im.size();
                    s_face[((long long)kk * 4 + ff) * n + q] = (int32_t)f_im.size();
                    f_im.push_back((int32_t)own);
                    f_ip.push_back((int32_t)nb);
                    f_tm.push_back((int32_t)slot);
                    f_tp.push_back((int32_t)(((long long)kk * 4 + ff) * n + q));
                    f_nx.push_back(nx / js);
                    f_ny.push_back(ny / js);
                    // over 8 (exact): the interface flux kernel forms 8 F
                    f_js.push_back(0.125 * js);
                    f_sx.push_back(0.125 * nx);
                    f_sy.push_back(0.125 * ny);
                    f_bm.push_back(bn[own]);
                    f_bp.push_back(bn[nb]);
                }
            }
            if (kk > k || (kk == k && ff > f)) ++nfaces;
        }

    // ---- device ----
    swe_ctx* c = new swe_ctx();
    cudaError_t err = cudaGetDevice(&c->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (err != cudaSuccess) {
        delete c;
        return cuda_fail(err, "swe_create: device query");
    }
    init_device_tables(c->device);
    c->p = *p;
    const double s0 = -4.0 * log10((double)N);
    c->sigma_min = isnan(p->sigma_min) ? s0 - 1.0 : p->sigma_min;
    c->sigma_max = isnan(p->sigma_max) ? s0 + 1.0 : p->sigma_max;
    c->h_tol = isnan(p->h_tol) ? 1e-4 : p->h_tol;
    c->kv = (p->av && p->cfl_visc > 0.0) ? pow(N + 1.0, 3) * p->cfl / (8.0 * p->cfl_visc) : 0.0;
    DeviceMesh& m = c->m;
    m.N = N;
    m.n = n;
    m.K = K;
    m.nfaces = nfaces;
    m.nwall = nwall;
    m.KN = KN;
    m.KS = KS;
    m.g = g;
    m.r2g = 0.5 / g;
    cudaError_t e2 = cudaSuccess;
#define UP(dst, src)                                  \
    dst = dev_upload(c, src, e2);                     \
    if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: upload"); }
    UP(m.axx, axx) UP(m.axy, axy) UP(m.aex, aex) UP(m.aey, aey) UP(m.rJ, rJ) UP(m.wJ, wJ)
    UP(m.srcx, srcx) UP(m.srcy, srcy) UP(m.bn, bn) UP(m.nax, cfln) UP(m.rvol, rvol)
    UP(m.fwJ, fwJ) UP(m.fwJ2, fwJ2) UP(m.pm, pm) UP(m.ssx, ssx) UP(m.ssy, ssy)
    UP(m.f_im, f_im) UP(m.f_ip, f_ip) UP(m.f_tm, f_tm) UP(m.f_tp, f_tp) UP(m.f_nx, f_nx)
    UP(m.f_ny, f_ny) UP(m.f_js8, f_js) UP(m.f_sx8, f_sx) UP(m.f_sy8, f_sy) UP(m.f_bm, f_bm) UP(m.f_bp, f_bp)
    UP(m.s_nb, s_nb) UP(m.s_face, s_face) UP(m.s_nx, s_nx) UP(m.s_ny, s_ny) UP(m.s_rwa, s_rwa)
    UP(m.w_im, w_im) UP(m.w_tm, w_tm) UP(m.w_nx, w_nx) UP(m.w_ny, w_ny) UP(m.w_js, w_js)
#undef UP
    m.nae = nullptr;
    m.inst = nullptr;
    m.ninst = 1;
    if (inst) {
        std::vector<int32_t> iv(inst, inst + K);
        for (int32_t v : iv)
            if (v < 0 || v >= ninst) {
                free_all(c);
                delete c;
                return fail(SWE_ERR_ARG, "swe_create: instance index out of range");
            }
        m.inst = dev_upload(c, iv, e2);
        if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: upload"); }
        m.ninst = ninst;
    }
    Work& W = c->w;
#define AL(dst, count)                                \
    dst = dev_alloc(c, count, e2);                    \
    if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: allocation"); }
    AL(W.uv, 2 * KN) AL(W.Fout, 3 * KS) AL(W.Ustar, 2 * KS) AL(W.eps, K) AL(W.Kreg, 3 * KN)
    AL(W.Wn, 3 * KN) AL(W.R, 3 * KN) AL(W.part, 4 * RED_BLOCKS + 8) AL(W.dt, 3 * (size_t)m.ninst + 1)
    if (p->av) {
        AL(W.Fvt, 4 * KN) AL(W.Fvtr, 4 * KS) AL(W.Fvout, 2 * KS) AL(W.Lv, 2 * KN)
    }
#undef AL
    {
        void* q = nullptr;
        e2 = cudaMalloc(&q, 2 * sizeof(unsigned long long) * m.ninst + 16);
        if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: allocation"); }
        c->allocations.push_back(q);
        W.dtbits = static_cast<unsigned long long*>(q);
        W.status = reinterpret_cast<int*>(static_cast<char*>(q) + 2 * sizeof(unsigned long long) * m.ninst);
        if (shared_status) W.status = shared_status;
    }
    if (p->av) {
        void* q = nullptr;
        e2 = cudaMalloc(&q, sizeof(uint32_t) * ((size_t)K + 4));
        if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: allocation"); }
        c->allocations.push_back(q);
        W.touch = static_cast<uint32_t*>(q);
        cudaMemset(W.touch, 0, sizeof(uint32_t) * (size_t)K);
        q = nullptr;
        e2 = cudaMalloc(&q, sizeof(int) * ((size_t)K + 4));
        if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: allocation"); }
        c->allocations.push_back(q);
        W.vcount = static_cast<int*>(q);
        W.vlist = W.vcount + 4;
        cudaMemset(W.vcount, 0, sizeof(int) * ((size_t)K + 4));
    }
    c->side = KN >= (1LL << 20);
    if (c->side) {
        e2 = cudaStreamCreateWithFlags(&c->s_av, cudaStreamNonBlocking);
        if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
        if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&c->ev_first, cudaEventDisableTiming);
        if (e2 != cudaSuccess) { free_all(c); delete c; return cuda_fail(e2, "swe_create: stream"); }
    }
    if (!shared_status) cudaMemset(W.status, 0, sizeof(int));
    swe::prepare_volume(c);
    cudaMemset(W.eps, 0, sizeof(double) * K);
    // the viscous interface flux of solid-wall slots is zero and never rewritten
    if (p->av) cudaMemset(W.Fvout, 0, sizeof(double) * 2 * KS);
    e2 = cudaDeviceSynchronize();
    if (e2 != cudaSuccess) {
        free_all(c);
        delete c;
        return cuda_fail(e2, "swe_create");
    }
    *out = c;
    return SWE_OK;
}

}  // namespace swe

extern "C" int swe_create(int N, int K, const double* x, const double* y, const int32_t* EToE,
                          const int32_t* EToF, const int32_t* flip, const double* b, double g,
                          const swe_params* p, swe_ctx** out) {
    return swe::create_ctx(N, K, x, y, EToE, EToF, flip, b, g, p, nullptr, 1, nullptr, out);
}

extern "C" void swe_destroy(swe_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

// ---------------------------------------------------------------------------
// Right-hand side
// ---------------------------------------------------------------------------

namespace swe {

// The interface flux on s and, with AV, the smoothness indicator on the
// context's second stream: both read only W and its velocities. After the
// join, on s, the viscous fluxes (which read the BR1 interface values of the
// interface-flux kernel) and the viscous interface average. A step's first
// right-hand side also puts the step's own work on the second stream, after
// the indicator: the copy of the start state (save, for the rollback of a
// failed step) and the time step of W (dt_side; the viscous restriction
// reads the indicator's viscosities). ev_first marks its end, and the caller
// makes s wait for it before the first stage update, the first writer of W
// and reader of dt. Fork and joins are events, so all of it also runs
// inside a stream capture.
// Without c->side everything runs on s in the same order (same results).
void fluxes_and_viscosity(swe_ctx* c, const double* W, cudaStream_t s, const int* stop, bool save, bool dt_side) {
    const bool fork = c->side && (c->p.av || save || dt_side);
    cudaStream_t t = fork ? c->s_av : s;
    if (fork) {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(t, c->ev_fork, 0);
    }
    if (c->p.av) {
        launch_indicator(c, W, t, stop);
        if (fork) cudaEventRecord(c->ev_join, t);
    }
    if (save) launch_copy(c, W, c->w.Wn, 3 * c->m.KN, t, stop);
    if (dt_side) launch_dt(c, W, 0.0, t, stop);
    if (fork && (save || dt_side)) cudaEventRecord(c->ev_first, t);
    launch_surface(c, W, s, stop);
    if (c->p.av) {
        if (fork) cudaStreamWaitEvent(s, c->ev_join, 0);
        launch_visc_flux(c, W, s, stop);
        launch_visc_face(c, s, stop);
    }
}

void rhs_chain(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop, bool prim_done) {
    if (!prim_done) launch_prim(c, W, s, stop);
    fluxes_and_viscosity(c, W, s, stop, false, false);
    launch_volume(c, W, R, s, stop);
}

void step_once(swe_ctx* c, double* W, double dt, cudaStream_t s, const int* stop, bool save) {
    const bool adaptive = !(dt > 0.0);
    const double* dtd = adaptive ? c->w.dt : nullptr;
    const int stages = c->p.rk == 0 ? 5 : 3;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int stage = 0; stage < stages; ++stage) {
        if (stage == 0 && (adaptive || save)) {
            // the copy of the start state and its time step run on the
            // second stream beside the first right-hand side; the first
            // stage update waits for them
            fluxes_and_viscosity(c, W, s, stop, save, adaptive);
            launch_volume(c, W, c->w.R, s, stop);
            if (c->side) cudaStreamWaitEvent(s, c->ev_first, 0);
        } else {
            rhs_chain(c, W, c->w.R, s, stop, true);
        }
        if (c->p.rk == 0)
            launch_update(c, 1, W, kLsrkA[stage], kLsrkB[stage], dt, dtd, s, stop, true, stage + 1 < stages);
        else
            launch_update(c, 2, W, ca[stage], cb[stage], dt, dtd, s, stop, true);
    }
}

}  // namespace swe

namespace {

int check_launch(const char* where) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : cuda_fail(e, where);
}

}  // namespace

extern "C" int swe_rhs(swe_ctx* c, const double* W, double* R, void* stream) {
    if (!c || !W || !R) return fail(SWE_ERR_ARG, "swe_rhs: NULL argument");
    if (W == R) return fail(SWE_ERR_ARG, "swe_rhs: W and R must not overlap");
    swe::rhs_chain(c, W, R, (cudaStream_t)stream, nullptr, false);
    return check_launch("swe_rhs");
}

extern "C" int swe_limit(swe_ctx* c, double* W, void* stream) {
    if (!c || !W) return fail(SWE_ERR_ARG, "swe_limit: NULL argument");
    swe_params saved = c->p;
    c->p.limiter = 1;
    swe::launch_update(c, 0, W, 0.0, 0.0, 0.0, nullptr, (cudaStream_t)stream, nullptr, false);
    c->p = saved;
    return check_launch("swe_limit");
}

extern "C" int swe_max_dt(swe_ctx* c, const double* W, double* dt_cfl, double* dt_pos, void* stream) {
    if (!c || !W) return fail(SWE_ERR_ARG, "swe_max_dt: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    swe::launch_prim(c, W, s, nullptr);
    if (c->kv > 0.0) swe::launch_indicator(c, W, s, nullptr);  // the element viscosities of W (viscous restriction)
    swe::launch_dt(c, W, 0.0, s, nullptr);
    double h[4];
    cudaMemcpyAsync(h, c->w.dt, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_max_dt");
    if (dt_cfl) *dt_cfl = h[1];
    if (dt_pos) *dt_pos = h[2];
    return check_launch("swe_max_dt");
}

extern "C" int swe_step(swe_ctx* c, double* W, double dt, int nsteps, double* dt_last, void* stream) {
    if (!c || !W || nsteps < 0) return fail(SWE_ERR_ARG, "swe_step: bad argument");
    if (!(dt > 0.0) && !(c->p.cfl > 0.0)) return fail(SWE_ERR_ARG, "swe_step: dt <= 0 needs cfl > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int* stop = c->w.status;
    const long long n3 = 3 * c->m.KN;
    const bool adaptive = !(dt > 0.0);
    cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
    // Every stage update also writes the velocities of its new state, so only
    // the first stage of the call needs the primitives kernel.
    if (nsteps > 0) swe::launch_prim(c, W, s, stop);
    for (int st = 0; st < nsteps; ++st) swe::step_once(c, W, dt, s, stop);
    int rc = check_launch("swe_step");
    if (rc) return rc;
    int status = 0;
    double dth = dt;
    cudaMemcpyAsync(&status, c->w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (adaptive) cudaMemcpyAsync(&dth, c->w.dt, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_step");
    if (dt_last) *dt_last = dth;
    if (status) {
        cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
        cudaMemcpyAsync(W, c->w.Wn, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "swe_step: rollback");
        if (status & 2) return fail(SWE_ERR_NONFINITE, "swe_step: non-finite state; rolled back the failing step");
        return fail(SWE_ERR_NEG_MEAN, "swe_step: negative element mean water height; rolled back the failing step");
    }
    return SWE_OK;
}

extern "C" int swe_step_integrals(swe_ctx* c, double* W, double dt, int nsteps, double* dt_last, double* out4,
                                  void* stream) {
    if (!c || !W || !out4 || nsteps < 1) return fail(SWE_ERR_ARG, "swe_step_integrals: bad argument");
    if (!(dt > 0.0) && !(c->p.cfl > 0.0)) return fail(SWE_ERR_ARG, "swe_step_integrals: dt <= 0 needs cfl > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int* stop = c->w.status;
    cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
    swe::launch_prim(c, W, s, stop);
    for (int st = 0; st < nsteps; ++st) swe::step_once(c, W, dt, s, stop);
    swe::launch_reduce_dev(c, W, 2, true, s);
    int rc = check_launch("swe_step_integrals");
    if (rc) return rc;
    // integrals, step size and status in one copy
    double h[6];
    cudaMemcpyAsync(h, c->w.part + 4 * swe::RED_BLOCKS, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_step_integrals");
    const int status = (int)h[5];
    if (status) {
        cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
        cudaMemcpyAsync(W, c->w.Wn, 3 * c->m.KN * sizeof(double), cudaMemcpyDeviceToDevice, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "swe_step_integrals: rollback");
        if (status & 2) return fail(SWE_ERR_NONFINITE, "swe_step_integrals: non-finite state; rolled back the failing step");
        return fail(SWE_ERR_NEG_MEAN, "swe_step_integrals: negative element mean water height; rolled back the failing step");
    }
    for (int i = 0; i < 4; ++i) out4[i] = h[i];
    if (dt_last) *dt_last = dt > 0.0 ? dt : h[4];
    return SWE_OK;
}

extern "C" int swe_step_async(swe_ctx* c, double* W, double dt, int nsteps, double* out6, void* stream) {
    if (!c || !W || !out6 || nsteps < 1) return fail(SWE_ERR_ARG, "swe_step_async: bad argument");
    if (!(dt > 0.0) && !(c->p.cfl > 0.0)) return fail(SWE_ERR_ARG, "swe_step_async: dt <= 0 needs cfl > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int* stop = c->w.status;
    cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
    swe::launch_prim(c, W, s, stop);
    for (int st = 0; st < nsteps; ++st) swe::step_once(c, W, dt, s, stop);
    swe::launch_restore(c, W, s);
    swe::launch_reduce_dev(c, W, 2, true, s, out6);
    return check_launch("swe_step_async");
}

// ---------------------------------------------------------------------------
// Launch-shape tuning
// ---------------------------------------------------------------------------

namespace swe {

namespace {

// Milliseconds of `reps` launches by fn on s, after one untimed launch.
template <class F>
float time_launches(cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int reps, F fn) {
    fn();
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) return INFINITY;
    float ms = INFINITY;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

}  // namespace

int autotune_ctx(swe_ctx* c, const double* W, cudaStream_t s) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(e, "swe_autotune");
    }
    const bool timing = c->timing;
    c->timing = false;
    constexpr int kReps = 5;
    // A switch away from the default shape must gain more than the noise.
    constexpr float kMargin = 0.98f;
    // The volume kernel needs the interface fluxes, viscosities and gradients
    // of W: one right-hand side into the scratch buffer provides them.
    rhs_chain(c, W, c->w.R, s, nullptr, false);
    int best_v = 128;
    c->vol_tpb = 128;
    float t_best = time_launches(s, a, b, kReps, [&] { launch_volume(c, W, c->w.R, s, nullptr); });
    for (int tpb : {64, 256}) {
        if (!volume_shape_valid(c->m.N, tpb)) continue;
        c->vol_tpb = tpb;
        const float t = time_launches(s, a, b, kReps, [&] { launch_volume(c, W, c->w.R, s, nullptr); });
        if (t < kMargin * t_best) {
            t_best = t;
            best_v = tpb;
        }
    }
    c->vol_tpb = best_v;
    // Stage update (2N-storage stage with a = b = 0: the register takes R, the
    // state is only limited) on a scratch copy of W.
    launch_copy(c, W, c->w.Wn, 3 * c->m.KN, s, nullptr);
    int best_u = 4;
    c->upd_wpb = 4;
    auto upd = [&] { launch_update(c, 1, c->w.Wn, 0.0, 0.0, 0.0, nullptr, s, nullptr, false); };
    t_best = time_launches(s, a, b, kReps, upd);
    for (int wpb : {2, 8}) {
        c->upd_wpb = wpb;
        const float t = time_launches(s, a, b, kReps, upd);
        if (t < kMargin * t_best) {
            t_best = t;
            best_u = wpb;
        }
    }
    c->upd_wpb = best_u;
    c->timing = timing;
    e = cudaStreamSynchronize(s);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : cuda_fail(e, "swe_autotune");
}

}  // namespace swe

extern "C" int swe_autotune(swe_ctx* c, const double* W, void* stream) {
    if (!c || !W) return fail(SWE_ERR_ARG, "swe_autotune: NULL argument");
    return swe::autotune_ctx(c, W, (cudaStream_t)stream);
}

extern "C" int swe_get_tuning(const swe_ctx* c, int* vol_threads, int* upd_warps) {
    if (!c) return fail(SWE_ERR_ARG, "swe_get_tuning: NULL context");
    if (vol_threads) *vol_threads = c->vol_tpb;
    if (upd_warps) *upd_warps = c->upd_wpb;
    return SWE_OK;
}

extern "C" int swe_set_tuning(swe_ctx* c, int vol_threads, int upd_warps) {
    if (!c) return fail(SWE_ERR_ARG, "swe_set_tuning: NULL context");
    if (!swe::volume_shape_valid(c->m.N, vol_threads))
        return fail(SWE_ERR_ARG, "swe_set_tuning: volume threads per block must be 64, 128 or 256 "
                                 "(and the shape must fit the shared memory at this degree)");
    if (upd_warps != 2 && upd_warps != 4 && upd_warps != 8)
        return fail(SWE_ERR_ARG, "swe_set_tuning: update warps per block must be 2, 4 or 8");
    c->vol_tpb = vol_threads;
    c->upd_wpb = upd_warps;
    return SWE_OK;
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------

namespace {

void dev_free(swe_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocations.size(); ++i)
        if (c->allocations[i] == p) {
            c->allocations.erase(c->allocations.begin() + i);
            break;
        }
    cudaFree(p);
}

// Step records: nslots sets of the stage data of one step (stage inputs,
// pre-limit results, viscosities, limiter plans). Replaces earlier records.
int ensure_slots(swe_ctx* c, int nslots) {
    swe::AdjWork& A = c->adj;
    if (A.slots >= nslots) return SWE_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint: synchronise");
    dev_free(c, A.Xs);
    dev_free(c, A.Ys);
    dev_free(c, A.Es);
    dev_free(c, A.act);
    dev_free(c, A.amin);
    A.Xs = A.Ys = A.Es = nullptr;
    A.act = A.cut = nullptr;
    A.amin = nullptr;
    A.slots = 0;
    const size_t KN = c->m.KN, K = c->m.K, S = (size_t)A.stages * nslots;
    A.Xs = dev_alloc(c, S * 3 * KN, e);
    if (e == cudaSuccess) A.Ys = dev_alloc(c, S * 3 * KN, e);
    if (e == cudaSuccess) A.Es = dev_alloc(c, S * K, e);
    void* q = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&q, S * (K + KN) + 16);
    if (e == cudaSuccess) {
        c->allocations.push_back(q);
        A.act = static_cast<uint8_t*>(q);
        A.cut = A.act + S * K;
        q = nullptr;
        e = cudaMalloc(&q, sizeof(int32_t) * S * K + 16);
    }
    if (e == cudaSuccess) {
        c->allocations.push_back(q);
        A.amin = static_cast<int32_t*>(q);
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint: step records");
    A.slots = nslots;
    return SWE_OK;
}

int ensure_adjoint(swe_ctx* c) {
    swe::AdjWork& A = c->adj;
    if (A.ready) return SWE_OK;
    const size_t KN = c->m.KN, KS = c->m.KS;
    cudaError_t e = cudaSuccess;
#define ADJ_AL(dst, count)                                                  \
    dst = dev_alloc(c, count, e);                                           \
    if (e != cudaSuccess) return cuda_fail(e, "adjoint: allocation");
    ADJ_AL(A.Ga, 3 * KN) ADJ_AL(A.Guv, 2 * KN) ADJ_AL(A.Gsl, 4 * KS) ADJ_AL(A.Gfo, 3 * KS)
    ADJ_AL(A.GUs, 2 * KS) ADJ_AL(A.Gfvt, 4 * KN) ADJ_AL(A.Gfvo, 2 * KS) ADJ_AL(A.Gfvtr, 4 * KS)
    ADJ_AL(A.Gsrc, 2 * KN) ADJ_AL(A.Gsrc_acc, 2 * KN) ADJ_AL(A.Khb, 3 * KN) ADJ_AL(A.Rb, 3 * KN)
    ADJ_AL(A.Wnb, 3 * KN) ADJ_AL(A.Ws, 3 * KN)
#undef ADJ_AL
    A.stages = 5;  // stages of the longer scheme
    if (int rc = ensure_slots(c, 1)) return rc;
    // wall slots of the side-node viscous cotangents are never written
    e = cudaMemset(A.Gfvtr, 0, sizeof(double) * 4 * KS);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint: initialisation");
    A.ready = true;
    return SWE_OK;
}

int adjoint_args(swe_ctx* c, const void* W, const void* cot, const void* Wbar, const char* where) {
    if (!c || !W || !cot || !Wbar) return fail(SWE_ERR_ARG, std::string(where) + ": NULL argument");
    if (c->p.volume != 0)
        return fail(SWE_ERR_ARG, std::string(where) + ": the adjoint covers the split (entropy-stable) form only");
    return ensure_adjoint(c);
}

}  // namespace

// The forward quantities the reverse sweep reads at W: velocities and, with
// the viscosity on, the BR1 interface values, the element viscosities (unless
// given) and the list of viscous elements. The interface flux, the volume term
// and the viscous interface average themselves are not needed.
static void adjoint_prerequisites(swe_ctx* c, const double* W, cudaStream_t s, bool eps_given) {
    swe::launch_prim(c, W, s, nullptr);
    if (!c->p.av) return;
    swe::launch_ustar(c, s);
    if (!eps_given) swe::launch_av(c, W, s, nullptr);
    else swe::launch_visc_list(c, s);  // the list of the recorded viscosities
}

extern "C" int swe_rhs_adjoint(swe_ctx* c, const double* W, const double* Rbar, double* Wbar, double* bbar,
                               void* stream) {
    if (int rc = adjoint_args(c, W, Rbar, Wbar, "swe_rhs_adjoint")) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    adjoint_prerequisites(c, W, s, false);
    swe::launch_rhs_adjoint(c, W, Rbar, Wbar, bbar, s);
    return check_launch("swe_rhs_adjoint");
}

namespace {

// One step of size dt on W (advanced in place) with the stage inputs, the
// pre-limit stage results, the viscosities and the limiter's plans stored in
// record `slot`. The same kernels and arithmetic as swe_step's, so W1 is
// bitwise swe_step's result (the limiter runs separately to record its plan,
// with the fused update's arithmetic). On failure W is restored from the
// record (its first stage input) and the status error is returned.
int record_step(swe_ctx* c, double* W, double dt, int slot, cudaStream_t s, const char* where) {
    swe::AdjWork& A = c->adj;
    const long long KN = c->m.KN, K = c->m.K, n3 = 3 * KN;
    const int stages = c->p.rk == 0 ? 5 : 3, S = A.stages;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const int lim = c->p.limiter;
    double* Xs = A.Xs + (size_t)slot * S * n3;
    double* Ys = A.Ys + (size_t)slot * S * n3;
    double* Es = A.Es + (size_t)slot * S * K;
    uint8_t* act = A.act + (size_t)slot * S * K;
    uint8_t* cut = A.cut + (size_t)slot * S * KN;
    int32_t* amin = A.amin + (size_t)slot * S * K;
    cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
    if (c->p.rk == 1) cudaMemcpyAsync(c->w.Wn, W, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    swe::launch_prim(c, W, s, nullptr);
    for (int st = 0; st < stages; ++st) {
        cudaMemcpyAsync(Xs + st * n3, W, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        swe::rhs_chain(c, W, c->w.R, s, nullptr, true);
        cudaMemcpyAsync(Es + st * K, c->w.eps, K * sizeof(double), cudaMemcpyDeviceToDevice, s);
        c->p.limiter = 0;  // the limiter runs separately, recording its plan
        if (c->p.rk == 0)
            swe::launch_update(c, 1, W, kLsrkA[st], kLsrkB[st], dt, nullptr, s, nullptr, true);
        else
            swe::launch_update(c, 2, W, ca[st], cb[st], dt, nullptr, s, nullptr, true);
        c->p.limiter = lim;
        cudaMemcpyAsync(Ys + st * n3, W, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (lim) swe::launch_limit_record(c, W, act + st * K, amin + st * K, cut + st * KN, s);
    }
    if (int rc = check_launch(where)) return rc;
    int status = 0;
    cudaMemcpyAsync(&status, c->w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, where);
    if (status) {
        cudaMemcpyAsync(W, Xs, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
        return fail((status & 2) ? SWE_ERR_NONFINITE : SWE_ERR_NEG_MEAN,
                    std::string(where) + ": the step failed (status bits set); W restored");
    }
    return SWE_OK;
}

// The reverse sweep of the step recorded in `slot` (size dt): Wbar becomes
// the cotangent of the step's start state; the bathymetry cotangent is added
// to bbar (nullable).
int reverse_step(swe_ctx* c, int slot, double dt, double* Wbar, double* bbar, cudaStream_t s, const char* where) {
    swe::AdjWork& A = c->adj;
    const long long KN = c->m.KN, K = c->m.K, n3 = 3 * KN;
    const int stages = c->p.rk == 0 ? 5 : 3, S = A.stages;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const double* Xs = A.Xs + (size_t)slot * S * n3;
    const double* Ys = A.Ys + (size_t)slot * S * n3;
    const double* Es = A.Es + (size_t)slot * S * K;
    const uint8_t* act = A.act + (size_t)slot * S * K;
    const uint8_t* cut = A.cut + (size_t)slot * S * KN;
    const int32_t* amin = A.amin + (size_t)slot * S * K;
    cudaMemsetAsync(A.Khb, 0, n3 * sizeof(double), s);
    if (c->p.rk == 1) cudaMemsetAsync(A.Wnb, 0, n3 * sizeof(double), s);
    // the stages' source-coefficient cotangents are summed and carried to
    // bbar once, after the sweep
    if (bbar) cudaMemsetAsync(A.Gsrc_acc, 0, 2 * KN * sizeof(double), s);
    for (int st = stages - 1; st >= 0; --st) {
        const double a = c->p.rk == 0 ? kLsrkA[st] : ca[st], b = c->p.rk == 0 ? kLsrkB[st] : cb[st];
        swe::launch_update_adjoint(c, c->p.rk == 0 ? 1 : 2, Wbar, Ys + st * n3, act + st * K, amin + st * K,
                                   cut + st * KN, A.Khb, A.Rb, A.Wnb, a, b, dt, s);
        const double* X = Xs + st * n3;
        cudaMemcpyAsync(c->w.eps, Es + st * K, K * sizeof(double), cudaMemcpyDeviceToDevice, s);
        adjoint_prerequisites(c, X, s, true);
        swe::launch_rhs_adjoint(c, X, A.Rb, Wbar, bbar, s, true);
    }
    if (bbar) swe::launch_src_adjoint(c, A.Gsrc_acc, bbar, s);
    if (c->p.rk == 1) swe::launch_axpy(c, n3, 1.0, A.Wnb, Wbar, s);
    if (int rc = check_launch(where)) return rc;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, where);
    return SWE_OK;
}

}  // namespace

extern "C" int swe_step_adjoint(swe_ctx* c, const double* W0, double dt, double* Wbar, double* bbar,
                                void* stream) {
    if (int rc = adjoint_args(c, W0, W0, Wbar, "swe_step_adjoint")) return rc;
    if (!(dt > 0.0)) return fail(SWE_ERR_ARG, "swe_step_adjoint: dt must be the step's positive size");
    cudaStream_t s = (cudaStream_t)stream;
    swe::AdjWork& A = c->adj;
    // the step is recomputed from a copy of W0, recorded in slot 0
    cudaMemcpyAsync(A.Ws, W0, 3 * c->m.KN * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (int rc = record_step(c, A.Ws, dt, 0, s, "swe_step_adjoint"))
        return rc == SWE_ERR_CUDA ? rc : fail(SWE_ERR_NEG_MEAN, "swe_step_adjoint: the recomputed step failed");
    return reverse_step(c, 0, dt, Wbar, bbar, s, "swe_step_adjoint");
}

extern "C" int swe_adjoint_slots(swe_ctx* c, int nslots) {
    if (!c || nslots < 1) return fail(SWE_ERR_ARG, "swe_adjoint_slots: bad argument");
    if (c->p.volume != 0)
        return fail(SWE_ERR_ARG, "swe_adjoint_slots: the adjoint covers the split (entropy-stable) form only");
    if (int rc = ensure_adjoint(c)) return rc;
    return ensure_slots(c, nslots);
}

extern "C" int swe_step_record(swe_ctx* c, double* W, double dt, int slot, void* stream) {
    if (int rc = adjoint_args(c, W, W, W, "swe_step_record")) return rc;
    if (!(dt > 0.0)) return fail(SWE_ERR_ARG, "swe_step_record: dt must be positive");
    if (slot < 0 || slot >= c->adj.slots) return fail(SWE_ERR_ARG, "swe_step_record: slot out of range");
    return record_step(c, W, dt, slot, (cudaStream_t)stream, "swe_step_record");
}

extern "C" int swe_step_adjoint_recorded(swe_ctx* c, int slot, double dt, double* Wbar, double* bbar,
                                         void* stream) {
    if (int rc = adjoint_args(c, Wbar, Wbar, Wbar, "swe_step_adjoint_recorded")) return rc;
    if (!(dt > 0.0)) return fail(SWE_ERR_ARG, "swe_step_adjoint_recorded: dt must be the step's positive size");
    if (slot < 0 || slot >= c->adj.slots) return fail(SWE_ERR_ARG, "swe_step_adjoint_recorded: slot out of range");
    return reverse_step(c, slot, dt, Wbar, bbar, (cudaStream_t)stream, "swe_step_adjoint_recorded");
}

extern "C" int swe_gauge_misfit(swe_ctx* c, const double* W, int ngauge, const int32_t* elem, const double* wts,
                                const double* target, double* values, double* loss, double* Wbar, void* stream) {
    if (!c || !W || ngauge < 0 || (ngauge > 0 && (!elem || !wts)))
        return fail(SWE_ERR_ARG, "swe_gauge_misfit: bad argument");
    if (ngauge == 0) return SWE_OK;
    swe::launch_gauge(c, W, ngauge, elem, wts, target, values, loss, Wbar, (cudaStream_t)stream);
    return check_launch("swe_gauge_misfit");
}

// ---------------------------------------------------------------------------
// Diagnostics, status, timing
// ---------------------------------------------------------------------------

extern "C" int swe_mass(swe_ctx* c, const double* W, double* out3, void* stream) {
    if (!c || !W || !out3) return fail(SWE_ERR_ARG, "swe_mass: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    double h[4];
    swe::launch_reduce(c, W, 0, h, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_mass");
    for (int i = 0; i < 3; ++i) out3[i] = h[i];
    return check_launch("swe_mass");
}

extern "C" int swe_entropy(swe_ctx* c, const double* W, double* E, void* stream) {
    if (!c || !W || !E) return fail(SWE_ERR_ARG, "swe_entropy: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    double h[4];
    swe::launch_prim(c, W, s, nullptr);  // the kinetic energy reads the velocities
    swe::launch_reduce(c, W, 1, h, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_entropy");
    *E = h[3];
    return check_launch("swe_entropy");
}

extern "C" int swe_entropy_rate(swe_ctx* c, const double* W, double* rate, double* scale, void* stream) {
    if (!c || !W || !rate) return fail(SWE_ERR_ARG, "swe_entropy_rate: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    swe::rhs_chain(c, W, c->w.R, s, nullptr, false);
    double h[4];
    swe::launch_rate(c, W, c->w.R, h, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_entropy_rate");
    *rate = h[0];
    if (scale) *scale = h[1];
    return check_launch("swe_entropy_rate");
}

extern "C" int swe_integrals(swe_ctx* c, const double* W, double* out4, void* stream) {
    if (!c || !W || !out4) return fail(SWE_ERR_ARG, "swe_integrals: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    double h[4];
    swe::launch_prim(c, W, s, nullptr);  // the kinetic energy reads the velocities
    swe::launch_reduce(c, W, 2, h, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_integrals");
    for (int i = 0; i < 4; ++i) out4[i] = h[i];
    return check_launch("swe_integrals");
}

extern "C" int swe_get_epsilon(swe_ctx* c, double* eps, void* stream) {
    if (!c || !eps) return fail(SWE_ERR_ARG, "swe_get_epsilon: NULL argument");
    cudaError_t e = cudaMemcpyAsync(eps, c->w.eps, sizeof(double) * c->m.K, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? SWE_OK : cuda_fail(e, "swe_get_epsilon");
}

extern "C" int swe_status(swe_ctx* c, int* bits, void* stream) {
    if (!c || !bits) return fail(SWE_ERR_ARG, "swe_status: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    cudaMemcpyAsync(&v, c->w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemsetAsync(c->w.status, 0, sizeof(int), s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "swe_status");
    *bits = v;
    return SWE_OK;
}

extern "C" int swe_timing(swe_ctx* c, int on) {
    if (!c) return fail(SWE_ERR_ARG, "swe_timing: NULL context");
    if (on && c->ev.empty()) {
        c->ev.resize(2 * kEventPairs);
        c->ev_class.assign(kEventPairs, -1);
        for (auto& e : c->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(r, "swe_timing");
        }
    }
    c->timing = on != 0;
    c->timing_mask = ~0u;
    c->ev_used = 0;
    return SWE_OK;
}

extern "C" int swe_timing_classes(swe_ctx* c, unsigned mask) {
    if (!c) return fail(SWE_ERR_ARG, "swe_timing_classes: NULL context");
    const int rc = swe_timing(c, mask != 0u);
    if (rc) return rc;
    c->timing_mask = mask;
    return SWE_OK;
}

extern "C" int swe_timing_read(swe_ctx* c, int which, double* ms, int64_t* launches) {
    if (!c || !ms || !launches) return fail(SWE_ERR_ARG, "swe_timing_read: NULL argument");
    double tot = 0.0;
    int64_t cnt = 0;
    for (int i = 0; i < c->ev_used; ++i) {
        if (c->ev_class[i] != which) continue;
        cudaError_t e = cudaEventSynchronize(c->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "swe_timing_read");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "swe_timing_read");
        tot += t;
        ++cnt;
    }
    *ms = tot;
    *launches = cnt;
    return SWE_OK;
}

extern "C" int64_t swe_launches(const swe_ctx* c) { return c ? c->launches : 0; }

extern "C" int swe_info(const swe_ctx* c, int* N, int* K, int* nfaces) {
    if (!c) return fail(SWE_ERR_ARG, "swe_info: NULL context");
    if (N) *N = c->m.N;
    if (K) *K = c->m.K;
    if (nfaces) *nfaces = c->m.nfaces;
    return SWE_OK;
}

extern "C" const char* swe_last_error(void) { return g_last_error.c_str(); }
