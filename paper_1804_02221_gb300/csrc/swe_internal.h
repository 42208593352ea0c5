// Internal declarations of the swedg library (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/swedg.h"

namespace swe {

constexpr int NMAX = SWE_NMAX;
constexpr int NFACE = 4;
// Blocks of the fixed-grid reductions; the work buffer `part` holds their
// partials [4][RED_BLOCKS] followed by the results.
constexpr int RED_BLOCKS = 608;

// Basis of degree N on LGL nodes (Sec. 2.2) and the inverse Vandermonde
// matrix of the normalised Legendre polynomials (App. A), row-major n x n.
struct Basis {
    int N = 0;
    std::vector<double> xi, w, D, Vinv;
};
Basis make_basis(int N);

// Offsets of degree N's tables inside the packed constant arrays.
constexpr int mat_offset(int N) {  // sum_{M<N} (M+1)^2
    int s = 0;
    for (int M = 1; M < N; ++M) s += (M + 1) * (M + 1);
    return s;
}
constexpr int vec_offset(int N) {  // sum_{M<N} (M+1)
    int s = 0;
    for (int M = 1; M < N; ++M) s += M + 1;
    return s;
}
constexpr int MAT_TOTAL = mat_offset(NMAX + 1);
constexpr int VEC_TOTAL = vec_offset(NMAX + 1);

// Packed tables of all degrees 1..NMAX (D, Vinv, w), filled once per process.
struct Tables {
    double D[MAT_TOTAL];
    double Vinv[MAT_TOTAL];
    double w[VEC_TOTAL];
};
const Tables& tables();

// Parameters of the element viscosity (App. A).
struct EpsParams {
    double eps0, smin, smax;
    double rmin, rmax;  // 10^smin, 10^smax
};

// Kernel classes for timing.
enum KernelClass {
    KC_VOLUME = 0,
    KC_FACE = 1,
    KC_PRIM = 2,
    KC_AV = 3,
    KC_VFACE = 4,
    KC_UPDATE = 5,
    KC_DT = 6,
    KC_REDUCE = 7,
    KC_ADJ = 8,
    KC_ADJ_VOL = 9,  // the adjoint of the volume kernel (the other adjoint kernels: KC_ADJ)
    KC_COUNT = 10
};

// Degrees whose split-form volume kernel sums the pressure parts of the
// pair fluxes per node and starts those sums from the bathymetry source (the
// host stores the source as DeviceMesh::ssx, ssy for them).
constexpr bool pressure_sums_degree(int N) {
    return N >= 1;
}

// Device-side data of one context. Nodal arrays are [K][n][n] planes,
// side arrays [K][4][n] (element side node), face arrays [nfaces][n].
struct DeviceMesh {
    int N, n, K, nfaces;
    long long KN;       // K*n*n
    long long KS;       // K*4*n
    double g;
    double r2g;         // 0.5 / g (the interface dissipation's eigenvalue scale)
    // per node
    const double* axx;  // contravariant xi vector (y_eta, -x_eta)
    const double* axy;
    const double* aex;  // contravariant eta vector (-y_xi, x_xi)
    const double* aey;
    const double* rJ;   // 1/J
    const double* wJ;   // w_i w_j J
    const double* srcx; // -(g/2) gamma_x / J  (source of the x momentum is h*srcx)
    const double* srcy; // -(g/2) gamma_y / J
    const double* bn;   // bathymetry
    const double* nax;  // |a_xi| / J
    const double* nae;  // |a_eta| / J
    const double* rvol; // [K] 1 / sum_ij w_i w_j J
    const double* fwJ;  // -1 / (w_i w_j J)
    const double* fwJ2; // -2 / (w_i w_j J) (the split volume kernel's mass row; empty otherwise)
    const double* ssx;  // w_i w_j gamma_x / 4: h srcx = -(2g h) ssx / (w_i w_j J) (the split
    const double* ssy;  //   volume kernel's pressure sums, pressure_sums_degree; empty otherwise)
    // Pair constants of the volume kernel, [K][2 directions][N(N+1)/2 pairs][n lines][2]:
    // w_i w_j D_iq / 4 * (a_i + a_q) for the pair (i, q), i < q, of each line; the
    // two components of a line are adjacent (one 16-byte load).
    const double* pm;
    // per unique face node
    const int32_t* f_im;   // owner node id (k*n*n + j*n + i)
    const int32_t* f_ip;   // neighbour node id
    const int32_t* f_tm;   // owner side slot ((k*4+f)*n + p)
    const int32_t* f_tp;   // neighbour side slot
    const double* f_nx;    // owner outward unit normal
    const double* f_ny;
    const double* f_js8;   // surface Jacobian |outward unscaled normal| / 8
    const double* f_sx8;   // owner outward unscaled normal / 8 (unit normal times f_js8)
    const double* f_sy8;
    const double* f_bm;    // bathymetry on both sides
    const double* f_bp;
    // per element side node
    const int32_t* s_nb;   // node id of the neighbour's matching node (-1: solid wall)
    const int32_t* s_face; // unique face node (index into the f_* arrays) of the slot (-1: solid wall)
    const double* s_nx;    // own outward unit normal
    const double* s_ny;
    const double* s_rwa;   // 1/(omega_0 a), a = J/Jsurf (Lemma PosPres)
    // per solid-wall face node (nwall wall faces): own node id, own side
    // slot, outward unit normal, surface Jacobian
    int nwall;
    const int32_t* w_im;
    const int32_t* w_tm;
    const double* w_nx;
    const double* w_ny;
    const double* w_js;
    // ensembles: instance of every element (nullable: one instance), count
    const int32_t* inst;
    int ninst;
};

struct Work {
    double* uv;     // [2][KN] velocities
    double* Fout;   // [3][KS] outward interface flux (x Jsurf)
    double* Ustar;  // [2][KS] BR1 interface values
    double* Fvt;    // [4][KN] contravariant viscous fluxes Ft2, Ft3, Gt2, Gt3
    double* Fvtr;   // [4][KS] physical viscous fluxes at side nodes F2, F3, G2, G3
                    // (written for viscous elements only; read only for them)
    double* Fvout;  // [2][KS] outward viscous interface flux
    double* Lv;     // [2][KN] volume part of the viscous divergence, sum_q D_iq F~v + D_jq G~v
                    // (components 2, 3; written and read for viscous elements only)
    uint32_t* touch; // [K] bit f: a viscous flux crosses side f (the element or its face-f neighbour is viscous)
    int* vlist;     // [K] viscous elements (AV indicator), vcount of them
    int* vcount;
    double* eps;    // [K]
    double* Kreg;   // [3][KN] 2N-storage register
    double* Wn;     // [3][KN] state at the start of a step
    double* R;      // [3][KN] right-hand side of the current stage
    double* part;   // reduction partials [4][RED_BLOCKS], then the results (4 + dt + status)
    double* dt;     // [3][ninst]: dt in use, dt_cfl, dt_pos of every instance
    unsigned long long* dtbits;  // [ninst][2]: max of lambda/J, max of inverse positivity dt
    int* status;    // [1] status bits (shared by the groups of an ensemble)
};

// Buffers of the adjoint (allocated at the first adjoint call).
struct AdjWork {
    bool ready = false;
    int stages = 0;
    double* Ga = nullptr;     // [3][KN] node cotangents of (h, hu, hv), direct paths
    double* Guv = nullptr;    // [2][KN] node cotangents of (u, v)
    double* Gsl = nullptr;    // [4][KS] side-slot cotangents of (h, u, v, b)
    double* Gfo = nullptr;    // [3][KS] interface-flux cotangents
    double* GUs = nullptr;    // [2][KS] BR1 interface-value cotangents
    double* Gfvt = nullptr;   // [4][KN] contravariant viscous-flux cotangents
    double* Gfvo = nullptr;   // [2][KS] viscous interface-flux cotangents
    double* Gfvtr = nullptr;  // [4][KS] side-node viscous-flux cotangents (wall slots stay 0)
    double* Gsrc = nullptr;   // [2][KN] source-coefficient cotangents
    double* Gsrc_acc = nullptr;  // [2][KN] their sum over the stages of a step adjoint
    double* Khb = nullptr;    // [3][KN] 2N-storage register cotangent
    double* Rb = nullptr;     // [3][KN] right-hand-side cotangent of a stage
    double* Wnb = nullptr;    // [3][KN] step-start cotangent (SSP)
    double* Ws = nullptr;     // [3][KN] recomputed state
    // step records, [slots] of: (the stage data of one recorded step)
    int slots = 0;
    double* Xs = nullptr;     // [slots][stages][3][KN] stage inputs
    double* Ys = nullptr;     // [slots][stages][3][KN] pre-limit stage results
    double* Es = nullptr;     // [slots][stages][K] element viscosities
    uint8_t* act = nullptr;   // [slots][stages][K] limited elements
    int32_t* amin = nullptr;  // [slots][stages][K] node of the minimum
    uint8_t* cut = nullptr;   // [slots][stages][KN] h_tol cut
};

}  // namespace swe

struct swe_ctx {
    int device = 0;
    int sms = 152;  // multiprocessors of the device (grid size of persistent kernels)
    swe_params p{};
    double sigma_min = 0, sigma_max = 0, h_tol = 1e-4;
    swe::DeviceMesh m{};
    swe::Work w{};
    swe::AdjWork adj{};
    std::vector<void*> allocations;
    int64_t launches = 0;
    // launch shapes (swe_autotune): volume threads per block, update warps per block
    int vol_tpb = 128;
    int upd_wpb = 4;
    // the smoothness indicator of a right-hand side (and a step's copy of its
    // start state and its time step) run on this second stream beside the
    // interface flux, forked from the caller's stream by ev_fork and joined
    // back by ev_join (indicator) and ev_first (copy and time step, before
    // the first stage update); only on meshes of at least 2^20 nodes (side):
    // on smaller ones the launches, not the kernels, set the pace, and the
    // fork and joins cost more than the overlap gains
    bool side = false;
    cudaStream_t s_av = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_first = nullptr;
    // viscous time-step factor kv = (N+1)^3 cfl / (8 cfl_visc); 0 = the paper's rule
    double kv = 0.0;
    // timing: on, and the kernel classes whose launches get events (bit c = class c)
    bool timing = false;
    unsigned timing_mask = ~0u;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_class;
    int ev_used = 0;
};

namespace swe {

// Kernel launchers (one translation unit per family).
void init_tables_volume();
void init_tables_face();
void init_tables_av();
void init_tables_volume_std();
void init_tables_adjoint();

// Per-process kernel attributes of the context's degree (called at creation,
// so that later launches, also inside a stream capture, change no state).
void prepare_volume(swe_ctx* c);
// Volume-kernel launch shapes (threads per block 64, 128, 256; one
// translation unit each). launch returns false if the shape does not fit the
// degree (then nothing is launched); prepare returns whether it fits.
void volume_init_64();
void volume_init_128();
void volume_init_256();
bool volume_prepare_64(int N);
bool volume_prepare_128(int N);
bool volume_prepare_256(int N);
bool volume_launch_64(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop);
bool volume_launch_128(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop);
bool volume_launch_256(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop);
bool volume_shape_valid(int N, int tpb);

void launch_prim(swe_ctx* c, const double* W, cudaStream_t s, const int* stop);
void launch_surface(swe_ctx* c, const double* W, cudaStream_t s, const int* stop);
// Volume term of the context's form (p.volume): the split-form kernel in the
// tuned launch shape, or the standard-form kernel.
void launch_volume(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop);
void launch_volume_std(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop);
EpsParams eps_params(const swe_ctx* c);
// The element viscosities of W and the list of viscous elements (indicator).
void launch_indicator(swe_ctx* c, const double* W, cudaStream_t s, const int* stop);
// For the listed viscous elements: the BR1 gradients (from the interface
// values in w.Ustar), viscous fluxes and the volume part of their divergence.
void launch_visc_flux(swe_ctx* c, const double* W, cudaStream_t s, const int* stop);
// Both of the above.
void launch_av(swe_ctx* c, const double* W, cudaStream_t s, const int* stop);
// The list of viscous elements (w.vlist, w.vcount) from the viscosities in w.eps.
void launch_visc_list(swe_ctx* c, cudaStream_t s);
void launch_visc_face(swe_ctx* c, cudaStream_t s, const int* stop);
void launch_ustar(swe_ctx* c, cudaStream_t s);
// mode 0: limiter only; 1: 2N-storage stage Kh = a Kh + R, W += (b dt) Kh
// (the register holds K/dt); 2: SSP stage W = a Wn + b (W + dt R).
// write_uv: also write the velocities of the new state into the work buffer;
// write_reg (mode 1): store the register (not needed after the last stage).
void launch_update(swe_ctx* c, int mode, double* W, double a, double b, double dt_host,
                   const double* dt_dev, cudaStream_t s, const int* stop, bool write_uv, bool write_reg = true);
void launch_dt(swe_ctx* c, const double* W, double dt_fixed, cudaStream_t s, const int* stop);
void launch_copy(swe_ctx* c, const double* src, double* dst, long long count, cudaStream_t s,
                 const int* stop);
// sum J w w W (what = 0), sum J w w e(W) (what = 1) or all four (what = 2)
// into host_out[4] (asynchronous copy).
void launch_reduce(swe_ctx* c, const double* W, int what, double* host_out, cudaStream_t s);
// The same into the device results w.part[4 * RED_BLOCKS + c] (or dst[c],
// when given); pack: also the step size in use (+4) and the status word (+5).
void launch_reduce_dev(swe_ctx* c, const double* W, int what, bool pack, cudaStream_t s,
                       double* dst = nullptr);
// W = the state saved at the start of the step (w.Wn) where the status word
// is set: the rollback of a failed step without a host synchronisation.
void launch_restore(swe_ctx* c, double* W, cudaStream_t s);
// Per-instance (mass, momenta, entropy) of an ensemble group into device
// out[4 * ninst]; ebeg (device, ninst + 1) holds the element ranges.
void launch_reduce_inst(swe_ctx* c, const double* W, const long long* ebeg, double* out, cudaStream_t s);
// host_out[0] = sum J w w q(W).R, host_out[1] = sum J w w |q_c R_c| (asynchronous copy)
void launch_rate(swe_ctx* c, const double* W, const double* R, double* host_out, cudaStream_t s);

// One right-hand side R(W) (prim_done: the velocities of W are already in
// the work buffer, written by the previous stage update).
void rhs_chain(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop, bool prim_done);
// One Runge-Kutta step of W (dt <= 0: adaptive, from the device time step of
// every instance). Expects the velocities of W in the work buffer and leaves
// those of the new state there. save: first copy the start state to w.Wn
// (callers that run several contexts concurrently on one status word make
// all those copies before any of the steps, so that a failure in one
// context cannot stop another's copy).
void step_once(swe_ctx* c, double* W, double dt, cudaStream_t s, const int* stop, bool save = true);

// Pick the fastest launch shapes of the volume kernel and the stage update
// for this context on W (scratch buffers only); synchronises s.
int autotune_ctx(swe_ctx* c, const double* W, cudaStream_t s);

// Adjoint launchers (k_adjoint.cu). launch_rhs_adjoint expects the forward
// intermediates of W in the work buffers (rhs_chain just ran on W) and adds
// (dR/dW)^T Rb to Wbar and (dR/db)^T Rb to bbar (nullable). With defer_src,
// the source-coefficient cotangents are added to adj.Gsrc_acc instead of
// being carried to bbar; launch_src_adjoint later adds their (linear,
// state-independent) image under the source's bathymetry derivatives to
// bbar, once for all the stages that accumulated.
void launch_rhs_adjoint(swe_ctx* c, const double* W, const double* Rb, double* Wbar, double* bbar, cudaStream_t s,
                        bool defer_src = false);
void launch_src_adjoint(swe_ctx* c, const double* Gsrc, double* bbar, cudaStream_t s);
void launch_limit_record(swe_ctx* c, double* W, uint8_t* act, int32_t* amin, uint8_t* cut, cudaStream_t s);
void launch_update_adjoint(swe_ctx* c, int mode, double* Wb, const double* Y, const uint8_t* act,
                           const int32_t* amin, const uint8_t* cut, double* Khb, double* Rb, double* Wnb, double a,
                           double b, double dt, cudaStream_t s);
void launch_gauge(swe_ctx* c, const double* W, int ng, const int32_t* elem, const double* wts,
                  const double* target, double* values, double* loss, double* Wb, cudaStream_t s);
void launch_axpy(swe_ctx* c, long long count, double a, const double* x, double* y, cudaStream_t s);

// Context construction (swe_create; ensembles pass an instance map and a
// status word shared by their groups).
int create_ctx(int N, int K, const double* x, const double* y, const int32_t* EToE, const int32_t* EToF,
               const int32_t* flip, const double* b, double g, const swe_params* p, const int32_t* inst,
               int ninst, int* shared_status, swe_ctx** out);

// Record the text of an error for swe_last_error() and return code.
int set_last_error(int code, const std::string& msg);

// Grid of a warp-per-element kernel whose blocks loop over element groups:
// at most `per_sm` blocks of `wpb` warps per multiprocessor (the default
// gives every group its own block, which measured fastest for these
// short-lived warps), never more blocks than groups.
inline int persistent_grid(const swe_ctx* c, int wpb, int per_sm = 1 << 20) {
    const long long groups = (c->m.K + wpb - 1) / wpb;
    const long long cap = (long long)c->sms * per_sm;
    return (int)(groups < cap ? (groups > 0 ? groups : 1) : cap);
}

// Timing bracket of one launch.
struct Timed {
    swe_ctx* c;
    cudaStream_t s;
    int idx = -1;
    Timed(swe_ctx* c, int cls, cudaStream_t s);
    ~Timed();
};

}  // namespace swe
