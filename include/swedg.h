/*
 * swedg: GB300-native right-hand side and time stepping of the entropy-stable
 * nodal DGSEM for the 2D shallow water equations on curvilinear quadrilateral
 * meshes with wet/dry fronts (Wintermeyer, Winters, Gassner, Warburton 2018).
 *
 * C ABI: plain pointers and sizes. All floating point is IEEE binary64.
 *
 * Nodal layout (every nodal array, host or device): [K][n][n], n = N+1,
 * index (k*n + j)*n + i, i the xi index (fastest), j the eta index. A state
 * W or a right-hand side R is three such planes (h, hu, hv) back to back:
 * W[c*K*n*n + (k*n + j)*n + i].
 *
 * Element faces: 0: eta=-1 (j=0), 1: xi=+1 (i=N), 2: eta=+1 (j=N),
 * 3: xi=-1 (i=0). Face node p runs along increasing xi (faces 0, 2) or eta
 * (faces 1, 3). Node p of face (k,f) meets node (flip ? N-p : p) of face
 * (EToE[k*4+f], EToF[k*4+f]); the connectivity must be reciprocal.
 * EToE[k*4+f] = -1 makes the face a solid wall (EToF, flip ignored there):
 * the interface flux and the positivity time step take the mirror state
 * (same h and b, normal velocity reversed), BR1 takes the own velocity as
 * U* and no viscous flux crosses the wall. The paper uses solid walls in its
 * dam-break cases but states no wall formula; this is the library's.
 *
 * Ownership: the caller owns W, R and every pointer it passes; a context owns
 * the geometry and the scratch buffers it allocates on the device at
 * swe_create and releases at swe_destroy. Device pointers must stay valid
 * while work queued on the given stream runs. A NULL stream is the legacy
 * default stream. A context's scratch buffers serve one call at a time:
 * calls on one context that may overlap on the GPU (different streams, or
 * different host threads) must be serialised by the caller. A context of at
 * least 2^20 nodes also owns a second stream: parts of a right-hand side and
 * of a step (the smoothness indicator, a step's start-state copy and time
 * step) run there beside the interface flux, forked from and joined back into
 * the caller's stream by events, so the caller's stream order holds and the
 * calls stay capturable in a CUDA graph.
 *
 * Errors: every int-returning call returns SWE_OK (0) or a negative code; the
 * text of the last error of the calling thread is swe_last_error(). No call
 * traps or waits without bound on the device.
 */
#ifndef SWEDG_H
#define SWEDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWE_OK 0
#define SWE_ERR_ARG (-1)       /* invalid argument or unsupported input */
#define SWE_ERR_GEOM (-2)      /* non-positive Jacobian at a node */
#define SWE_ERR_NEG_MEAN (-3)  /* an element mean water height became negative */
#define SWE_ERR_NONFINITE (-4) /* a non-finite value appeared in the state */
#define SWE_ERR_CUDA (-5)      /* a CUDA runtime call failed */

#define SWE_NMAX 12

typedef struct swe_ctx swe_ctx;

/* Scheme parameters.
 * flux:      0 entropy-conservative interface flux (Eq. surfaceFluxes),
 *            1 entropy-stable flux (Eq. fesandges, rotated as in App. B).
 * av:        1 adds the BR1 artificial viscosity of Sec. 3 (Thm. 1) with the
 *            element viscosity of App. A.
 * eps0:      base viscosity epsilon_0 of App. A.
 * sigma_min, sigma_max: ramp of App. A; NaN selects -4 log10(N) -/+ 1 (the
 *            paper gives no values).
 * limiter:   1 applies the positivity limiter (Eq. PosPres) and the h_tol
 *            momentum cut after every Runge-Kutta stage.
 * h_tol:     water height below which the momentum is set to zero (Sec. 6.1,
 *            1e-4); NaN selects 1e-4.
 * rk:        0 five-stage fourth-order 2N-storage Runge-Kutta (Carpenter &
 *            Kennedy), 1 SSPRK3 (Eq. RKSSP).
 * cfl:       CFL number of the time-step rule
 *            dt = cfl * 2/(N+1) * min_nodes J / (lambda_xi + lambda_eta).
 * volume:    0 split-form volume term by flux differencing (Eq. fluxDiffFormF,
 *            Eq. Fmij) with the well-balanced split source (Eq. SourceDisc);
 *            1 the standard volume term of Eq. VolInt (second line), D applied
 *            to the nodal contravariant fluxes, with the non-split source
 *            -g h J grad b (the paper's comparison scheme: neither entropy
 *            stable nor well balanced).
 * cfl_visc:  0 keeps the paper's time-step rule. > 0 (with av) adds the
 *            viscous restriction of the AV term, which the paper does not
 *            have: a node of an element with viscosity eps_k (of the state
 *            at the start of the step) adds the rate eps_k kv a^2 to
 *            lambda/J, a = (|a_xi| + |a_eta|)/J, kv = (N+1)^3 cfl /
 *            (8 cfl_visc); alone it limits dt to
 *            16 cfl_visc / (eps_k a^2 (N+1)^4), i.e. cfl_visc dx^2 /
 *            (eps_k (N+1)^4) on an affine square element of side dx. With a
 *            fixed eps0 the explicit AV term otherwise becomes unstable as
 *            the mesh is refined (0.25 keeps the 4.2M-node dam break of
 *            the benchmark stable). Appended last: callers that zero the
 *            struct get the paper's rule. */
typedef struct {
    int flux;
    int av;
    double eps0;
    double sigma_min;
    double sigma_max;
    int limiter;
    double h_tol;
    int rk;
    double cfl;
    int volume;
    double cfl_visc;
} swe_params;

/* Build a context (Sec. 2.1: curvilinear map, metric terms, Jacobian
 * Eq. JacobianDef, surface Jacobian Eq. SurfJac; Eq. SourceDisc's split-form
 * bathymetry derivatives). Host inputs, copied:
 *   x, y, b  [K][n][n] node coordinates and bathymetry (b must agree on the
 *            two sides of every face node);
 *   EToE, EToF, flip [K][4] connectivity as described above;
 *   g > 0 gravity; p parameters (copied).
 * Uses the current CUDA device. 1 <= N <= SWE_NMAX, K >= 1.
 * Returns SWE_ERR_GEOM if J <= 0 at a node, SWE_ERR_ARG for bad
 * connectivity (non-reciprocal, out of range other than the wall mark -1),
 * sizes or parameters, SWE_ERR_CUDA on allocation failure. */
int swe_create(int N, int K, const double* x, const double* y, const int32_t* EToE,
               const int32_t* EToF, const int32_t* flip, const double* b, double g,
               const swe_params* p, swe_ctx** out);

/* Release a context (waits for its work on the device to finish). */
void swe_destroy(swe_ctx* ctx);

/* Semi-discrete operator R = W_t of Eq. CurvilinearECDGSEMviscous divided by
 * J (Eq. Curvilinear ECDGSEM without viscosity when av = 0): volume term by
 * flux differencing (Eq. fluxDiffFormF, Eq. Fmij, Eq. volumeFluxes),
 * interface flux, source, BR1 viscous terms (Eq. BR1, Eq. ViscTermsDisc).
 * W, R: device pointers, 3*K*n*n doubles each, not overlapping. Asynchronous
 * on `stream` (a cudaStream_t). */
int swe_rhs(swe_ctx* ctx, const double* W, double* R, void* stream);

/* Positivity limiter (Eq. PosPres) and the h_tol momentum cut on device
 * state W in place. Asynchronous; an element with a negative mean is left as
 * is and recorded in the status read by swe_status. */
int swe_limit(swe_ctx* ctx, double* W, void* stream);

/* Largest admissible time step for device state W: the CFL rule (dt_cfl,
 * including the viscous restriction when cfl_visc > 0, for which the element
 * viscosities of W are computed first) and the positivity restrictions of
 * Lemma PosPres, Eq. CFLConstraints (dt_pos, +inf when limiter = 0 or
 * flux = 0). Host outputs; synchronises `stream`; overwrites the context's
 * scratch buffers (velocities, and with cfl_visc > 0 the interface and AV
 * work buffers). */
int swe_max_dt(swe_ctx* ctx, const double* W, double* dt_cfl, double* dt_pos, void* stream);

/* Advance device state W in place by nsteps steps of the chosen Runge-Kutta
 * scheme (with the limiter after every stage when enabled). dt > 0 is a fixed
 * step; dt <= 0 recomputes min(dt_cfl, dt_pos) at the start of every step on
 * the device. Synchronises `stream` at the end and checks the device status:
 * if an element mean became negative or a value became non-finite, W is
 * restored to the state at the start of the failing step, and
 * SWE_ERR_NEG_MEAN or SWE_ERR_NONFINITE is returned (the caller may retry
 * with a smaller dt). dt_last (host, nullable) receives the last step size. */
int swe_step(swe_ctx* ctx, double* W, double dt, int nsteps, double* dt_last, void* stream);

/* Discrete integrals of device state W: out3 = sum_k sum_ij J w_i w_j W
 * (mass and momenta), E = sum J w_i w_j e(W) with e of Eq. entropyFunction.
 * Host outputs; synchronise `stream`; deterministic summation order. */
int swe_mass(swe_ctx* ctx, const double* W, double* out3, void* stream);
int swe_entropy(swe_ctx* ctx, const double* W, double* E, void* stream);
/* Both in one pass: out4 = (mass, x momentum, y momentum, entropy), host. */
int swe_integrals(swe_ctx* ctx, const double* W, double* out4, void* stream);
/* swe_step (nsteps >= 1) followed by swe_integrals of the new state, with one
 * synchronisation of `stream` and one device-to-host copy for the integrals,
 * the step size and the status (swe_step and swe_integrals synchronise once
 * each). On success W and out4 are bitwise what swe_step and swe_integrals
 * give; on a failed step W is restored as by swe_step and out4 is left
 * untouched. */
int swe_step_integrals(swe_ctx* ctx, double* W, double dt, int nsteps, double* dt_last, double* out4,
                       void* stream);
/* swe_step_integrals without any host synchronisation: enqueues the nsteps
 * steps and the integrals of the resulting state on `stream` and returns.
 * out6 (device, 6 doubles, owned by the caller) receives (mass, x momentum,
 * y momentum, entropy, step size of the last step, status bits as a
 * double). A failed step (status bit 1: negative element mean, bit 2:
 * non-finite value) stops the call's remaining kernels and a device-side
 * copy restores W to the start of the failing step, as swe_step does; the
 * integrals are then those of the restored state, and the status stays set
 * for swe_status until the next step call. Only argument errors and launch
 * errors are returned here. Makes no host synchronisation and no
 * allocation, so a CUDA graph may capture it (with timing off). */
int swe_step_async(swe_ctx* ctx, double* W, double dt, int nsteps, double* out6, void* stream);

/* Discrete entropy rate of device state W (Sec. 2: the entropy variables
 * q = (g(h+b) - (u^2+v^2)/2, u, v) of Eq. entropyVariables contracted with
 * the semi-discrete operator): rate = sum_k sum_ij J w_i w_j q(W_ij).R_ij
 * with R = swe_rhs(W), the time derivative of swe_entropy along the
 * semi-discrete flow (zero up to rounding for the entropy-conservative
 * flux on a periodic or walled mesh without viscosity, <= 0 for the
 * entropy-stable flux and the artificial viscosity). scale (host, nullable)
 * receives sum J w_i w_j sum_c |q_c R_c|, the size of the terms that cancel.
 * Evaluates R into the context's work buffer (not during a step);
 * synchronises `stream`. */
int swe_entropy_rate(swe_ctx* ctx, const double* W, double* rate, double* scale, void* stream);

/* Copy the element viscosities epsilon_k (App. A) of the last swe_rhs into
 * device array eps[K]. Asynchronous. */
int swe_get_epsilon(swe_ctx* ctx, double* eps, void* stream);

/* Device status bits accumulated since the last call (1: negative element
 * mean, 2: non-finite value), then cleared. Synchronises `stream`. */
int swe_status(swe_ctx* ctx, int* bits, void* stream);

/* Kernel timing of the library's own launches. After swe_timing(ctx, 1),
 * every kernel launch is bracketed by CUDA events on its stream;
 * swe_timing_read returns, for kernel class `which` (0 volume, 1 interface
 * flux, 2 primitives, 3 AV indicator/gradient, 4 viscous interface, 5 stage
 * update/limiter, 6 time step, 7 reductions, 8 adjoint kernels other than 9,
 * 9 adjoint of the volume kernel), the summed event time in
 * milliseconds and the launch count since swe_timing(ctx, 1) (synchronises).
 * swe_launches returns the number of kernels the context launched so far. */
int swe_timing(swe_ctx* ctx, int on);
/* As swe_timing, for the kernel classes of `mask` only (bit c = class c;
 * 0 turns timing off): the launches of the other classes get no events, so
 * a timed loop that needs one class's launch time carries no event overhead
 * for the rest. */
int swe_timing_classes(swe_ctx* ctx, unsigned mask);
int swe_timing_read(swe_ctx* ctx, int which, double* ms, int64_t* launches);
int64_t swe_launches(const swe_ctx* ctx);

/* Launch shapes (a performance choice only: every shape evaluates every
 * element with the same instructions in the same order, so results are
 * bitwise identical). The volume kernel runs blocks of vol_threads/(N+1)
 * elements, one thread per element line (vol_threads 64, 128 or 256; a
 * shape whose shared-memory staging exceeds 227 KB at this degree is
 * rejected); the stage update runs one warp per element in blocks of
 * upd_warps warps (2, 4 or 8). Defaults 128 and 4.
 * swe_autotune times each shape on device state W (writing only the
 * context's scratch buffers) and keeps the fastest; synchronises `stream`.
 * swe_set_tuning returns SWE_ERR_ARG for a shape not listed above. */
int swe_autotune(swe_ctx* ctx, const double* W, void* stream);
int swe_get_tuning(const swe_ctx* ctx, int* vol_threads, int* upd_warps);
int swe_set_tuning(swe_ctx* ctx, int vol_threads, int upd_warps);

/* ---------------------------------------------------------------------------
 * Adjoint (the paper has none; this is the library's). Vector-Jacobian
 * products of the discrete operator for gradients with respect to the state
 * and the bathymetry, exact up to rounding, with the decisions of the
 * forward pass held fixed: the element viscosities eps_k (App. A), the
 * limiter's active set (limited elements and the node of their minimum;
 * theta of Eq. PosPres is differentiated), the nodes cut by h_tol and the
 * step size. At dry nodes the velocity and the celerity have zero
 * derivative. Split (entropy-stable) volume form only (volume = 0); other
 * contexts get SWE_ERR_ARG. The first adjoint call allocates the adjoint's
 * buffers (about 40 doubles per node plus 5 stage states).
 *
 * swe_rhs_adjoint: for R = swe_rhs(W), Wbar += (dR/dW)^T Rbar and, when bbar
 * is not NULL, bbar += (dR/db)^T Rbar. W, Rbar, Wbar: device, 3*K*n*n;
 * bbar: device, K*n*n. Asynchronous on `stream`.
 *
 * swe_step_adjoint: for one step W1 = step(W0, dt) of swe_step with the
 * given dt > 0 (the size the forward step used), replaces Wbar (on entry the
 * cotangent of W1) by the cotangent of W0, and adds the step's bathymetry
 * cotangent to bbar (nullable). The step is recomputed from W0 (device,
 * unchanged) with its decisions recorded, then swept in reverse stage by
 * stage. Synchronises `stream`; SWE_ERR_NEG_MEAN if the recomputed step
 * fails.
 *
 * Recorded steps, for a reverse sweep that does not recompute its steps:
 * swe_adjoint_slots reserves nslots >= 1 step records on the device (each
 * about 6 S + 2 doubles per node for S = 5 or 3 stages), discarding earlier
 * records; it synchronises the device. swe_step_record advances W (device,
 * in place) by one step of swe_step with the given dt > 0 and stores the
 * step's stage inputs, pre-limit stage results and decisions in record
 * `slot` (0 <= slot < nslots); W1 is bitwise swe_step's result. It
 * synchronises `stream`; if the step fails, W is restored to its start
 * state and SWE_ERR_NEG_MEAN or SWE_ERR_NONFINITE is returned.
 * swe_step_adjoint_recorded is swe_step_adjoint for the step recorded in
 * `slot` (same dt), without recomputing it. swe_step_adjoint itself records
 * its step in slot 0.
 *
 * swe_gauge_misfit: gauge values h_g = sum over the nodes of element elem[g]
 * of wts[g][node] h (ngauge gauges; wts [ngauge][n*n] are interpolation
 * weights; all device arrays). values (nullable) receives h_g; loss
 * (nullable, one double) += sum_g (h_g - target_g)^2 (target nullable: 0);
 * Wbar (nullable) += 2 (h_g - target_g) wts[g] on the h plane. Gauges are
 * processed in order by one block (deterministic). Asynchronous. */
int swe_rhs_adjoint(swe_ctx* ctx, const double* W, const double* Rbar, double* Wbar, double* bbar, void* stream);
int swe_step_adjoint(swe_ctx* ctx, const double* W0, double dt, double* Wbar, double* bbar, void* stream);
int swe_adjoint_slots(swe_ctx* ctx, int nslots);
int swe_step_record(swe_ctx* ctx, double* W, double dt, int slot, void* stream);
int swe_step_adjoint_recorded(swe_ctx* ctx, int slot, double dt, double* Wbar, double* bbar, void* stream);
int swe_gauge_misfit(swe_ctx* ctx, const double* W, int ngauge, const int32_t* elem, const double* wts,
                     const double* target, double* values, double* loss, double* Wbar, void* stream);

/* Sizes of a context: N, K and the number of unique faces. */
int swe_info(const swe_ctx* ctx, int* N, int* K, int* nfaces);

/* Allocation-free diagnostic integrals, for callers that cannot call
 * cudaMalloc (the paper has no counterpart: this is an interface for
 * embedding). Such callers include code running while a host framework's
 * caching allocator owns the device memory pool, real-time loops that cannot
 * afford the device synchronisation implied by cudaMalloc/cudaFree, and hosts
 * with a memory budget fixed at start-up. The call computes the same sums as
 * swe_mass and swe_entropy without a context:
 *   out4[0..2] = sum_k sum_ij wJ W_c,  out4[3] = sum_k sum_ij wJ e(W),
 *   e = (hu^2 + hv^2)/(2h) + g h^2/2 + g h b  (kinetic part 0 where h <= 0),
 * with
 *   W    device, 3*K*(N+1)^2 doubles, the state planes (h, hu, hv);
 *   wJ   device, K*(N+1)^2 doubles, w_i w_j J at every node;
 *   b    device, K*(N+1)^2 doubles, the bathymetry;
 *   out4 device, 4 doubles, written asynchronously on `stream`.
 * All four must be device (or managed) memory of the current device, and
 * `stream` must belong to it: a pointer of another device or of host memory
 * is rejected with SWE_ERR_ARG before any launch. The sizes are the caller's
 * promise: the kernels read exactly 3*K*(N+1)^2, K*(N+1)^2 and K*(N+1)^2
 * doubles and write 4.
 * It allocates nothing: the per-element partial sums live in one fixed
 * device array of 4*SWE_NOALLOC_MAX_ELEMENTS doubles (2 MiB), which every GPU
 * that loads the library holds until the process exits. K above
 * SWE_NOALLOC_MAX_ELEMENTS is rejected with SWE_ERR_ARG. The first call on
 * each device resolves that array's device address (cudaGetSymbolAddress,
 * with the device current), so make the first call on a device before any
 * stream capture. Every call writes each partial it later reads, so nothing
 * needs clearing, but all calls share the one array: calls that may overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller. */
#define SWE_NOALLOC_MAX_ELEMENTS 65536
int swe_integrals_noalloc(int N, int K, const double* W, const double* wJ, const double* b, double g,
                          double* out4, void* stream);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent periodic meshes, of mixed degree and size,
 * advanced together (the paper runs one mesh per launch; this batched form,
 * with its layout, is this library's own). Each instance is the problem of
 * swe_create: its own mesh, bathymetry and state, the shared g and
 * parameters, and its own time step.
 *
 * State layout of an ensemble: one device buffer of swe_ens_size doubles.
 * The instances of one degree form a group; a group's planes h, hu, hv each
 * hold the [K][n][n] nodes of its instances back to back (in instance order),
 * and group planes start on 256-byte boundaries. swe_ens_layout gives, for
 * instance i, the offset (doubles) of its h nodes and the plane stride, so
 * that its (h, hu, hv) planes start at W + offset + c*plane_stride and are
 * laid out as in a single context.
 *
 * Every kernel evaluates each element, face and node exactly as it does for a
 * single context, so an instance's right-hand side and steps are bitwise
 * those of swe_create/swe_rhs/swe_step on that instance alone. */
typedef struct swe_ens swe_ens;

/* One instance (host arrays, copied at creation; layout as for swe_create).
 * EToE is local to the instance: 0 <= EToE < K, or -1 for a solid wall. */
typedef struct {
    int N;
    int K;
    const double* x;
    const double* y;
    const double* b;
    const int32_t* EToE;
    const int32_t* EToF;
    const int32_t* flip;
} swe_instance;

/* Build an ensemble of ninst >= 1 instances on the current CUDA device, with
 * gravity g and parameters p shared by all. Errors as swe_create (the text
 * names the failing degree group); SWE_ERR_ARG also for EToE outside an
 * instance. */
int swe_ens_create(int ninst, const swe_instance* inst, double g, const swe_params* p, swe_ens** out);
void swe_ens_destroy(swe_ens* ens);

/* Doubles of an ensemble state (total) and the number of degree groups. */
int swe_ens_size(const swe_ens* ens, int64_t* total, int* ngroups);
/* Where instance i lives in an ensemble state (see above), its N and K. */
int swe_ens_layout(const swe_ens* ens, int i, int64_t* offset, int64_t* plane_stride, int* N, int* K);

/* swe_rhs of every instance: W, R device buffers of swe_ens_size doubles, not
 * overlapping. Asynchronous on `stream`. */
int swe_ens_rhs(swe_ens* ens, const double* W, double* R, void* stream);

/* swe_max_dt of every instance: host outputs dt_cfl[ninst], dt_pos[ninst]
 * (nullable). Synchronises `stream`. */
int swe_ens_max_dt(swe_ens* ens, const double* W, double* dt_cfl, double* dt_pos, void* stream);

/* swe_step of every instance (dt <= 0: each instance takes its own
 * min(dt_cfl, dt_pos) at the start of every step). One step of all groups is
 * a CUDA graph, captured at the first call for a given (W, dt) and replayed
 * nsteps times on `stream`. The status is shared: if any instance fails
 * (negative mean or non-finite value), every instance is restored to the
 * start of the failing step and SWE_ERR_NEG_MEAN or SWE_ERR_NONFINITE is
 * returned. dt_last (host [ninst], nullable) receives each instance's last
 * step size. Synchronises `stream`. */
int swe_ens_step(swe_ens* ens, double* W, double dt, int nsteps, double* dt_last, void* stream);

/* swe_integrals of every instance: out (host [ninst][4]) = (mass, x momentum,
 * y momentum, entropy) per instance, in a fixed summation order.
 * Synchronises `stream`. */
int swe_ens_integrals(swe_ens* ens, const double* W, double* out, void* stream);

/* Kernels launched so far (graph replays count their kernels). */
int64_t swe_ens_launches(const swe_ens* ens);

/* swe_autotune for every degree group on its part of ensemble state W (the
 * step graph is captured again at the next swe_ens_step). Synchronises. */
int swe_ens_autotune(swe_ens* ens, const double* W, void* stream);
/* Degree group g (0 <= g < ngroups, increasing N): its N, member count and
 * launch shapes. */
int swe_ens_group(const swe_ens* ens, int g, int* N, int* members, int* vol_threads, int* upd_warps);

/* Text of the last error on the calling thread ("" if none). */
const char* swe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
