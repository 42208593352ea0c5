/*
 * Oracle for the entropy-stable nodal DGSEM of the 2D shallow water equations
 * with artificial viscosity and a positivity-preserving limiter
 * (Wintermeyer, Winters, Gassner, Warburton, "An entropy stable discontinuous
 * Galerkin method for the shallow water equations on curvilinear meshes with
 * wet/dry fronts accelerated by GPUs", 2018).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow FP64 CPU restatement of the
 * paper's equations, used to check the CUDA library. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never calls it. It shares no code, header or table with the CUDA
 * library.
 *
 * Layout of every nodal array: [K][n][n] with n = N+1, index (k*n + j)*n + i,
 * i the xi-index (fastest), j the eta-index. The state W is three such planes
 * (h, hu, hv). Element faces: 0: eta=-1 (j=0), 1: xi=+1 (i=N), 2: eta=+1
 * (j=N), 3: xi=-1 (i=0); face node p runs along increasing xi (faces 0,2) or
 * eta (faces 1,3). Node p of face (k,f) meets node (flip ? N-p : p) of face
 * (EToE[k][f], EToF[k][f]); EToE[k][f] = -1 makes the face a solid wall
 * (mirror state for the interface flux and the time step, U* = own value
 * and no viscous flux for BR1).
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NMAX 16

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_GEOM (-2)
#define ORC_ERR_NEG_MEAN (-3)
#define ORC_ERR_NONFINITE (-4)

typedef struct {
    int flux;         /* 0: entropy-conservative surface flux, 1: entropy-stable (Eq. fesandges) */
    int av;           /* 1: artificial viscosity (Sec. 3, App. A) */
    double eps0;      /* base viscosity epsilon_0 */
    double sigma_min; /* NaN: default -4 log10(N) - 1 */
    double sigma_max; /* NaN: default -4 log10(N) + 1 */
    int limiter;      /* 1: positivity limiter after every stage (Eq. PosPres) */
    double h_tol;     /* NaN: 1e-4 (Sec. 6.1) */
    int rk;           /* 0: LSRK4(5) (Carpenter-Kennedy 2N-storage), 1: SSPRK3 (Eq. RKSSP) */
    double cfl;       /* CFL number of the time-step rule */
    int volume;       /* 0: split-form volume term (Eq. fluxDiffFormF with Eq. Fmij),
                         1: standard volume term (Eq. VolInt, second line) with the
                         non-split source -g h J grad b (reading in orc.c) */
    double cfl_visc;  /* 0: the paper's time-step rule; > 0 (with av): also the viscous
                         restriction of the AV term (not in the paper; see orc_max_dt) */
} orc_params;

typedef struct orc_mesh orc_mesh;

/* LGL basis of degree N: nodes xi[n], weights w[n], D[n*n] (D[i*n+j] = l_j'(xi_i)),
 * Vandermonde V[n*n] (V[i*n+j] = L_j(xi_i) sqrt(j+1/2)) and its inverse. */
int orc_basis(int N, double* xi, double* w, double* D, double* V, double* Vinv);

int orc_create(int N, int K, const double* x, const double* y, const int* EToE,
               const int* EToF, const int* flip, const double* b, double g,
               const orc_params* p, orc_mesh** out);
void orc_destroy(orc_mesh* m);

/* Geometry as the oracle computes it: x_xi, x_eta, y_xi, y_eta, J (each [K][n][n]). */
int orc_geometry(const orc_mesh* m, double* x_xi, double* x_eta, double* y_xi,
                 double* y_eta, double* J);

/* Semi-discrete operator R(W) (Eq. CurvilinearECDGSEMviscous divided by J). */
int orc_rhs(orc_mesh* m, const double* W, double* R);
/* Element viscosity of the last orc_rhs / orc_av_fields call ([K]). */
int orc_get_epsilon(const orc_mesh* m, double* eps);
/* eps[K] and the BR1 gradients U1,U2,V1,V2 (four [K][n][n] planes) of state W. */
int orc_av_fields(orc_mesh* m, const double* W, double* eps, double* grads);

int orc_limit(orc_mesh* m, double* W);
int orc_max_dt(orc_mesh* m, const double* W, double* dt_cfl, double* dt_pos);
int orc_step(orc_mesh* m, double* W, double dt, int nsteps, double* dt_last);

int orc_mass(const orc_mesh* m, const double* W, double* out3);
int orc_entropy(const orc_mesh* m, const double* W, double* E);
/* Discrete entropy rate sum J w w q(W).R(W) (entropy variables of Eq.
 * entropyVariables, R = orc_rhs(W)); scale (nullable): sum J w w |q_c R_c|. */
int orc_entropy_rate(orc_mesh* m, const double* W, double* rate, double* scale);

/* Pointwise fluxes (for the flux pins). */
void orc_volume_flux(double g, const double* Wa, const double* Wb, double* Fs, double* Gs);
void orc_surface_flux(double g, int es, const double* Wm, const double* Wp, double bm,
                      double bp, double nx, double ny, double* F);

/* The five-stage 2N-storage coefficients A[5], B[5] used by orc_step. */
void orc_lsrk_coefficients(double* A, double* B);

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int orc_threads(void);
/* Number of OpenMP threads of later calls (timing only). */
void orc_set_threads(int t);

#ifdef __cplusplus
}
#endif
#endif
