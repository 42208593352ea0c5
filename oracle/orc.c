/*
 * Oracle: plain FP64 restatement of the entropy-stable DGSEM for the 2D
 * shallow water equations (Wintermeyer, Winters, Gassner, Warburton 2018).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h). Written for readability, not speed:
 * every loop follows the paper's formula in the paper's notation, the
 * volume term is evaluated without the symmetry of the two-point flux, and
 * each face is visited once by its owning element.
 *
 * Readings of the paper taken here (where it is garbled or silent):
 *  - Eq. Fmij: the eta volume flux is G~ = -F# {y_xi} + G# {x_xi} (the printed
 *    version pairs {x_xi} with F#, contradicting Eq. ContravariantFluxes).
 *  - Eq. fluxDiffFormF: the eta sum is sum_m D~_{jm} G~_{i,(j,m)} (index order
 *    as in Eq. VolInt).
 *  - Eq. SourceDisc: S2 = -(g/2) h beta_x, S3 = +(g/2) h beta_y with
 *    beta_x = y_eta D_xi b + D_xi(y_eta b) - y_xi D_eta b - D_eta(y_xi b),
 *    beta_y = x_eta D_xi b + D_xi(x_eta b) - x_xi D_eta b - D_eta(x_xi b)
 *    (plain D; the printed factor 2 and the sign of the y source would break
 *    the lake at rest).
 *  - Eq. BR1: the left side is J*U, the eta lift of U1/V1 and the xi lift of
 *    U2/V2 carry a minus sign (the outward normal's components), and U* is
 *    taken at the face node of the respective face.
 *  - App. A: Qhat = Vinv Q Vinv^T with the exact inverse of V; Q = h; a zero
 *    energy gives eps = 0; for N = 1 only the first energy ratio is used;
 *    the middle branch of eps is sigma_min < sigma < sigma_max; defaults
 *    sigma_min/max = -4 log10(N) -/+ 1.
 *  - Lemma PosPres: omega_0 = 2/(N(N+1)) (the LGL end weight).
 *  - Time step: dt_CFL = CFL * 2/(N+1) * min_nodes J/(lambda_xi + lambda_eta).
 *  - u = hu/h for h > 0, else 0; c = sqrt(g max(h,0)); {c} = (c- + c+)/2.
 *  - The limiter and the h_tol momentum cut act after every RK stage.
 *  - Standard volume term (Eq. VolInt, second line; the paper states only the
 *    volume integral of the standard DGSEM): D applied to the nodal
 *    contravariant fluxes F~ = y_eta f - x_eta g, G~ = -y_xi f + x_xi g of
 *    the physical fluxes, the same interface flux and lift as the split form
 *    in strong form (F* - F~_own at the face nodes), and the non-split source
 *    -g h J b_x, -g h J b_y with J b_x = y_eta b_xi - y_xi b_eta,
 *    J b_y = -x_eta b_xi + x_xi b_eta (the continuous limit of the split
 *    source).
 *
 * Time step: orc_max_dt follows the paper's rule (CFL and positivity); with
 * cfl_visc > 0 it adds a viscous restriction of the AV term that the paper
 * does not have (see orc_max_dt).
 *
 * Pins: every function is checked by the CPU tests against closed forms,
 * identities or brute force. The solid-wall term of the positivity time
 * step in orc_max_dt (mirror state at a wall face) is pinned by its closed
 * form w0 (J/|n|)/(2c) on an element closed by walls (Lemma PosPres with
 * {u~} = 0 and B = 0 there).
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 4

static const double PI = 3.14159265358979323846;

struct orc_mesh {
    int N, n, K;
    double g;
    orc_params p;
    double sigma_min, sigma_max, h_tol;
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1];
    double D[ORC_NMAX + 1][ORC_NMAX + 1];    /* D_ij = l_j'(xi_i), Eq. DmatDef */
    double Dt[ORC_NMAX + 1][ORC_NMAX + 1];   /* D~ = 2D + S, Eq. Dmat_modification */
    double Dh[ORC_NMAX + 1][ORC_NMAX + 1];   /* D^ = -M^-1 D^T M (Sec. 2.2) */
    double Vinv[ORC_NMAX + 1][ORC_NMAX + 1]; /* inverse Vandermonde, App. A */
    double *x, *y, *b;
    double *x_xi, *x_eta, *y_xi, *y_eta, *J;
    double *beta_x, *beta_y;
    double *jbx, *jby;      /* J b_x, J b_y of the standard-form source */
    int *EToE, *EToF, *flip;
    double *eps;
    /* work arrays */
    double *u, *v;          /* primitive velocities */
    double *Fstar;          /* [K][4][n][3] outward numerical flux per element side */
    double *Ustar;          /* [K][4][n][2] BR1 interface values {u}, {v} */
    double *grad;           /* [4][K][n][n] U1, U2, V1, V2 */
    double *Fvstar;         /* [K][4][n][2] outward viscous interface flux */
};

/* ------------------------------------------------------------------ */
/* Indexing helpers                                                    */
/* ------------------------------------------------------------------ */

static size_t nid(const orc_mesh* m, int k, int i, int j) {
    return ((size_t)k * m->n + j) * m->n + i;
}

static size_t sid(const orc_mesh* m, int k, int f, int p) {
    return ((size_t)k * NF + f) * m->n + p;
}

/* Volume node (i,j) of face node p on face f. */
static void face_node(int N, int f, int p, int* i, int* j) {
    switch (f) {
    case 0: *i = p; *j = 0; break;
    case 1: *i = N; *j = p; break;
    case 2: *i = p; *j = N; break;
    default: *i = 0; *j = p; break;
    }
}

/* Outward unscaled normal at face node p of face f of element k: the
 * contravariant direction (y_eta, -x_eta) on xi faces and (-y_xi, x_xi) on
 * eta faces, negated on the xi=-1 and eta=-1 faces. Its length is the
 * surface Jacobian of Eq. SurfJac. */
static void outward_normal(const orc_mesh* m, int k, int f, int p, double* nx, double* ny) {
    int i, j;
    face_node(m->N, f, p, &i, &j);
    size_t id = nid(m, k, i, j);
    switch (f) {
    case 0: *nx = m->y_xi[id]; *ny = -m->x_xi[id]; break;
    case 1: *nx = m->y_eta[id]; *ny = -m->x_eta[id]; break;
    case 2: *nx = -m->y_xi[id]; *ny = m->x_xi[id]; break;
    default: *nx = -m->y_eta[id]; *ny = m->x_eta[id]; break;
    }
}

/* A face is computed by its owner: the element with the smaller index
 * (or, for a face joined to the same element, the smaller face index). */
static int is_owner(const orc_mesh* m, int k, int f) {
    int kk = m->EToE[NF * k + f], ff = m->EToF[NF * k + f];
    return kk > k || (kk == k && ff > f);
}

static int is_wall(const orc_mesh* m, int k, int f) { return m->EToE[NF * k + f] < 0; }

/* Solid wall: the mirror state of W (same h, normal velocity reversed about
 * the unit normal (nx, ny), tangential velocity kept). */
static void wall_state(const double* W, double nx, double ny, double* Wg) {
    double mn = W[1] * nx + W[2] * ny;
    Wg[0] = W[0];
    Wg[1] = W[1] - 2.0 * mn * nx;
    Wg[2] = W[2] - 2.0 * mn * ny;
}

static int neighbour_node(const orc_mesh* m, int k, int f, int p) {
    return m->flip[NF * k + f] ? m->N - p : p;
}

/* ------------------------------------------------------------------ */
/* Basis (Sec. 2.2, App. A)                                            */
/* ------------------------------------------------------------------ */

/* Legendre polynomials L_0..L_N at x (three-term recurrence). */
static void legendre_all(int N, double x, double* L) {
    L[0] = 1.0;
    if (N >= 1) L[1] = x;
    for (int k = 1; k < N; ++k)
        L[k + 1] = ((2.0 * k + 1.0) * x * L[k] - k * L[k - 1]) / (k + 1.0);
}

/* L_N(x) and L_N'(x). */
static void legendre_d(int N, double x, double* P, double* dP) {
    double L[ORC_NMAX + 2];
    legendre_all(N, x, L);
    *P = L[N];
    /* derivative from the recurrence L'_{k+1} = L'_{k-1} + (2k+1) L_k */
    double d[ORC_NMAX + 2];
    d[0] = 0.0;
    if (N >= 1) d[1] = 1.0;
    for (int k = 1; k < N; ++k) d[k + 1] = d[k - 1] + (2.0 * k + 1.0) * L[k];
    *dP = d[N];
}

static int invert(int n, double A[ORC_NMAX + 1][ORC_NMAX + 1], double Ainv[ORC_NMAX + 1][ORC_NMAX + 1]) {
    double M[ORC_NMAX + 1][2 * (ORC_NMAX + 1)];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            M[i][j] = A[i][j];
            M[i][n + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0.0) return ORC_ERR_ARG;
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t;
            }
        double s = M[c][c];
        for (int j = 0; j < 2 * n; ++j) M[c][j] /= s;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = M[r][c];
            for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i][j] = M[i][n + j];
    return ORC_OK;
}

static int basis(int N, double* xi, double* w, double D[ORC_NMAX + 1][ORC_NMAX + 1],
                 double V[ORC_NMAX + 1][ORC_NMAX + 1], double Vinv[ORC_NMAX + 1][ORC_NMAX + 1]) {
    if (N < 1 || N > ORC_NMAX) return ORC_ERR_ARG;
    int n = N + 1;
    /* LGL nodes: -1, +1 and the roots of L_N' (Newton, with L_N'' from
     * Legendre's equation (1-x^2) L'' = 2x L' - N(N+1) L). */
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int k = 1; k < N; ++k) {
        double x = -cos(PI * k / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre_d(N, x, &P, &dP);
            double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
            double dx = dP / d2P;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[k] = x;
    }
    /* weights omega_k = 2 / (N(N+1) L_N(xi_k)^2) */
    for (int k = 0; k < n; ++k) {
        double P, dP;
        legendre_d(N, xi[k], &P, &dP);
        w[k] = 2.0 / (N * (N + 1.0) * P * P);
    }
    /* D_ij = l_j'(xi_i) from the product form of the Lagrange polynomial */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (i != j) {
                double num = 1.0, den = 1.0;
                for (int m = 0; m < n; ++m) {
                    if (m != i && m != j) num *= xi[i] - xi[m];
                    if (m != j) den *= xi[j] - xi[m];
                }
                D[i][j] = num / den;
            } else {
                double s = 0.0;
                for (int m = 0; m < n; ++m)
                    if (m != i) s += 1.0 / (xi[i] - xi[m]);
                D[i][i] = s;
            }
        }
    /* Vandermonde of the normalised Legendre polynomials (Eq. Vandermonde) */
    for (int i = 0; i < n; ++i) {
        double L[ORC_NMAX + 2];
        legendre_all(N, xi[i], L);
        for (int j = 0; j < n; ++j) V[i][j] = L[j] * sqrt(j + 0.5);
    }
    return invert(n, V, Vinv);
}

int orc_basis(int N, double* xi, double* w, double* D, double* V, double* Vinv) {
    double Dm[ORC_NMAX + 1][ORC_NMAX + 1], Vm[ORC_NMAX + 1][ORC_NMAX + 1], Vi[ORC_NMAX + 1][ORC_NMAX + 1];
    double x[ORC_NMAX + 1], ww[ORC_NMAX + 1];
    int rc = basis(N, x, ww, Dm, Vm, Vi);
    if (rc) return rc;
    int n = N + 1;
    for (int i = 0; i < n; ++i) {
        if (xi) xi[i] = x[i];
        if (w) w[i] = ww[i];
        for (int j = 0; j < n; ++j) {
            if (D) D[i * n + j] = Dm[i][j];
            if (V) V[i * n + j] = Vm[i][j];
            if (Vinv) Vinv[i * n + j] = Vi[i][j];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Mesh, geometry (Sec. 2.1)                                           */
/* ------------------------------------------------------------------ */

static double* dalloc(size_t count) { return (double*)calloc(count ? count : 1, sizeof(double)); }

/* d/dxi and d/deta of a nodal field of element k by the derivative matrix. */
static double dxi(const orc_mesh* m, const double* f, int k, int i, int j) {
    double s = 0.0;
    for (int q = 0; q < m->n; ++q) s += m->D[i][q] * f[nid(m, k, q, j)];
    return s;
}

static double deta(const orc_mesh* m, const double* f, int k, int i, int j) {
    double s = 0.0;
    for (int q = 0; q < m->n; ++q) s += m->D[j][q] * f[nid(m, k, i, q)];
    return s;
}

/* D_xi and D_eta of f - c for a constant c (the same derivative, as D
 * annihilates constants). Used for the coordinates, with c the element's
 * first node: differencing first keeps the coordinates' magnitude, which can
 * exceed the element's size by orders of magnitude, out of the sums. */
static double dxi_rel(const orc_mesh* m, const double* f, double c, int k, int i, int j) {
    double s = 0.0;
    for (int q = 0; q < m->n; ++q) s += m->D[i][q] * (f[nid(m, k, q, j)] - c);
    return s;
}

static double deta_rel(const orc_mesh* m, const double* f, double c, int k, int i, int j) {
    double s = 0.0;
    for (int q = 0; q < m->n; ++q) s += m->D[j][q] * (f[nid(m, k, i, q)] - c);
    return s;
}

void orc_destroy(orc_mesh* m) {
    if (!m) return;
    double* arrs[] = {m->x, m->y, m->b, m->x_xi, m->x_eta, m->y_xi, m->y_eta, m->J,
                      m->beta_x, m->beta_y, m->jbx, m->jby, m->eps, m->u, m->v, m->Fstar, m->Ustar,
                      m->grad, m->Fvstar};
    for (size_t a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a) free(arrs[a]);
    free(m->EToE);
    free(m->EToF);
    free(m->flip);
    free(m);
}

int orc_create(int N, int K, const double* x, const double* y, const int* EToE,
               const int* EToF, const int* flip, const double* b, double g,
               const orc_params* p, orc_mesh** out) {
    if (!out || !x || !y || !EToE || !EToF || !flip || !b || !p) return ORC_ERR_ARG;
    *out = NULL;
    if (N < 1 || N > ORC_NMAX || K < 1 || !(g > 0.0)) return ORC_ERR_ARG;
    if (!(p->cfl_visc >= 0.0) || isinf(p->cfl_visc)) return ORC_ERR_ARG;
    orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
    m->N = N;
    m->n = N + 1;
    m->K = K;
    m->g = g;
    m->p = *p;
    double s0 = -4.0 * log10((double)N);
    m->sigma_min = isnan(p->sigma_min) ? s0 - 1.0 : p->sigma_min;
    m->sigma_max = isnan(p->sigma_max) ? s0 + 1.0 : p->sigma_max;
    m->h_tol = isnan(p->h_tol) ? 1e-4 : p->h_tol;
    double V[ORC_NMAX + 1][ORC_NMAX + 1];
    if (basis(N, m->xi, m->w, m->D, V, m->Vinv)) { orc_destroy(m); return ORC_ERR_ARG; }
    int n = m->n;
    /* D~ = 2D + S with S = diag(1/omega_0, 0, ..., 0, -1/omega_N) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            m->Dt[i][j] = 2.0 * m->D[i][j];
            m->Dh[i][j] = -m->D[j][i] * m->w[j] / m->w[i];
        }
    m->Dt[0][0] += 1.0 / m->w[0];
    m->Dt[N][N] -= 1.0 / m->w[N];

    size_t nn = (size_t)K * n * n;
    m->x = dalloc(nn); m->y = dalloc(nn); m->b = dalloc(nn);
    memcpy(m->x, x, nn * sizeof(double));
    memcpy(m->y, y, nn * sizeof(double));
    memcpy(m->b, b, nn * sizeof(double));
    m->EToE = (int*)malloc(sizeof(int) * NF * K);
    m->EToF = (int*)malloc(sizeof(int) * NF * K);
    m->flip = (int*)malloc(sizeof(int) * NF * K);
    memcpy(m->EToE, EToE, sizeof(int) * NF * K);
    memcpy(m->EToF, EToF, sizeof(int) * NF * K);
    memcpy(m->flip, flip, sizeof(int) * NF * K);
    /* connectivity must be reciprocal; EToE = -1 marks a solid wall */
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < NF; ++f) {
            int kk = EToE[NF * k + f], ff = EToF[NF * k + f];
            if (kk == -1) continue;
            if (kk < 0 || kk >= K || ff < 0 || ff >= NF || (kk == k && ff == f) ||
                EToE[NF * kk + ff] != k || EToF[NF * kk + ff] != f ||
                flip[NF * kk + ff] != flip[NF * k + f]) {
                orc_destroy(m);
                return ORC_ERR_ARG;
            }
        }
    m->x_xi = dalloc(nn); m->x_eta = dalloc(nn); m->y_xi = dalloc(nn); m->y_eta = dalloc(nn);
    m->J = dalloc(nn);
    m->beta_x = dalloc(nn); m->beta_y = dalloc(nn);
    m->jbx = dalloc(nn); m->jby = dalloc(nn);
    m->eps = dalloc(K);
    m->u = dalloc(nn); m->v = dalloc(nn);
    m->Fstar = dalloc((size_t)K * NF * n * 3);
    m->Ustar = dalloc((size_t)K * NF * n * 2);
    m->Fvstar = dalloc((size_t)K * NF * n * 2);
    m->grad = dalloc(4 * nn);
    /* metric terms by differentiating the nodal mapping (coordinates taken
     * relative to the element's first node); J by Eq. JacobianDef */
    for (int k = 0; k < K; ++k) {
        const double x0 = m->x[nid(m, k, 0, 0)], y0 = m->y[nid(m, k, 0, 0)];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                m->x_xi[id] = dxi_rel(m, m->x, x0, k, i, j);
                m->x_eta[id] = deta_rel(m, m->x, x0, k, i, j);
                m->y_xi[id] = dxi_rel(m, m->y, y0, k, i, j);
                m->y_eta[id] = deta_rel(m, m->y, y0, k, i, j);
                m->J[id] = m->x_xi[id] * m->y_eta[id] - m->x_eta[id] * m->y_xi[id];
                if (!(m->J[id] > 0.0)) { orc_destroy(m); return ORC_ERR_GEOM; }
            }
    }
    /* split-form bathymetry derivatives of Eq. SourceDisc (plain D, see header) */
    double* tmp1 = dalloc(nn);
    double* tmp2 = dalloc(nn);
    double* tmp3 = dalloc(nn);
    double* tmp4 = dalloc(nn);
    for (size_t id = 0; id < nn; ++id) {
        tmp1[id] = m->y_eta[id] * m->b[id];
        tmp2[id] = m->y_xi[id] * m->b[id];
        tmp3[id] = m->x_eta[id] * m->b[id];
        tmp4[id] = m->x_xi[id] * m->b[id];
    }
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double bxi = dxi(m, m->b, k, i, j), beta = deta(m, m->b, k, i, j);
                m->beta_x[id] = m->y_eta[id] * bxi + dxi(m, tmp1, k, i, j)
                              - m->y_xi[id] * beta - deta(m, tmp2, k, i, j);
                m->beta_y[id] = m->x_eta[id] * bxi + dxi(m, tmp3, k, i, j)
                              - m->x_xi[id] * beta - deta(m, tmp4, k, i, j);
                m->jbx[id] = m->y_eta[id] * bxi - m->y_xi[id] * beta;
                m->jby[id] = -m->x_eta[id] * bxi + m->x_xi[id] * beta;
            }
    free(tmp1); free(tmp2); free(tmp3); free(tmp4);
    *out = m;
    return ORC_OK;
}

int orc_geometry(const orc_mesh* m, double* x_xi, double* x_eta, double* y_xi, double* y_eta,
                 double* J) {
    if (!m) return ORC_ERR_ARG;
    size_t nn = (size_t)m->K * m->n * m->n;
    if (x_xi) memcpy(x_xi, m->x_xi, nn * sizeof(double));
    if (x_eta) memcpy(x_eta, m->x_eta, nn * sizeof(double));
    if (y_xi) memcpy(y_xi, m->y_xi, nn * sizeof(double));
    if (y_eta) memcpy(y_eta, m->y_eta, nn * sizeof(double));
    if (J) memcpy(J, m->J, nn * sizeof(double));
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Pointwise fluxes                                                    */
/* ------------------------------------------------------------------ */

static double velocity(double h, double hu) { return h > 0.0 ? hu / h : 0.0; }

/* Physical fluxes f, g of the shallow water equations (Sec. 2). */
static void physical_flux(double g, const double* W, double* f, double* gf) {
    double h = W[0], u = velocity(h, W[1]), v = velocity(h, W[2]);
    f[0] = W[1];
    f[1] = W[1] * u + 0.5 * g * h * h;
    f[2] = W[1] * v;
    gf[0] = W[2];
    gf[1] = W[2] * u;
    gf[2] = W[2] * v + 0.5 * g * h * h;
}

/* Entropy-conservative, well-balanced two-point volume fluxes F#, G#
 * (Eq. volumeFluxes). */
void orc_volume_flux(double g, const double* Wa, const double* Wb, double* Fs, double* Gs) {
    double ha = Wa[0], hb = Wb[0];
    double ua = velocity(ha, Wa[1]), va = velocity(ha, Wa[2]);
    double ub = velocity(hb, Wb[1]), vb = velocity(hb, Wb[2]);
    double h_avg = 0.5 * (ha + hb), h2_avg = 0.5 * (ha * ha + hb * hb);
    double hu_avg = 0.5 * (Wa[1] + Wb[1]), hv_avg = 0.5 * (Wa[2] + Wb[2]);
    double u_avg = 0.5 * (ua + ub), v_avg = 0.5 * (va + vb);
    Fs[0] = hu_avg;
    Fs[1] = hu_avg * u_avg + g * h_avg * h_avg - 0.5 * g * h2_avg;
    Fs[2] = hu_avg * v_avg;
    Gs[0] = hv_avg;
    Gs[1] = hv_avg * u_avg;
    Gs[2] = hv_avg * v_avg + g * h_avg * h_avg - 0.5 * g * h2_avg;
}

/* Numerical interface flux through the unit normal (nx, ny): rotate the
 * velocities into the normal frame (Eq. rotatingVelocities), evaluate the
 * x-direction flux of Eq. surfaceFlux2DCurved with the eigen-structure of
 * Eqs. RightEigenvectors2DCurved and ScalingMatrix2DCurved (entropy-stable
 * when es != 0, entropy-conservative Eq. surfaceFluxes otherwise), and
 * rotate back (Eq. surfaceFlux2DRotated). Wm is the state on the side the
 * normal points away from. */
void orc_surface_flux(double g, int es, const double* Wm, const double* Wp, double bm,
                      double bp, double nx, double ny, double* F) {
    double hm = Wm[0], hp = Wp[0];
    double um = velocity(hm, Wm[1]), vm = velocity(hm, Wm[2]);
    double up = velocity(hp, Wp[1]), vp = velocity(hp, Wp[2]);
    double utm = nx * um + ny * vm, vtm = -ny * um + nx * vm;
    double utp = nx * up + ny * vp, vtp = -ny * up + nx * vp;
    double h_avg = 0.5 * (hm + hp), h2_avg = 0.5 * (hm * hm + hp * hp);
    double ut_avg = 0.5 * (utm + utp), vt_avg = 0.5 * (vtm + vtp);
    double Fr[3];
    Fr[0] = h_avg * ut_avg;
    Fr[1] = h_avg * ut_avg * ut_avg + 0.5 * g * h2_avg;
    Fr[2] = h_avg * ut_avg * vt_avg;
    if (es) {
        double cm = sqrt(g * fmax(hm, 0.0)), cp = sqrt(g * fmax(hp, 0.0));
        double c_avg = 0.5 * (cm + cp);
        /* jump of the rotated entropy variables q = (g(h+b) - (u^2+v^2)/2, u, v) */
        double qm[3] = {g * (hm + bm) - 0.5 * (utm * utm + vtm * vtm), utm, vtm};
        double qp[3] = {g * (hp + bp) - 0.5 * (utp * utp + vtp * vtp), utp, vtp};
        double dq[3] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2]};
        double R[3][3] = {{1.0, 0.0, 1.0},
                          {ut_avg + c_avg, 0.0, ut_avg - c_avg},
                          {vt_avg, 1.0, vt_avg}};
        double Lam[3] = {fabs(ut_avg + c_avg) / (2.0 * g),
                         fabs(h_avg * ut_avg),
                         fabs(ut_avg - c_avg) / (2.0 * g)};
        double t[3];
        for (int a = 0; a < 3; ++a) {
            t[a] = 0.0;
            for (int c = 0; c < 3; ++c) t[a] += R[c][a] * dq[c]; /* R^T [[q]] */
            t[a] *= Lam[a];
        }
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += R[a][c] * t[c];
            Fr[a] -= 0.5 * s;
        }
    }
    F[0] = Fr[0];
    F[1] = nx * Fr[1] - ny * Fr[2];
    F[2] = ny * Fr[1] + nx * Fr[2];
}

/* ------------------------------------------------------------------ */
/* Artificial viscosity indicator (App. A)                             */
/* ------------------------------------------------------------------ */

static double element_epsilon(const orc_mesh* m, const double* h, int k) {
    int n = m->n, N = m->N;
    if (m->p.eps0 == 0.0) return 0.0;
    double Q[ORC_NMAX + 1][ORC_NMAX + 1], T[ORC_NMAX + 1][ORC_NMAX + 1], Qh[ORC_NMAX + 1][ORC_NMAX + 1];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[i][j] = h[nid(m, k, i, j)];
    /* modal coefficients Qhat = Vinv Q Vinv^T (Eq. TransformationToModal) */
    for (int a = 0; a < n; ++a)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += m->Vinv[a][i] * Q[i][j];
            T[a][j] = s;
        }
    for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += T[a][j] * m->Vinv[c][j];
            Qh[a][c] = s;
        }
    /* energy ratios of Eq. sigmadof (simplified form) */
    double num1 = Qh[N][N] * Qh[N][N], den1 = 0.0;
    for (int i = 0; i < N; ++i) num1 += Qh[i][N] * Qh[i][N] + Qh[N][i] * Qh[N][i];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) den1 += Qh[i][j] * Qh[i][j];
    double ratio = den1 > 0.0 ? num1 / den1 : 0.0;
    if (N >= 2) {
        double num2 = Qh[N - 1][N - 1] * Qh[N - 1][N - 1], den2 = 0.0;
        for (int i = 0; i < N - 1; ++i)
            num2 += Qh[i][N - 1] * Qh[i][N - 1] + Qh[N - 1][i] * Qh[N - 1][i];
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) den2 += Qh[i][j] * Qh[i][j];
        double ratio2 = den2 > 0.0 ? num2 / den2 : 0.0;
        if (ratio2 > ratio) ratio = ratio2;
    }
    if (!(ratio > 0.0)) return 0.0;
    double sigma = log10(ratio);
    double smin = m->sigma_min, smax = m->sigma_max;
    if (sigma <= smin) return 0.0;
    if (sigma >= smax) return m->p.eps0;
    double Delta = 1.0 + sin(PI * (sigma - 0.5 * (smax + smin)) / (smax - smin));
    return 0.5 * m->p.eps0 * Delta;
}

/* ------------------------------------------------------------------ */
/* Right-hand side                                                     */
/* ------------------------------------------------------------------ */

static void primitives(orc_mesh* m, const double* W) {
    size_t nn = (size_t)m->K * m->n * m->n;
    for (size_t id = 0; id < nn; ++id) {
        m->u[id] = velocity(W[id], W[nn + id]);
        m->v[id] = velocity(W[id], W[2 * nn + id]);
    }
}

static void state_at(const orc_mesh* m, const double* W, size_t id, double* s) {
    size_t nn = (size_t)m->K * m->n * m->n;
    s[0] = W[id];
    s[1] = W[nn + id];
    s[2] = W[2 * nn + id];
}

/* Interface quantities of every face, computed once by the owner and
 * stored for both sides (outward fluxes change sign on the neighbour). */
static void interface_terms(orc_mesh* m, const double* W) {
    int n = m->n;
    for (int k = 0; k < m->K; ++k)
        for (int f = 0; f < NF; ++f) {
            if (is_wall(m, k, f)) {
                /* the numerical flux against the mirror state; BR1 takes the
                   own value as U* (no gradient lift at walls) */
                for (int p = 0; p < n; ++p) {
                    int i, j;
                    face_node(m->N, f, p, &i, &j);
                    size_t im = nid(m, k, i, j);
                    double Wm[3], Wg[3], F[3], nx, ny;
                    state_at(m, W, im, Wm);
                    outward_normal(m, k, f, p, &nx, &ny);
                    double Jsurf = sqrt(nx * nx + ny * ny);
                    wall_state(Wm, nx / Jsurf, ny / Jsurf, Wg);
                    orc_surface_flux(m->g, m->p.flux, Wm, Wg, m->b[im], m->b[im], nx / Jsurf, ny / Jsurf, F);
                    for (int c = 0; c < 3; ++c) m->Fstar[sid(m, k, f, p) * 3 + c] = Jsurf * F[c];
                    m->Ustar[sid(m, k, f, p) * 2 + 0] = m->u[im];
                    m->Ustar[sid(m, k, f, p) * 2 + 1] = m->v[im];
                }
                continue;
            }
            if (!is_owner(m, k, f)) continue;
            int kk = m->EToE[NF * k + f], ff = m->EToF[NF * k + f];
            for (int p = 0; p < n; ++p) {
                int q = neighbour_node(m, k, f, p);
                int i, j, ii, jj;
                face_node(m->N, f, p, &i, &j);
                face_node(m->N, ff, q, &ii, &jj);
                size_t im = nid(m, k, i, j), ip = nid(m, kk, ii, jj);
                double Wm[3], Wp[3], F[3];
                state_at(m, W, im, Wm);
                state_at(m, W, ip, Wp);
                double nx, ny;
                outward_normal(m, k, f, p, &nx, &ny);
                double Jsurf = sqrt(nx * nx + ny * ny);
                orc_surface_flux(m->g, m->p.flux, Wm, Wp, m->b[im], m->b[ip], nx / Jsurf,
                                 ny / Jsurf, F);
                for (int c = 0; c < 3; ++c) {
                    m->Fstar[sid(m, k, f, p) * 3 + c] = Jsurf * F[c];
                    m->Fstar[sid(m, kk, ff, q) * 3 + c] = -Jsurf * F[c];
                }
                /* BR1 interface states U* = {u}, V* = {v} */
                double us = 0.5 * (m->u[im] + m->u[ip]), vs = 0.5 * (m->v[im] + m->v[ip]);
                m->Ustar[sid(m, k, f, p) * 2 + 0] = us;
                m->Ustar[sid(m, k, f, p) * 2 + 1] = vs;
                m->Ustar[sid(m, kk, ff, q) * 2 + 0] = us;
                m->Ustar[sid(m, kk, ff, q) * 2 + 1] = vs;
            }
        }
}

/* Numerical flux of Eq. fluxDiffFormF in the contravariant direction of the
 * face: the outward flux on xi=+1 / eta=+1 faces, its negative on the others. */
static double contravariant_star(const orc_mesh* m, const double* star, int ncomp, int k, int f,
                                 int p, int c) {
    double s = star[sid(m, k, f, p) * ncomp + c];
    return (f == 1 || f == 2) ? s : -s;
}

/* BR1 gradients (Eq. BR1) and element viscosities. */
static void av_gradients(orc_mesh* m, const double* W) {
    int n = m->n, N = m->N, K = m->K;
    size_t nn = (size_t)K * n * n;
    double *U1 = m->grad, *U2 = m->grad + nn, *V1 = m->grad + 2 * nn, *V2 = m->grad + 3 * nn;
    for (int k = 0; k < K; ++k) {
        m->eps[k] = element_epsilon(m, W, k);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double du_xi = 0.0, du_eta = 0.0, dv_xi = 0.0, dv_eta = 0.0;
                for (int q = 0; q < n; ++q) {
                    du_xi += m->Dh[i][q] * m->u[nid(m, k, q, j)];
                    dv_xi += m->Dh[i][q] * m->v[nid(m, k, q, j)];
                    du_eta += m->Dh[j][q] * m->u[nid(m, k, i, q)];
                    dv_eta += m->Dh[j][q] * m->v[nid(m, k, i, q)];
                }
                /* interface terms: U* at xi = +-1 (faces 1, 3) and eta = +-1 (faces 2, 0) */
                double Uxi = 0.0, Vxi = 0.0, Ueta = 0.0, Veta = 0.0;
                if (i == N) { Uxi += m->Ustar[sid(m, k, 1, j) * 2]; Vxi += m->Ustar[sid(m, k, 1, j) * 2 + 1]; }
                if (i == 0) { Uxi -= m->Ustar[sid(m, k, 3, j) * 2]; Vxi -= m->Ustar[sid(m, k, 3, j) * 2 + 1]; }
                if (j == N) { Ueta += m->Ustar[sid(m, k, 2, i) * 2]; Veta += m->Ustar[sid(m, k, 2, i) * 2 + 1]; }
                if (j == 0) { Ueta -= m->Ustar[sid(m, k, 0, i) * 2]; Veta -= m->Ustar[sid(m, k, 0, i) * 2 + 1]; }
                double yeta = m->y_eta[id], yxi = m->y_xi[id], xeta = m->x_eta[id], xxi = m->x_xi[id];
                double JU1 = yeta * du_xi - yxi * du_eta + yeta / m->w[i] * Uxi - yxi / m->w[j] * Ueta;
                double JU2 = -xeta * du_xi + xxi * du_eta - xeta / m->w[i] * Uxi + xxi / m->w[j] * Ueta;
                double JV1 = yeta * dv_xi - yxi * dv_eta + yeta / m->w[i] * Vxi - yxi / m->w[j] * Veta;
                double JV2 = -xeta * dv_xi + xxi * dv_eta - xeta / m->w[i] * Vxi + xxi / m->w[j] * Veta;
                U1[id] = JU1 / m->J[id];
                U2[id] = JU2 / m->J[id];
                V1[id] = JV1 / m->J[id];
                V2[id] = JV2 / m->J[id];
            }
    }
}

/* Physical viscous fluxes (components 2 and 3) at node id of element k. */
static void viscous_flux(const orc_mesh* m, const double* W, int k, size_t id, double* Fv, double* Gv) {
    size_t nn = (size_t)m->K * m->n * m->n;
    double he = W[id] * m->eps[k];
    Fv[0] = he * m->grad[id];          /* h eps U1 */
    Fv[1] = he * m->grad[2 * nn + id]; /* h eps V1 */
    Gv[0] = he * m->grad[nn + id];     /* h eps U2 */
    Gv[1] = he * m->grad[3 * nn + id]; /* h eps V2 */
}

/* BR1 interface viscous flux {F^v . n} (outward for the owner). */
static void viscous_interface(orc_mesh* m, const double* W) {
    int n = m->n;
    for (int k = 0; k < m->K; ++k)
        for (int f = 0; f < NF; ++f) {
            if (is_wall(m, k, f)) {
                /* no viscous flux through a wall */
                for (int p = 0; p < n; ++p)
                    for (int c = 0; c < 2; ++c) m->Fvstar[sid(m, k, f, p) * 2 + c] = 0.0;
                continue;
            }
            if (!is_owner(m, k, f)) continue;
            int kk = m->EToE[NF * k + f], ff = m->EToF[NF * k + f];
            for (int p = 0; p < n; ++p) {
                int q = neighbour_node(m, k, f, p);
                int i, j, ii, jj;
                face_node(m->N, f, p, &i, &j);
                face_node(m->N, ff, q, &ii, &jj);
                size_t im = nid(m, k, i, j), ip = nid(m, kk, ii, jj);
                double nx, ny, Fm[2], Gm[2], Fp[2], Gp[2];
                outward_normal(m, k, f, p, &nx, &ny);
                viscous_flux(m, W, k, im, Fm, Gm);
                viscous_flux(m, W, kk, ip, Fp, Gp);
                for (int c = 0; c < 2; ++c) {
                    double avg = 0.5 * ((nx * Fm[c] + ny * Gm[c]) + (nx * Fp[c] + ny * Gp[c]));
                    m->Fvstar[sid(m, k, f, p) * 2 + c] = avg;
                    m->Fvstar[sid(m, kk, ff, q) * 2 + c] = -avg;
                }
            }
        }
}

int orc_av_fields(orc_mesh* m, const double* W, double* eps, double* grads) {
    if (!m || !W) return ORC_ERR_ARG;
    primitives(m, W);
    interface_terms(m, W);
    av_gradients(m, W);
    size_t nn = (size_t)m->K * m->n * m->n;
    if (eps) memcpy(eps, m->eps, sizeof(double) * m->K);
    if (grads) memcpy(grads, m->grad, 4 * nn * sizeof(double));
    return ORC_OK;
}

/* Standard volume term of Eq. VolInt (second line) at node (i, j) of
 * element k in strong form: D applied to the nodal contravariant fluxes and,
 * at face nodes, the lift (F* - F~_own)/omega in the contravariant
 * direction. */
static void standard_volume(const orc_mesh* m, const double* W, int k, int i, int j, double* Lxi,
                            double* Leta) {
    int n = m->n, N = m->N;
    double g = m->g;
    for (int q = 0; q < n; ++q) {
        double Wq[3], f[3], gf[3];
        size_t iq = nid(m, k, q, j);
        state_at(m, W, iq, Wq);
        physical_flux(g, Wq, f, gf);
        for (int c = 0; c < 3; ++c) Lxi[c] += m->D[i][q] * (m->y_eta[iq] * f[c] - m->x_eta[iq] * gf[c]);
        size_t jq = nid(m, k, i, q);
        state_at(m, W, jq, Wq);
        physical_flux(g, Wq, f, gf);
        for (int c = 0; c < 3; ++c) Leta[c] += m->D[j][q] * (-m->y_xi[jq] * f[c] + m->x_xi[jq] * gf[c]);
    }
    size_t id = nid(m, k, i, j);
    double Wo[3], f[3], gf[3];
    state_at(m, W, id, Wo);
    physical_flux(g, Wo, f, gf);
    for (int c = 0; c < 3; ++c) {
        double Ft = m->y_eta[id] * f[c] - m->x_eta[id] * gf[c];
        double Gt = -m->y_xi[id] * f[c] + m->x_xi[id] * gf[c];
        if (i == N) Lxi[c] += (contravariant_star(m, m->Fstar, 3, k, 1, j, c) - Ft) / m->w[N];
        if (i == 0) Lxi[c] -= (contravariant_star(m, m->Fstar, 3, k, 3, j, c) - Ft) / m->w[0];
        if (j == N) Leta[c] += (contravariant_star(m, m->Fstar, 3, k, 2, i, c) - Gt) / m->w[N];
        if (j == 0) Leta[c] -= (contravariant_star(m, m->Fstar, 3, k, 0, i, c) - Gt) / m->w[0];
    }
}

int orc_rhs(orc_mesh* m, const double* W, double* R) {
    if (!m || !W || !R) return ORC_ERR_ARG;
    int n = m->n, N = m->N, K = m->K;
    size_t nn = (size_t)K * n * n;
    double g = m->g;
    primitives(m, W);
    interface_terms(m, W);
    if (m->p.av) {
        av_gradients(m, W);
        viscous_interface(m, W);
    } else {
        for (int k = 0; k < K; ++k) m->eps[k] = 0.0;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < K; ++k) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double Wij[3], Lxi[3] = {0, 0, 0}, Leta[3] = {0, 0, 0};
                state_at(m, W, id, Wij);
                double S[3];
                if (m->p.volume == 1) {
                    standard_volume(m, W, k, i, j, Lxi, Leta);
                    S[0] = 0.0;
                    S[1] = -g * Wij[0] * m->jbx[id];
                    S[2] = -g * Wij[0] * m->jby[id];
                } else {
                /* volume term of Eq. fluxDiffFormF with the fluxes of Eq. Fmij */
                for (int q = 0; q < n; ++q) {
                    size_t iq = nid(m, k, q, j);
                    double Wq[3], Fs[3], Gs[3];
                    state_at(m, W, iq, Wq);
                    orc_volume_flux(g, Wij, Wq, Fs, Gs);
                    double yeta_avg = 0.5 * (m->y_eta[id] + m->y_eta[iq]);
                    double xeta_avg = 0.5 * (m->x_eta[id] + m->x_eta[iq]);
                    for (int c = 0; c < 3; ++c)
                        Lxi[c] += m->Dt[i][q] * (Fs[c] * yeta_avg - Gs[c] * xeta_avg);
                }
                for (int q = 0; q < n; ++q) {
                    size_t iq = nid(m, k, i, q);
                    double Wq[3], Fs[3], Gs[3];
                    state_at(m, W, iq, Wq);
                    orc_volume_flux(g, Wij, Wq, Fs, Gs);
                    double yxi_avg = 0.5 * (m->y_xi[id] + m->y_xi[iq]);
                    double xxi_avg = 0.5 * (m->x_xi[id] + m->x_xi[iq]);
                    for (int c = 0; c < 3; ++c)
                        Leta[c] += m->Dt[j][q] * (-Fs[c] * yxi_avg + Gs[c] * xxi_avg);
                }
                /* surface term of Eq. fluxDiffFormF */
                for (int c = 0; c < 3; ++c) {
                    if (i == N) Lxi[c] += contravariant_star(m, m->Fstar, 3, k, 1, j, c) / m->w[N];
                    if (i == 0) Lxi[c] -= contravariant_star(m, m->Fstar, 3, k, 3, j, c) / m->w[0];
                    if (j == N) Leta[c] += contravariant_star(m, m->Fstar, 3, k, 2, i, c) / m->w[N];
                    if (j == 0) Leta[c] -= contravariant_star(m, m->Fstar, 3, k, 0, i, c) / m->w[0];
                }
                /* source term (Eq. SourceDisc, reading in the header) */
                S[0] = 0.0;
                S[1] = -0.5 * g * Wij[0] * m->beta_x[id];
                S[2] = 0.5 * g * Wij[0] * m->beta_y[id];
                }
                /* viscous terms (Eq. ViscTermsDisc) */
                double Lv[3] = {0.0, 0.0, 0.0};
                if (m->p.av) {
                    for (int c = 0; c < 2; ++c) {
                        double sxi = 0.0, seta = 0.0;
                        for (int q = 0; q < n; ++q) {
                            double Fv[2], Gv[2];
                            size_t iq = nid(m, k, q, j);
                            viscous_flux(m, W, k, iq, Fv, Gv);
                            sxi += m->D[i][q] * (m->y_eta[iq] * Fv[c] - m->x_eta[iq] * Gv[c]);
                            size_t jq = nid(m, k, i, q);
                            viscous_flux(m, W, k, jq, Fv, Gv);
                            seta += m->D[j][q] * (-m->y_xi[jq] * Fv[c] + m->x_xi[jq] * Gv[c]);
                        }
                        double Fv[2], Gv[2];
                        viscous_flux(m, W, k, id, Fv, Gv);
                        double Ft = m->y_eta[id] * Fv[c] - m->x_eta[id] * Gv[c];
                        double Gt = -m->y_xi[id] * Fv[c] + m->x_xi[id] * Gv[c];
                        if (i == N) sxi += (contravariant_star(m, m->Fvstar, 2, k, 1, j, c) - Ft) / m->w[N];
                        if (i == 0) sxi -= (contravariant_star(m, m->Fvstar, 2, k, 3, j, c) - Ft) / m->w[0];
                        if (j == N) seta += (contravariant_star(m, m->Fvstar, 2, k, 2, i, c) - Gt) / m->w[N];
                        if (j == 0) seta -= (contravariant_star(m, m->Fvstar, 2, k, 0, i, c) - Gt) / m->w[0];
                        Lv[c + 1] = sxi + seta;
                    }
                }
                /* Eq. CurvilinearECDGSEMviscous solved for W_t */
                for (int c = 0; c < 3; ++c)
                    R[c * nn + id] = (-Lxi[c] - Leta[c] + S[c] + Lv[c]) / m->J[id];
            }
    }
    return ORC_OK;
}

int orc_get_epsilon(const orc_mesh* m, double* eps) {
    if (!m || !eps) return ORC_ERR_ARG;
    memcpy(eps, m->eps, sizeof(double) * m->K);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Positivity limiter (Eq. PosPres) and h_tol momentum cut             */
/* ------------------------------------------------------------------ */

int orc_limit(orc_mesh* m, double* W) {
    if (!m || !W) return ORC_ERR_ARG;
    int n = m->n, K = m->K;
    size_t nn = (size_t)K * n * n;
    int rc = ORC_OK;
    for (int k = 0; k < K; ++k) {
        double vol = 0.0, mean[3] = {0, 0, 0}, hmin = INFINITY;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double wJ = m->w[i] * m->w[j] * m->J[id];
                vol += wJ;
                for (int c = 0; c < 3; ++c) mean[c] += wJ * W[c * nn + id];
                if (W[id] < hmin) hmin = W[id];
            }
        for (int c = 0; c < 3; ++c) mean[c] /= vol;
        if (!isfinite(mean[0])) { rc = ORC_ERR_NONFINITE; continue; }
        if (mean[0] < 0.0) { rc = ORC_ERR_NEG_MEAN; continue; }
        if (hmin < 0.0 && mean[0] - hmin > 0.0) {
            double theta = fmin(1.0, mean[0] / (mean[0] - hmin));
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    size_t id = nid(m, k, i, j);
                    for (int c = 0; c < 3; ++c)
                        W[c * nn + id] = theta * (W[c * nn + id] - mean[c]) + mean[c];
                }
        }
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                if (W[id] < m->h_tol) { W[nn + id] = 0.0; W[2 * nn + id] = 0.0; }
            }
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Time step (CFL rule and Lemma PosPres restrictions)                 */
/* ------------------------------------------------------------------ */

int orc_max_dt(orc_mesh* m, const double* W, double* dt_cfl, double* dt_pos) {
    if (!m || !W) return ORC_ERR_ARG;
    int n = m->n, N = m->N, K = m->K;
    size_t nn = (size_t)K * n * n;
    double g = m->g;
    double min_ratio = INFINITY; /* min over nodes of J / (lambda_xi + lambda_eta) */
    /* Optional viscous restriction of the AV term (cfl_visc > 0; not in the
     * paper, whose rule has none): a node whose element has viscosity eps_k
     * (App. A, of the state W itself) adds the rate J eps_k kv a^2 with
     * a = (|a_xi| + |a_eta|)/J and kv = (N+1)^3 CFL / (8 cfl_visc), so that
     * this term alone gives dt = 16 cfl_visc / (eps_k a^2 (N+1)^4), i.e.
     * cfl_visc dx^2 / (eps_k (N+1)^4) on an affine square element of side dx. */
    double kv = (m->p.av && m->p.cfl_visc > 0.0) ? pow(N + 1.0, 3) * m->p.cfl / (8.0 * m->p.cfl_visc) : 0.0;
    double* epsk = kv > 0.0 ? dalloc((size_t)K) : NULL;
    for (int k = 0; kv > 0.0 && k < K; ++k) epsk[k] = element_epsilon(m, W, k);
    for (size_t id = 0; id < nn; ++id) {
        double h = W[id], u = velocity(h, W[nn + id]), v = velocity(h, W[2 * nn + id]);
        double c = sqrt(g * fmax(h, 0.0));
        double axi = sqrt(m->y_eta[id] * m->y_eta[id] + m->x_eta[id] * m->x_eta[id]);
        double aeta = sqrt(m->y_xi[id] * m->y_xi[id] + m->x_xi[id] * m->x_xi[id]);
        double lxi = fabs(m->y_eta[id] * u - m->x_eta[id] * v) + c * axi;
        double leta = fabs(-m->y_xi[id] * u + m->x_xi[id] * v) + c * aeta;
        double lam = lxi + leta;
        if (kv > 0.0) {
            double a = (axi + aeta) / m->J[id];
            lam += m->J[id] * epsk[id / ((size_t)n * n)] * kv * a * a;
        }
        if (lam > 0.0) {
            double t = m->J[id] / lam;
            if (t < min_ratio) min_ratio = t;
        }
    }
    free(epsk);
    double cfl = m->p.cfl * 2.0 / (N + 1.0) * min_ratio;
    double pos = INFINITY;
    double w0 = 2.0 / (N * (N + 1.0));
    if (m->p.limiter && m->p.flux) {
        for (int k = 0; k < K; ++k)
            for (int f = 0; f < NF; ++f) {
                int kk = m->EToE[NF * k + f], ff = m->EToF[NF * k + f];
                int wall = kk < 0;
                for (int p = 0; p < n; ++p) {
                    int i, j;
                    face_node(N, f, p, &i, &j);
                    size_t im = nid(m, k, i, j), ip = im;
                    if (!wall) {
                        int q = neighbour_node(m, k, f, p), ii, jj;
                        face_node(N, ff, q, &ii, &jj);
                        ip = nid(m, kk, ii, jj);
                    }
                    double nx, ny;
                    outward_normal(m, k, f, p, &nx, &ny);
                    double Jsurf = sqrt(nx * nx + ny * ny);
                    nx /= Jsurf;
                    ny /= Jsurf;
                    double hm = W[im], hp = W[ip];
                    double utm = nx * velocity(hm, W[nn + im]) + ny * velocity(hm, W[2 * nn + im]);
                    /* the mirror state at a wall reverses the normal velocity */
                    double utp = wall ? -utm : nx * velocity(hp, W[nn + ip]) + ny * velocity(hp, W[2 * nn + ip]);
                    double ut_avg = 0.5 * (utm + utp);
                    double c_avg = 0.5 * (sqrt(g * fmax(hm, 0.0)) + sqrt(g * fmax(hp, 0.0)));
                    double A = fabs(ut_avg + c_avg) + fabs(ut_avg - c_avg);
                    double B = fabs(ut_avg + c_avg) - fabs(ut_avg - c_avg);
                    double a = m->J[im] / Jsurf;
                    double den = A + 2.0 * ut_avg;
                    if (den > 0.0) pos = fmin(pos, w0 * a / den);
                    double jump = utp - utm;
                    if (hm > 0.0 && B * jump < 0.0)
                        pos = fmin(pos, fabs(w0 * a * g * hm / (c_avg * B * jump)));
                }
            }
    }
    if (dt_cfl) *dt_cfl = cfl;
    if (dt_pos) *dt_pos = pos;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Time integration                                                    */
/* ------------------------------------------------------------------ */

/* Carpenter & Kennedy (1994) five-stage, fourth-order 2N-storage scheme. */
static const double LSRK_A[5] = {0.0,
                                 -567301805773.0 / 1357537059087.0,
                                 -2404267990393.0 / 2016746695238.0,
                                 -3550918686646.0 / 2091501179385.0,
                                 -1275806237668.0 / 842570457699.0};
static const double LSRK_B[5] = {1432997174477.0 / 9575080441755.0,
                                 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0,
                                 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};

void orc_lsrk_coefficients(double* A, double* B) {
    for (int s = 0; s < 5; ++s) {
        A[s] = LSRK_A[s];
        B[s] = LSRK_B[s];
    }
}

static int stage_limit(orc_mesh* m, double* W) {
    return m->p.limiter ? orc_limit(m, W) : ORC_OK;
}

int orc_step(orc_mesh* m, double* W, double dt_in, int nsteps, double* dt_last) {
    if (!m || !W || nsteps < 0) return ORC_ERR_ARG;
    size_t nn3 = 3 * (size_t)m->K * m->n * m->n;
    double* Wn = dalloc(nn3);
    double* Rw = dalloc(nn3);
    double* Kr = dalloc(nn3);
    int rc = ORC_OK;
    for (int s = 0; s < nsteps && rc == ORC_OK; ++s) {
        double dt = dt_in;
        if (!(dt > 0.0)) {
            double dc, dp;
            orc_max_dt(m, W, &dc, &dp);
            dt = fmin(dc, dp);
        }
        if (dt_last) *dt_last = dt;
        memcpy(Wn, W, nn3 * sizeof(double));
        if (m->p.rk == 0) {
            for (size_t a = 0; a < nn3; ++a) Kr[a] = 0.0;
            for (int st = 0; st < 5 && rc == ORC_OK; ++st) {
                orc_rhs(m, W, Rw);
                for (size_t a = 0; a < nn3; ++a) {
                    Kr[a] = LSRK_A[st] * Kr[a] + dt * Rw[a];
                    W[a] = W[a] + LSRK_B[st] * Kr[a];
                }
                rc = stage_limit(m, W);
            }
        } else {
            /* Eq. RKSSP */
            orc_rhs(m, W, Rw);
            for (size_t a = 0; a < nn3; ++a) W[a] = Wn[a] + dt * Rw[a];
            rc = stage_limit(m, W);
            if (rc == ORC_OK) {
                orc_rhs(m, W, Rw);
                for (size_t a = 0; a < nn3; ++a) W[a] = 0.75 * Wn[a] + 0.25 * (W[a] + dt * Rw[a]);
                rc = stage_limit(m, W);
            }
            if (rc == ORC_OK) {
                orc_rhs(m, W, Rw);
                for (size_t a = 0; a < nn3; ++a)
                    W[a] = Wn[a] / 3.0 + 2.0 / 3.0 * (W[a] + dt * Rw[a]);
                rc = stage_limit(m, W);
            }
        }
        if (rc != ORC_OK) memcpy(W, Wn, nn3 * sizeof(double));
    }
    free(Wn);
    free(Rw);
    free(Kr);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics                                                         */
/* ------------------------------------------------------------------ */

int orc_mass(const orc_mesh* m, const double* W, double* out3) {
    if (!m || !W || !out3) return ORC_ERR_ARG;
    int n = m->n;
    size_t nn = (size_t)m->K * n * n;
    for (int c = 0; c < 3; ++c) out3[c] = 0.0;
    for (int k = 0; k < m->K; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double wJ = m->w[i] * m->w[j] * m->J[id];
                for (int c = 0; c < 3; ++c) out3[c] += wJ * W[c * nn + id];
            }
    return ORC_OK;
}

/* Total entropy sum J w_i w_j e(W_ij) with e of Eq. entropyFunction. */
int orc_entropy(const orc_mesh* m, const double* W, double* E) {
    if (!m || !W || !E) return ORC_ERR_ARG;
    int n = m->n;
    size_t nn = (size_t)m->K * n * n;
    double s = 0.0;
    for (int k = 0; k < m->K; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double h = W[id], u = velocity(h, W[nn + id]), v = velocity(h, W[2 * nn + id]);
                double e = 0.5 * h * (u * u + v * v) + 0.5 * m->g * h * h + m->g * h * m->b[id];
                s += m->w[i] * m->w[j] * m->J[id] * e;
            }
    *E = s;
    return ORC_OK;
}

/* Discrete entropy rate: sum J w_i w_j q(W_ij) . R_ij with the entropy
 * variables q = (g(h+b) - (u^2+v^2)/2, u, v) of Eq. entropyVariables and
 * R = orc_rhs(W) (Sec. 2: the entropy function contracted with the
 * semi-discrete time derivative). scale (nullable) receives
 * sum J w_i w_j sum_c |q_c R_c|. */
int orc_entropy_rate(orc_mesh* m, const double* W, double* rate, double* scale) {
    if (!m || !W || !rate) return ORC_ERR_ARG;
    int n = m->n;
    size_t nn = (size_t)m->K * n * n;
    double* R = (double*)malloc(3 * nn * sizeof(double));
    if (!R) return ORC_ERR_ARG;
    int rc = orc_rhs(m, W, R);
    if (rc != ORC_OK) {
        free(R);
        return rc;
    }
    double s = 0.0, a = 0.0;
    for (int k = 0; k < m->K; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                size_t id = nid(m, k, i, j);
                double h = W[id], u = velocity(h, W[nn + id]), v = velocity(h, W[2 * nn + id]);
                double q[3] = {m->g * (h + m->b[id]) - 0.5 * (u * u + v * v), u, v};
                double wJ = m->w[i] * m->w[j] * m->J[id];
                for (int c = 0; c < 3; ++c) {
                    s += wJ * q[c] * R[c * nn + id];
                    a += wJ * fabs(q[c] * R[c * nn + id]);
                }
            }
    free(R);
    *rate = s;
    if (scale) *scale = a;
    return ORC_OK;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
