// LGL basis of degree N (Sec. 2.2) and the inverse Vandermonde matrix of the
// normalised Legendre polynomials (App. A), computed on the host once.
//
// Nodes: Newton iteration on x L_N(x) - L_{N-1}(x), whose zeros are the N+1
// LGL nodes (including +-1), started from Chebyshev-Gauss-Lobatto points.
// Weights: 2 / (N (N+1) L_N(x)^2). Derivative matrix: barycentric formula with
// the diagonal set to minus the row sum (so D annihilates constants exactly
// up to rounding of that sum). Inverse Vandermonde: the Gauss-quadrature
// projection of App. A, Vinv_ij = sum_l Ltilde_i(xg_l) l_j(xg_l) wg_l, which
// is exact because Ltilde_i l_j has degree <= 2N.
#include <cmath>

#include "swe_internal.h"

namespace swe {
namespace {

const double kPi = 3.14159265358979323846;

// L_0..L_N at x.
void legendre(int N, double x, double* L) {
    L[0] = 1.0;
    if (N >= 1) L[1] = x;
    for (int k = 2; k <= N; ++k) L[k] = ((2 * k - 1) * x * L[k - 1] - (k - 1) * L[k - 2]) / k;
}

std::vector<double> lgl_nodes(int N) {
    std::vector<double> x(N + 1);
    double L[NMAX + 2];
    for (int i = 0; i <= N; ++i) {
        double xi = std::cos(kPi * i / N);
        for (int it = 0; it < 200; ++it) {
            legendre(N, xi, L);
            double f = xi * L[N] - L[N - 1];
            double dx = f / ((N + 1) * L[N]);
            xi -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        x[N - i] = xi;  // ascending order
    }
    x[0] = -1.0;
    x[N] = 1.0;
    return x;
}

// Gauss-Legendre nodes and weights with n points.
void gauss(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    double L[NMAX + 3];
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dP = 1.0;
        for (int it = 0; it < 200; ++it) {
            legendre(n, z, L);
            dP = n * (z * L[n] - L[n - 1]) / (z * z - 1.0);
            double dz = L[n] / dP;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        legendre(n, z, L);
        dP = n * (z * L[n] - L[n - 1]) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
    }
}

}  // namespace

Basis make_basis(int N) {
    Basis B;
    B.N = N;
    const int n = N + 1;
    B.xi = lgl_nodes(N);
    B.w.resize(n);
    double L[NMAX + 2];
    for (int i = 0; i < n; ++i) {
        legendre(N, B.xi[i], L);
        B.w[i] = 2.0 / (N * (N + 1.0) * L[N] * L[N]);
    }
    // barycentric weights
    std::vector<double> lam(n, 1.0);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k)
            if (k != j) lam[j] /= (B.xi[j] - B.xi[k]);
    B.D.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double row = 0.0;
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            double d = (lam[j] / lam[i]) / (B.xi[i] - B.xi[j]);
            B.D[i * n + j] = d;
            row += d;
        }
        B.D[i * n + i] = -row;
    }
    // inverse Vandermonde by Gauss projection
    std::vector<double> xg, wg;
    gauss(n, xg, wg);
    B.Vinv.assign(n * n, 0.0);
    for (int l = 0; l < n; ++l) {
        double Lg[NMAX + 2];
        legendre(N, xg[l], Lg);
        // Lagrange basis on the LGL nodes at xg[l] (barycentric form)
        // (when N is even, the Gauss and LGL node sets share x = 0)
        double s = 0.0, lag[NMAX + 1];
        int hit = -1;
        for (int j = 0; j < n; ++j) {
            if (xg[l] == B.xi[j] || std::fabs(xg[l] - B.xi[j]) < 1e-15) hit = j;
        }
        for (int j = 0; j < n; ++j) {
            if (hit >= 0) {
                lag[j] = (j == hit) ? 1.0 : 0.0;
                continue;
            }
            lag[j] = lam[j] / (xg[l] - B.xi[j]);
            s += lag[j];
        }
        if (hit < 0)
            for (int j = 0; j < n; ++j) lag[j] /= s;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                B.Vinv[i * n + j] += std::sqrt(i + 0.5) * Lg[i] * lag[j] * wg[l];
    }
    return B;
}

const Tables& tables() {
    static Tables T = [] {
        Tables t{};
        for (int N = 1; N <= NMAX; ++N) {
            Basis B = make_basis(N);
            const int n = N + 1;
            for (int a = 0; a < n * n; ++a) {
                t.D[mat_offset(N) + a] = B.D[a];
                t.Vinv[mat_offset(N) + a] = B.Vinv[a];
            }
            for (int a = 0; a < n; ++a) t.w[vec_offset(N) + a] = B.w[a];
        }
        return t;
    }();
    return T;
}

}  // namespace swe
