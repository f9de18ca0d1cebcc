// tables.cpp -- 1-D reference tables of the GPU path (host code).
//
// Gauss-Legendre points (p+2 per direction) are the eigenvalues of the
// symmetric Jacobi matrix of the Legendre recurrence (Golub-Welsch), found
// here by Sturm-sequence bisection; weights 2/((1-x^2) P'_n(x)^2).  The
// Gauss-Lobatto-Legendre nodes are -1, 1 and the roots of P'_p, found by
// Newton from Chebyshev-Lobatto guesses.  Lagrange values and derivatives use
// the barycentric form.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>
#include "common.cuh"

namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence
void legendre(int n, double x, double* P, double* dP) {
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        double d2 = d0 + (2 * k - 1) * p1;          // P'_k = P'_{k-2} + (2k-1) P_{k-1}
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *P = p1; *dP = d1;
}

// number of eigenvalues < x of the Jacobi matrix (Sturm count); off-diagonal
// b_k = k / sqrt(4k^2 - 1), zero diagonal
int sturm_count(int n, double x) {
    int cnt = 0;
    double d = -x;
    if (d < 0) ++cnt;
    for (int k = 1; k < n; ++k) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        if (d == 0.0) d = 1e-300;
        d = -x - b * b / d;
        if (d < 0) ++cnt;
    }
    return cnt;
}

void gauss_points(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double lo = -1.0, hi = 1.0;      // i-th smallest eigenvalue
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (sturm_count(n, mid) > i) hi = mid; else lo = mid;
        }
        double z = 0.5 * (lo + hi), P, dP;
        for (int it = 0; it < 3; ++it) { legendre(n, z, &P, &dP); z -= P / dP; }   // polish
        legendre(n, z, &P, &dP);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
    }
}

void lobatto_nodes(int p, double* x) {
    x[0] = -1.0; x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double z = -std::cos(M_PI * i / p);
        for (int it = 0; it < 100; ++it) {
            // roots of P'_p: Newton on P'_p with P''_p from the Legendre ODE
            double P, dP;
            legendre(p, z, &P, &dP);
            double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
            double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
}

}  // namespace

void host_build_tables(int p, int m, Tab* t) {
    std::memset(t, 0, sizeof(*t));
    t->p = p; t->m = m; t->n = m * p + 1; t->ng = p + 2; t->nq = m * (p + 2);
    t->Nn = t->n * t->n * t->n; t->n2 = t->n * t->n;
    t->nl = (p + 1) * (p + 1) * (p + 1);
    t->npt = (p + 2) * (p + 2) * (p + 2);
    double xi[MEHDG_MAXP + 1], eta[MEHDG_MAXG], om[MEHDG_MAXG];
    lobatto_nodes(p, xi);
    gauss_points(p + 2, eta, om);
    // barycentric weights
    double bw[MEHDG_MAXP + 1];
    for (int l = 0; l <= p; ++l) {
        double s = 1.0;
        for (int j = 0; j <= p; ++j) if (j != l) s *= (xi[l] - xi[j]);
        bw[l] = 1.0 / s;
    }
    for (int g = 0; g < p + 2; ++g) {
        double z = eta[g];
        t->w[g] = om[g];
        // l(z) = prod (z - xi_j); L_l(z) = l(z) bw_l / (z - xi_l)  (z is never a node)
        double lz = 1.0, S1 = 0.0;
        for (int j = 0; j <= p; ++j) { lz *= (z - xi[j]); S1 += 1.0 / (z - xi[j]); }
        for (int l = 0; l <= p; ++l) {
            double Ll = lz * bw[l] / (z - xi[l]);
            t->L[g][l] = Ll;
            // L_l'(z) = L_l(z) * sum_{j != l} 1/(z - xi_j)
            t->dL[g][l] = Ll * (S1 - 1.0 / (z - xi[l]));
        }
    }
}

// 1-D operators of the gradient equation (eq. s32a) on the macro grid of one
// direction, for a reference micro-interval of length 2 (physical operators:
// M1 = (h/2) M1_ref, G1 = G1_ref):
//   M1_ref[a][b] = sum_e sum_g w_g phi_a phi_b,  G1_ref[a][b] = sum_e sum_g w_g phi_b dphi_a/dxi
// Outputs (n x n, row-major): Minv_ref = M1_ref^-1 and C1_ref = M1_ref^-1 G1_ref,
// so that A_qq^-1 A_qv acts along the d-lines as (2/h_d) C1_ref.
void host_build_qtables(const Tab& t, double* Minv_ref, double* C1_ref) {
    const int n = t.n, p = t.p, m = t.m;
    std::vector<double> M(n * n, 0.0), G(n * n, 0.0), A(n * 2 * n, 0.0);
    for (int e = 0; e < m; ++e)
        for (int g = 0; g < t.ng; ++g)
            for (int la = 0; la <= p; ++la)
                for (int lb = 0; lb <= p; ++lb) {
                    int a = e * p + la, b = e * p + lb;
                    M[a * n + b] += t.w[g] * t.L[g][la] * t.L[g][lb];
                    G[a * n + b] += t.w[g] * t.L[g][lb] * t.dL[g][la];
                }
    // Gauss-Jordan with partial pivoting on [M | I]
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) { A[i * 2 * n + j] = M[i * n + j]; A[i * 2 * n + n + j] = (i == j); }
    for (int c = 0; c < n; ++c) {
        int r = c;
        for (int i = c + 1; i < n; ++i) if (std::fabs(A[i * 2 * n + c]) > std::fabs(A[r * 2 * n + c])) r = i;
        if (r != c) for (int j = 0; j < 2 * n; ++j) std::swap(A[c * 2 * n + j], A[r * 2 * n + j]);
        double inv = 1.0 / A[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) A[c * 2 * n + j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            double f = A[i * 2 * n + c];
            if (f != 0.0) for (int j = 0; j < 2 * n; ++j) A[i * 2 * n + j] -= f * A[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Minv_ref[i * n + j] = A[i * 2 * n + n + j];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += Minv_ref[i * n + k] * G[k * n + j];
            C1_ref[i * n + j] = s;
        }
}
