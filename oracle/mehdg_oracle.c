/*
 * mehdg_oracle.c -- plain, slow FP64 CPU oracle for the per-macro-element
 * Newton step of the entropy-variable macro-element HDG method
 * (Badrkhani, ten Eikelder, Hasse, Schillinger, arXiv 2507.22195).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path: every table (Gauss and
 * Gauss-Lobatto points, Lagrange values) and every formula is restated here
 * from the paper.
 *
 * Conventions (the same interface layouts as the C-ABI, written out again):
 *   macro-element K = axis-aligned box, split into m^3 hexahedral micro-
 *   elements, each Q_p on Gauss-Lobatto-Legendre nodes, C0 inside K
 *   (Sec. 3.1 with hexahedra instead of simplices);  n = m p + 1 nodes per
 *   direction, node A = i + n (j + n k).
 *   v, v*  : [5][Nn]        entropy variables (eq. s222), Nn = n^3
 *   q      : [5][3][Nn]     gradient of v (eq. s32a)
 *   trace  : [6][5][n^2]    faces x-,x+,y-,y+,z-,z+; face node c = i_t1 + n i_t2
 *   Quadrature: tensor Gauss rule with p+2 points per direction per
 *   micro-element, on the volume and on the faces.
 *
 * Every point-wise physics function is written once over complex doubles so
 * that the same code gives the residual (imaginary part zero) and, by the
 * complex-step method (step 1e-30), derivatives exact to round-off.
 *
 * Readings of the paper taken here where it is silent or ambiguous are
 * documented beside the code that takes them.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Parameters                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    double gamma;   /* ratio of specific heats (Sec. 2.1)                     */
    double Re;      /* Reynolds number                                       */
    double Pr;      /* Prandtl number                                        */
    double Mach;    /* reference Mach number M_inf                           */
    double dt;      /* time step of the implicit stage term (eq. C242)       */
    int viscous;    /* 1: Navier-Stokes (G, G-hat), 0: Euler                 */
    int flux;       /* 0 EC (eq. EC), 1 ES (eq. Flux_En_Inv), 2 KEPES (eq. ES)*/
    int time_term;  /* 1: include (u(v)-u(v*))/dt (eq. C242, one stage)     */
} orc_params;

enum { ORC_EC = 0, ORC_ES = 1, ORC_KEPES = 2 };

/* ------------------------------------------------------------------ */
/* 1-D tables                                                          */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre rule with np points on [-1,1]: Newton iteration on the
 * Legendre polynomial P_np evaluated by its three-term recurrence. */
int orc_gauss(int np, double *x, double *w)
{
    if (np < 1 || np > 32) return -1;
    for (int i = 0; i < np; ++i) {
        double z = cos(M_PI * (i + 0.75) / (np + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= np; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (np == 1) { p1 = z; p0 = 1.0; }
            /* derivative of P_np */
            double dp = np * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= np; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        if (np == 1) { p1 = z; p0 = 1.0; }
        double dp = np * (z * p1 - p0) / (z * z - 1.0);
        x[np - 1 - i] = z;                       /* ascending order */
        w[np - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Gauss-Lobatto-Legendre nodes for degree p <= 4, closed forms. */
int orc_gll(int p, double *x)
{
    switch (p) {
    case 1: x[0] = -1; x[1] = 1; return 0;
    case 2: x[0] = -1; x[1] = 0; x[2] = 1; return 0;
    case 3: x[0] = -1; x[1] = -1.0 / sqrt(5.0); x[2] = 1.0 / sqrt(5.0); x[3] = 1; return 0;
    case 4: x[0] = -1; x[1] = -sqrt(3.0 / 7.0); x[2] = 0; x[3] = sqrt(3.0 / 7.0); x[4] = 1; return 0;
    default: return -1;
    }
}

/* Lagrange basis of the nodes xi[0..p] at point z: value and derivative,
 * product formula. */
static void lagrange(int p, const double *xi, double z, double *L, double *dL)
{
    for (int l = 0; l <= p; ++l) {
        double val = 1.0, der = 0.0;
        for (int mm = 0; mm <= p; ++mm) {
            if (mm == l) continue;
            double den = xi[l] - xi[mm];
            /* derivative of the product by the product rule */
            double prod = 1.0 / den;
            for (int r = 0; r <= p; ++r) {
                if (r == l || r == mm) continue;
                prod *= (z - xi[r]) / (xi[l] - xi[r]);
            }
            der += prod;
            val *= (z - xi[mm]) / den;
        }
        L[l] = val; dL[l] = der;
    }
}

/* ------------------------------------------------------------------ */
/* Geometry of one macro-element                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    int p, m, n, ng, nq, Nn, n2;
    double h[3];                 /* micro-element edge lengths            */
    double xi[8];                /* GLL nodes (p+1)                        */
    double eta[8], om[8];        /* Gauss points and weights (p+2)         */
    double Lv[8][8], Ld[8][8];   /* L_l(eta_g), dL_l/dxi(eta_g)            */
} geo_t;

static int geo_init(geo_t *g, int p, int m, const double box[6])
{
    if (p < 1 || p > 4 || m < 1) return -1;
    g->p = p; g->m = m; g->n = m * p + 1; g->ng = p + 2; g->nq = m * (p + 2);
    g->Nn = g->n * g->n * g->n; g->n2 = g->n * g->n;
    for (int d = 0; d < 3; ++d) g->h[d] = (box[3 + d] - box[d]) / m;
    if (orc_gll(p, g->xi)) return -1;
    orc_gauss(p + 2, g->eta, g->om);
    for (int gq = 0; gq < p + 2; ++gq) lagrange(p, g->xi, g->eta[gq], g->Lv[gq], g->Ld[gq]);
    return 0;
}

/* macro node index from the three per-direction node indices */
static inline int node3(const geo_t *g, int i, int j, int k) { return i + g->n * (j + g->n * k); }

/* tangential directions of face direction d, in increasing order */
static inline void face_dirs(int d, int *t1, int *t2)
{
    if (d == 0) { *t1 = 1; *t2 = 2; }
    else if (d == 1) { *t1 = 0; *t2 = 2; }
    else { *t1 = 0; *t2 = 1; }
}

/* macro node index of face node (c1, c2) of face f */
static inline int face_node(const geo_t *g, int f, int c1, int c2)
{
    int d = f / 2, side = f % 2, t1, t2, idx[3];
    face_dirs(d, &t1, &t2);
    idx[d] = side ? g->n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
    return node3(g, idx[0], idx[1], idx[2]);
}

/* ------------------------------------------------------------------ */
/* Point-wise physics over complex doubles                            */
/* ------------------------------------------------------------------ */

/* |x| for complex-step: x sgn(Re x), sgn(0) = +1 */
static inline cplx cabs_cs(cplx x) { return creal(x) >= 0 ? x : -x; }

/* Logarithmic mean (eq. avg) with the Ismail-Roe evaluation: zeta = b/a,
 * f = (zeta-1)/(zeta+1), u = f^2; series 1 + u/3 + u^2/5 + u^3/7 when
 * u < 1e-4 (threshold not printed in the paper; reading), else ln(zeta)/(2f);
 * mean = (a+b)/(2F). */
static cplx logmean(cplx a, cplx b)
{
    cplx zeta = b / a;
    cplx f = (zeta - 1.0) / (zeta + 1.0);
    cplx u = f * f;
    cplx F;
    if (creal(u) < 1e-4) F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
    else F = clog(zeta) / (2.0 * f);
    return (a + b) / (2.0 * F);
}

/* Primitive state from entropy variables: inverse of eq. s222.
 * beta = -v5, V = (v2,v3,v4)/beta, s = gamma - (gamma-1)(v1 + beta|V|^2/2),
 * rho = (beta e^s)^(1/(1-gamma)), P = rho/beta.                          */
typedef struct { cplx rho, V[3], P, beta, E; } prim_t;

static void prim_from_v(const cplx *v, double gm, prim_t *w)
{
    cplx b = -v[4];
    w->beta = b;
    for (int i = 0; i < 3; ++i) w->V[i] = v[1 + i] / b;
    cplx V2 = w->V[0] * w->V[0] + w->V[1] * w->V[1] + w->V[2] * w->V[2];
    cplx s = gm - (gm - 1.0) * (v[0] + b * V2 / 2.0);
    w->rho = cexp((clog(b) + s) / (1.0 - gm));
    w->P = w->rho / b;
    w->E = w->P / (gm - 1.0) + 0.5 * w->rho * V2;   /* rho E */
}

/* conservative variables u = (rho, rho V, rho E) (Sec. 2.1) */
static void cons_from_prim(const prim_t *w, cplx *u)
{
    u[0] = w->rho;
    for (int i = 0; i < 3; ++i) u[1 + i] = w->rho * w->V[i];
    u[4] = w->E;
}

/* inviscid flux column j: F_j = [rho V_j, rho V V_j + P e_j, V_j (rho E + P)] (eq. C5) */
static void flux_col(const prim_t *w, int j, cplx *Fj)
{
    Fj[0] = w->rho * w->V[j];
    for (int i = 0; i < 3; ++i) Fj[1 + i] = w->rho * w->V[i] * w->V[j] + (i == j ? w->P : 0.0);
    Fj[4] = w->V[j] * (w->E + w->P);
}

static void flux_normal(const prim_t *w, const double *n, cplx *Fn)
{
    cplx Fj[5];
    for (int k = 0; k < 5; ++k) Fn[k] = 0;
    for (int j = 0; j < 3; ++j) {
        if (n[j] == 0.0) continue;
        flux_col(w, j, Fj);
        for (int k = 0; k < 5; ++k) Fn[k] += Fj[k] * n[j];
    }
}

/* Entropy Jacobian A0 = du/dv in closed form (symmetric positive definite):
 * rows/cols (rho, rho V, rho E); E_t = rho E, H = (E_t+P)/rho, a^2 = gamma P/rho.
 *   [ rho,   rho V^T,            E_t                 ]
 *   [ rho V, rho V V^T + P I,    (E_t+P) V           ]
 *   [ E_t,   (E_t+P) V^T,        rho H^2 - a^2 P/(gamma-1) ]          */
static void A0_closed(const prim_t *w, double gm, cplx A[5][5])
{
    cplx Et = w->E, H = (Et + w->P) / w->rho, a2 = gm * w->P / w->rho;
    A[0][0] = w->rho;
    for (int i = 0; i < 3; ++i) {
        A[0][1 + i] = A[1 + i][0] = w->rho * w->V[i];
        A[4][1 + i] = A[1 + i][4] = (Et + w->P) * w->V[i];
        for (int j = 0; j < 3; ++j)
            A[1 + i][1 + j] = w->rho * w->V[i] * w->V[j] + (i == j ? w->P : 0.0);
    }
    A[0][4] = A[4][0] = Et;
    A[4][4] = w->rho * H * H - a2 * w->P / (gm - 1.0);
}

/* ES flux, eq. Flux_En_Inv: 1/2 (F(vh) + F(v)).n - 1/2 sigma(vh) A0(vh) [[v]],
 * sigma = lambda_max(vh) = |Vh.n| + c_h (reading: A0 and sigma at vh). */
static void flux_es(const cplx *vh, const cplx *v, const double *n, double gm, cplx *out)
{
    prim_t a, b; prim_from_v(v, gm, &a); prim_from_v(vh, gm, &b);
    cplx Fa[5], Fb[5], A0[5][5];
    flux_normal(&a, n, Fa); flux_normal(&b, n, Fb);
    A0_closed(&b, gm, A0);
    cplx vn = b.V[0] * n[0] + b.V[1] * n[1] + b.V[2] * n[2];
    cplx sig = cabs_cs(vn) + csqrt(gm * b.P / b.rho);
    for (int k = 0; k < 5; ++k) {
        cplx s = 0;
        for (int l = 0; l < 5; ++l) s += A0[k][l] * (vh[l] - v[l]);
        out[k] = 0.5 * (Fa[k] + Fb[k]) - 0.5 * sig * s;
    }
}

/* Averages shared by the EC and KEPES fluxes (eq. avg, eq. EC). */
typedef struct { cplx rln, bln, Vb[3], rb, bb, Pb, VV; prim_t a, b; } avg_t;

static void averages(const cplx *vh, const cplx *v, double gm, avg_t *s)
{
    prim_from_v(v, gm, &s->a); prim_from_v(vh, gm, &s->b);
    s->rln = logmean(s->a.rho, s->b.rho);
    s->bln = logmean(s->a.beta, s->b.beta);
    for (int i = 0; i < 3; ++i) s->Vb[i] = 0.5 * (s->a.V[i] + s->b.V[i]);
    s->rb = 0.5 * (s->a.rho + s->b.rho);
    s->bb = 0.5 * (s->a.beta + s->b.beta);
    s->Pb = s->rb / s->bb;
    cplx Va2 = 0, Vb2 = 0;
    for (int i = 0; i < 3; ++i) { Va2 += s->a.V[i] * s->a.V[i]; Vb2 += s->b.V[i] * s->b.V[i]; }
    s->VV = 0.5 * (Va2 + Vb2);          /* mean of |V|^2 */
}

/* EC (and KEP) flux, eq. EC. */
static void flux_ec_from(const avg_t *s, const double *n, double gm, cplx *out)
{
    cplx Vn = s->Vb[0] * n[0] + s->Vb[1] * n[1] + s->Vb[2] * n[2];
    cplx f1 = s->rln * Vn;
    cplx f2[3];
    for (int i = 0; i < 3; ++i) f2[i] = s->Vb[i] * f1 + s->Pb * n[i];
    cplx f3 = (1.0 / (s->bln * (gm - 1.0)) - s->VV / 2.0) * f1
            + s->Vb[0] * f2[0] + s->Vb[1] * f2[1] + s->Vb[2] * f2[2];
    out[0] = f1; out[1] = f2[0]; out[2] = f2[1]; out[3] = f2[2]; out[4] = f3;
}

/* Orthonormal tangents for an axis-aligned (or general) unit normal. */
static void tangents(const double *n, double *t1, double *t2)
{
    /* pick the axis least aligned with n, Gram-Schmidt, then t2 = n x t1 */
    double a[3] = {0, 0, 0};
    int im = 0;
    for (int i = 1; i < 3; ++i) if (fabs(n[i]) < fabs(n[im])) im = i;
    a[im] = 1.0;
    double dd = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
    for (int i = 0; i < 3; ++i) t1[i] = a[i] - dd * n[i];
    double nn = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int i = 0; i < 3; ++i) t1[i] /= nn;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

/* KEPES matrices (eqs. KEPES3-KEPES5): averaged right eigenvectors R (columns
 * rotated to the normal n), |Lambda| with the pressure-based hybrid theta,
 * and Barth's scaling T.  Eigenvalues (reading): |lambda_1| = |lambda_5| =
 * |vn| + c, |lambda_2..4| = |vn|, lambda_max = |vn| + c, all from averages. */
static void kepes_mats(const avg_t *s, const double *n, double gm,
                       cplx R[5][5], cplx Lam[5], cplx T[5])
{
    double t1[3], t2[3];
    tangents(n, t1, t2);
    cplx c = csqrt(gm * s->Pb / s->rln);
    cplx hb = gm / (s->bln * (gm - 1.0)) + 0.5 * s->VV;
    cplx vn = s->Vb[0] * n[0] + s->Vb[1] * n[1] + s->Vb[2] * n[2];
    cplx vt1 = s->Vb[0] * t1[0] + s->Vb[1] * t1[1] + s->Vb[2] * t1[2];
    cplx vt2 = s->Vb[0] * t2[0] + s->Vb[1] * t2[1] + s->Vb[2] * t2[2];
    /* column 0: 1, V - c n, h - c vn */
    R[0][0] = 1; R[4][0] = hb - c * vn;
    R[0][1] = 1; R[4][1] = 0.5 * s->VV;
    R[0][2] = 0; R[4][2] = vt1;
    R[0][3] = 0; R[4][3] = vt2;
    R[0][4] = 1; R[4][4] = hb + c * vn;
    for (int i = 0; i < 3; ++i) {
        R[1 + i][0] = s->Vb[i] - c * n[i];
        R[1 + i][1] = s->Vb[i];
        R[1 + i][2] = t1[i];
        R[1 + i][3] = t2[i];
        R[1 + i][4] = s->Vb[i] + c * n[i];
    }
    cplx avn = cabs_cs(vn);
    cplx lmax = avn + c;
    cplx x = (s->a.P - s->b.P) / (s->a.P + s->b.P);
    cplx theta = (creal(x) == 0.0) ? 0.0 : csqrt(cabs_cs(x));
    cplx lam[5] = { avn + c, avn, avn, avn, avn + c };
    for (int i = 0; i < 5; ++i) Lam[i] = (1.0 - theta) * lam[i] + theta * lmax;
    T[0] = s->rln / (2.0 * gm);
    T[1] = s->rln * (gm - 1.0) / gm;
    T[2] = s->Pb; T[3] = s->Pb;
    T[4] = s->rln / (2.0 * gm);
}

/* KEPES flux, eq. ES: Fbar - 1/2 R |Lambda| T R^T [[v]] */
static void flux_kepes(const cplx *vh, const cplx *v, const double *n, double gm, cplx *out)
{
    avg_t s; averages(vh, v, gm, &s);
    cplx Fb[5], R[5][5], Lam[5], T[5], w[5];
    flux_ec_from(&s, n, gm, Fb);
    kepes_mats(&s, n, gm, R, Lam, T);
    for (int i = 0; i < 5; ++i) {
        cplx t = 0;
        for (int k = 0; k < 5; ++k) t += R[k][i] * (vh[k] - v[k]);
        w[i] = t * Lam[i] * T[i];
    }
    for (int k = 0; k < 5; ++k) {
        cplx t = 0;
        for (int i = 0; i < 5; ++i) t += R[k][i] * w[i];
        out[k] = Fb[k] - 0.5 * t;
    }
}

static void flux_ec(const cplx *vh, const cplx *v, const double *n, double gm, cplx *out)
{
    avg_t s; averages(vh, v, gm, &s);
    flux_ec_from(&s, n, gm, out);
}

/* Viscous constants (reading): mu constant, bulk lambda = -2/3, effective
 * viscosity mu/Re_c = Mach/Re (acoustic Reynolds number), heat conduction
 * coefficient mu_eff c_p / Pr with c_p = 1/(gamma-1) (gamma P = rho T). */
static inline double mu_eff(const orc_params *pr) { return pr->Mach / pr->Re; }
static inline double kap_eff(const orc_params *pr) { return pr->Mach / pr->Re / ((pr->gamma - 1.0) * pr->Pr); }

/* Viscous flux G(v, q) (eqs. C5, C6), q = grad v in entropy variables:
 * V_i = -v_{i+1}/v5, T = -gamma/v5, chain rule for grad V and grad T.
 * G[k*3+j] = column j (flux in direction j).                               */
static void visc_flux(const cplx *v, const cplx *q, const orc_params *pr, cplx *G)
{
    double gm = pr->gamma, mu = mu_eff(pr), ka = kap_eff(pr);
    cplx v5 = v[4], V[3], dV[3][3], dT[3], tau[3][3];
    for (int i = 0; i < 3; ++i) V[i] = -v[1 + i] / v5;
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d)
            dV[i][d] = -q[(1 + i) * 3 + d] / v5 + v[1 + i] * q[4 * 3 + d] / (v5 * v5);
    for (int d = 0; d < 3; ++d) dT[d] = gm * q[4 * 3 + d] / (v5 * v5);
    cplx dv = dV[0][0] + dV[1][1] + dV[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            tau[i][j] = mu * (dV[i][j] + dV[j][i] - (i == j ? (2.0 / 3.0) * dv : 0.0));
    for (int j = 0; j < 3; ++j) {
        G[0 * 3 + j] = 0;
        for (int i = 0; i < 3; ++i) G[(1 + i) * 3 + j] = -tau[i][j];
        cplx tv = tau[j][0] * V[0] + tau[j][1] * V[1] + tau[j][2] * V[2];
        cplx phi = -ka * dT[j];
        G[4 * 3 + j] = -(tv - phi);
    }
}

/* Volume integrand at one point: U = (u(v) - u(v*))/dt, FG = F(v) + G(v,q). */
static void vol_point(const orc_params *pr, const cplx *v, const cplx *vs, const cplx *q,
                      cplx *U, cplx *FG)
{
    prim_t w; prim_from_v(v, pr->gamma, &w);
    if (pr->time_term) {
        prim_t ws; prim_from_v(vs, pr->gamma, &ws);
        cplx u[5], us[5];
        cons_from_prim(&w, u); cons_from_prim(&ws, us);
        for (int k = 0; k < 5; ++k) U[k] = (u[k] - us[k]) / pr->dt;
    } else {
        for (int k = 0; k < 5; ++k) U[k] = 0;
    }
    for (int j = 0; j < 3; ++j) {
        cplx Fj[5]; flux_col(&w, j, Fj);
        for (int k = 0; k < 5; ++k) FG[k * 3 + j] = Fj[k];
    }
    if (pr->viscous) {
        cplx G[15]; visc_flux(v, q, pr, G);
        for (int i = 0; i < 15; ++i) FG[i] += G[i];
    }
}

/* Face integrand F-hat + G-hat at one face point (eqs. Flux_En_Inv, EC, ES,
 * Flux_En_Vis); n = outward normal of the macro-element. */
static void face_point(const orc_params *pr, const cplx *vh, const cplx *v, const cplx *q,
                       const double *n, cplx *Fh)
{
    double gm = pr->gamma;
    if (pr->flux == ORC_EC) flux_ec(vh, v, n, gm, Fh);
    else if (pr->flux == ORC_ES) flux_es(vh, v, n, gm, Fh);
    else flux_kepes(vh, v, n, gm, Fh);
    if (pr->viscous) {
        cplx G[15]; visc_flux(vh, q, pr, G);      /* G(vh, q) . n */
        double sv[5];
        double M2 = pr->Mach * pr->Mach;
        sv[0] = 0; sv[1] = sv[2] = sv[3] = 1.0 / pr->Re;
        sv[4] = 1.0 / (pr->Re * (gm - 1.0) * M2 * pr->Pr);
        for (int k = 0; k < 5; ++k) {
            cplx gn = G[k * 3 + 0] * n[0] + G[k * 3 + 1] * n[1] + G[k * 3 + 2] * n[2];
            Fh[k] += gn - 0.5 * sv[k] * (vh[k] - v[k]);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Exported point-wise functions (for the pins)                        */
/* ------------------------------------------------------------------ */
static void to_c(const double *x, cplx *z, int n) { for (int i = 0; i < n; ++i) z[i] = x[i]; }

void orc_u_of_v(double gm, const double *v, double *u)
{
    cplx z[5], uu[5]; prim_t w; to_c(v, z, 5);
    prim_from_v(z, gm, &w); cons_from_prim(&w, uu);
    for (int k = 0; k < 5; ++k) u[k] = creal(uu[k]);
}

void orc_prim_of_v(double gm, const double *v, double *rho, double *V, double *P)
{
    cplx z[5]; prim_t w; to_c(v, z, 5); prim_from_v(z, gm, &w);
    *rho = creal(w.rho); *P = creal(w.P);
    for (int i = 0; i < 3; ++i) V[i] = creal(w.V[i]);
}

void orc_A0(double gm, const double *v, double *A)
{
    cplx z[5], M[5][5]; prim_t w; to_c(v, z, 5); prim_from_v(z, gm, &w);
    A0_closed(&w, gm, M);
    for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) A[i * 5 + j] = creal(M[i][j]);
}

/* complex-step du/dv */
void orc_dudv_cs(double gm, const double *v, double *J)
{
    const double h = 1e-30;
    for (int l = 0; l < 5; ++l) {
        cplx z[5], uu[5]; prim_t w; to_c(v, z, 5);
        z[l] += I * h;
        prim_from_v(z, gm, &w); cons_from_prim(&w, uu);
        for (int k = 0; k < 5; ++k) J[k * 5 + l] = cimag(uu[k]) / h;
    }
}

/* physical normal flux F(v).n */
void orc_flux_phys(double gm, const double *v, const double *n, double *Fn)
{
    cplx z[5], F[5]; prim_t w; to_c(v, z, 5); prim_from_v(z, gm, &w);
    flux_normal(&w, n, F);
    for (int k = 0; k < 5; ++k) Fn[k] = creal(F[k]);
}

/* numerical inviscid flux of the given kind */
void orc_flux_num(int kind, double gm, const double *vh, const double *v, const double *n, double *out)
{
    cplx a[5], b[5], o[5]; to_c(vh, a, 5); to_c(v, b, 5);
    if (kind == ORC_EC) flux_ec(a, b, n, gm, o);
    else if (kind == ORC_ES) flux_es(a, b, n, gm, o);
    else flux_kepes(a, b, n, gm, o);
    for (int k = 0; k < 5; ++k) out[k] = creal(o[k]);
}

/* full face integrand (inviscid + viscous) */
void orc_face_flux(const orc_params *pr, const double *vh, const double *v, const double *q,
                   const double *n, double *out)
{
    cplx a[5], b[5], qq[15], o[5]; to_c(vh, a, 5); to_c(v, b, 5);
    if (q) to_c(q, qq, 15); else for (int i = 0; i < 15; ++i) qq[i] = 0;
    face_point(pr, a, b, qq, n, o);
    for (int k = 0; k < 5; ++k) out[k] = creal(o[k]);
}

void orc_visc_flux(const orc_params *pr, const double *v, const double *q, double *G)
{
    cplx a[5], qq[15], o[15]; to_c(v, a, 5); to_c(q, qq, 15);
    visc_flux(a, qq, pr, o);
    for (int i = 0; i < 15; ++i) G[i] = creal(o[i]);
}

/* KEPES pieces for the Barth-scaling and entropy-stability pins:
 * R[25] row-major, Lam[5], T[5]. */
void orc_kepes_parts(double gm, const double *vh, const double *v, const double *n,
                     double *R, double *Lam, double *T)
{
    cplx a[5], b[5], RR[5][5], L[5], TT[5]; avg_t s;
    to_c(vh, a, 5); to_c(v, b, 5);
    averages(a, b, gm, &s);
    kepes_mats(&s, n, gm, RR, L, TT);
    for (int i = 0; i < 5; ++i) {
        Lam[i] = creal(L[i]); T[i] = creal(TT[i]);
        for (int j = 0; j < 5; ++j) R[i * 5 + j] = creal(RR[i][j]);
    }
}

double orc_logmean(double a, double b) { return creal(logmean(a, b)); }

/* ------------------------------------------------------------------ */
/* Residual of one macro-element (eq. s32 with the stage term C242)     */
/* ------------------------------------------------------------------ */

/* state at a volume point of micro-element (e1,e2,e3), Gauss point (g1,g2,g3) */
typedef struct {
    double W;                  /* quadrature weight incl. Jacobian        */
    int A[125];                /* macro nodes of the (p+1)^3 local nodes  */
    double phi[125], dphi[125][3];
    int nl;
} vpt_t;

static void vol_basis(const geo_t *g, int e1, int e2, int e3, int g1, int g2, int g3, vpt_t *P)
{
    int p = g->p;
    P->W = g->om[g1] * g->h[0] / 2 * g->om[g2] * g->h[1] / 2 * g->om[g3] * g->h[2] / 2;
    int t = 0;
    for (int l3 = 0; l3 <= p; ++l3)
        for (int l2 = 0; l2 <= p; ++l2)
            for (int l1 = 0; l1 <= p; ++l1, ++t) {
                P->A[t] = node3(g, e1 * p + l1, e2 * p + l2, e3 * p + l3);
                double a = g->Lv[g1][l1], b = g->Lv[g2][l2], c = g->Lv[g3][l3];
                P->phi[t] = a * b * c;
                P->dphi[t][0] = g->Ld[g1][l1] * 2.0 / g->h[0] * b * c;
                P->dphi[t][1] = a * g->Ld[g2][l2] * 2.0 / g->h[1] * c;
                P->dphi[t][2] = a * b * g->Ld[g3][l3] * 2.0 / g->h[2];
            }
    P->nl = t;
}

/* face point basis: face f, micro-face (e1,e2), Gauss point (g1,g2) */
typedef struct {
    double w;                  /* face weight                              */
    int A[25];                 /* macro node of each local face node       */
    int c[25];                 /* face node index c1 + n c2                */
    double mu[25];
    int nl;
    double nrm[3];
} fpt_t;

static void face_basis(const geo_t *g, int f, int e1, int e2, int g1, int g2, fpt_t *P)
{
    int p = g->p, d = f / 2, t1, t2;
    face_dirs(d, &t1, &t2);
    P->w = g->om[g1] * g->h[t1] / 2 * g->om[g2] * g->h[t2] / 2;
    int t = 0;
    for (int l2 = 0; l2 <= p; ++l2)
        for (int l1 = 0; l1 <= p; ++l1, ++t) {
            int c1 = e1 * p + l1, c2 = e2 * p + l2;
            P->A[t] = face_node(g, f, c1, c2);
            P->c[t] = c1 + g->n * c2;
            P->mu[t] = g->Lv[g1][l1] * g->Lv[g2][l2];
        }
    P->nl = t;
    P->nrm[0] = P->nrm[1] = P->nrm[2] = 0;
    P->nrm[d] = (f % 2) ? 1.0 : -1.0;
}

/* evaluate nodal fields at a volume point */
static void vol_values(const geo_t *g, const vpt_t *P, const double *v, const double *vs,
                       const double *q, double *vx, double *vsx, double *qx)
{
    int Nn = g->Nn;
    for (int k = 0; k < 5; ++k) { vx[k] = 0; vsx[k] = 0; }
    for (int i = 0; i < 15; ++i) qx[i] = 0;
    for (int t = 0; t < P->nl; ++t) {
        int A = P->A[t]; double ph = P->phi[t];
        for (int k = 0; k < 5; ++k) {
            vx[k] += ph * v[k * Nn + A];
            if (vs) vsx[k] += ph * vs[k * Nn + A];
        }
        if (q) for (int i = 0; i < 15; ++i) qx[i] += ph * q[i * Nn + A];
    }
}

static void face_values(const geo_t *g, int f, const fpt_t *P, const double *v, const double *vh,
                        const double *q, double *vx, double *vhx, double *qx)
{
    int Nn = g->Nn, n2 = g->n2;
    for (int k = 0; k < 5; ++k) { vx[k] = 0; vhx[k] = 0; }
    for (int i = 0; i < 15; ++i) qx[i] = 0;
    for (int t = 0; t < P->nl; ++t) {
        int A = P->A[t], c = P->c[t]; double mu = P->mu[t];
        for (int k = 0; k < 5; ++k) {
            vx[k] += mu * v[k * Nn + A];
            vhx[k] += mu * vh[(f * 5 + k) * n2 + c];
        }
        if (q) for (int i = 0; i < 15; ++i) qx[i] += mu * q[i * Nn + A];
    }
}

/* Residual of one macro-element:
 *  RV[k][A]   = sum_vol W [U_k phi_A - sum_j FG_kj d_j phi_A] + sum_faces w Fh_k mu_A
 *  RQ[k][d][A]= sum_vol W [q_kd phi_A + v_k d_d phi_A] - sum_faces w vh_k n_d mu_A
 *  RH[f][k][c]= sum_{face f} w Fh_k mu_c      (this element's side only)
 * vh: local trace [6][5][n^2].  q may be NULL for the Euler equations.      */
int orc_residual(const orc_params *pr, int p, int m, const double *box,
                 const double *v, const double *vs, const double *vh, const double *q,
                 double *RV, double *RQ, double *RH)
{
    geo_t g;
    if (geo_init(&g, p, m, box)) return -1;
    int Nn = g.Nn, n2 = g.n2, ng = g.ng;
    memset(RV, 0, sizeof(double) * 5 * Nn);
    if (RQ) memset(RQ, 0, sizeof(double) * 15 * Nn);
    memset(RH, 0, sizeof(double) * 30 * n2);
    vpt_t P;
    for (int e3 = 0; e3 < m; ++e3) for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g3 = 0; g3 < ng; ++g3) for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        vol_basis(&g, e1, e2, e3, g1, g2, g3, &P);
        double vx[5], vsx[5], qx[15];
        vol_values(&g, &P, v, vs, q, vx, vsx, qx);
        cplx cv[5], cvs[5], cq[15], U[5], FG[15];
        to_c(vx, cv, 5); to_c(vsx, cvs, 5); to_c(qx, cq, 15);
        vol_point(pr, cv, cvs, cq, U, FG);
        for (int t = 0; t < P.nl; ++t) {
            int A = P.A[t];
            for (int k = 0; k < 5; ++k) {
                double s = creal(U[k]) * P.phi[t];
                for (int j = 0; j < 3; ++j) s -= creal(FG[k * 3 + j]) * P.dphi[t][j];
                RV[k * Nn + A] += P.W * s;
                if (RQ) for (int d = 0; d < 3; ++d)
                    RQ[(k * 3 + d) * Nn + A] += P.W * (qx[k * 3 + d] * P.phi[t] + vx[k] * P.dphi[t][d]);
            }
        }
    }
    fpt_t F;
    for (int f = 0; f < 6; ++f)
    for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        face_basis(&g, f, e1, e2, g1, g2, &F);
        double vx[5], vhx[5], qx[15];
        face_values(&g, f, &F, v, vh, q, vx, vhx, qx);
        cplx cv[5], cvh[5], cq[15], Fh[5];
        to_c(vx, cv, 5); to_c(vhx, cvh, 5); to_c(qx, cq, 15);
        face_point(pr, cvh, cv, cq, F.nrm, Fh);
        int d = f / 2;
        for (int t = 0; t < F.nl; ++t) {
            int A = F.A[t], c = F.c[t];
            for (int k = 0; k < 5; ++k) {
                double val = F.w * creal(Fh[k]) * F.mu[t];
                RV[k * Nn + A] += val;
                RH[(f * 5 + k) * n2 + c] += val;
                if (RQ) RQ[(k * 3 + d) * Nn + A] -= F.w * vhx[k] * F.nrm[d] * F.mu[t];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Quadrature entropy defect, for the discrete entropy identity         */
/*  D_Q = (F(v_h), grad v_h)_Q - <Psi_n(v_h)>_{dK,Q},  Psi = rho V (eq. poen) */
/* ------------------------------------------------------------------ */
double orc_entropy_defect(const orc_params *pr, int p, int m, const double *box, const double *v)
{
    geo_t g;
    if (geo_init(&g, p, m, box)) return NAN;
    int Nn = g.Nn, ng = g.ng;
    double D = 0.0;
    vpt_t P;
    for (int e3 = 0; e3 < m; ++e3) for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g3 = 0; g3 < ng; ++g3) for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        vol_basis(&g, e1, e2, e3, g1, g2, g3, &P);
        double vx[5] = {0}, gv[5][3] = {{0}};
        for (int t = 0; t < P.nl; ++t)
            for (int k = 0; k < 5; ++k) {
                double a = v[k * Nn + P.A[t]];
                vx[k] += P.phi[t] * a;
                for (int j = 0; j < 3; ++j) gv[k][j] += P.dphi[t][j] * a;
            }
        cplx cv[5]; prim_t w; to_c(vx, cv, 5); prim_from_v(cv, pr->gamma, &w);
        for (int j = 0; j < 3; ++j) {
            cplx Fj[5]; flux_col(&w, j, Fj);
            for (int k = 0; k < 5; ++k) D += P.W * creal(Fj[k]) * gv[k][j];
        }
    }
    fpt_t F;
    for (int f = 0; f < 6; ++f)
    for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        face_basis(&g, f, e1, e2, g1, g2, &F);
        double vx[5] = {0};
        for (int t = 0; t < F.nl; ++t)
            for (int k = 0; k < 5; ++k) vx[k] += F.mu[t] * v[k * Nn + F.A[t]];
        cplx cv[5]; prim_t w; to_c(vx, cv, 5); prim_from_v(cv, pr->gamma, &w);
        cplx psin = w.rho * (w.V[0] * F.nrm[0] + w.V[1] * F.nrm[1] + w.V[2] * F.nrm[2]);
        D -= F.w * creal(psin);
    }
    return D;
}

/* ------------------------------------------------------------------ */
/* Local Jacobian blocks (eq. R1), by complex step on the point-wise     */
/* integrands and exact linear assembly with the basis.                 */
/* Index maps: V (k,A) -> k Nn + A; Q (k,d,A) -> (3k+d) Nn + A;           */
/* trace (f,k,c) -> (5f+k) n^2 + c.  Every output pointer may be NULL.   */
/* ------------------------------------------------------------------ */
typedef struct {
    double *Avv, *Avh, *Ahv, *Ahh, *Avq, *Ahq, *Aqq, *Aqv, *Aqh;
} orc_blocks;

int orc_jacobian(const orc_params *pr, int p, int m, const double *box,
                 const double *v, const double *vs, const double *vh, const double *q,
                 double *Avv, double *Avh, double *Ahv, double *Ahh,
                 double *Avq, double *Ahq, double *Aqq, double *Aqv, double *Aqh)
{
    geo_t g;
    if (geo_init(&g, p, m, box)) return -1;
    int Nn = g.Nn, n2 = g.n2, ng = g.ng;
    long Nv = 5L * Nn, Nq = 15L * Nn, Nt = 30L * n2;
    const double hcs = 1e-30;
    if (Avv) memset(Avv, 0, sizeof(double) * Nv * Nv);
    if (Avh) memset(Avh, 0, sizeof(double) * Nv * Nt);
    if (Ahv) memset(Ahv, 0, sizeof(double) * Nt * Nv);
    if (Ahh) memset(Ahh, 0, sizeof(double) * Nt * Nt);
    if (Avq) memset(Avq, 0, sizeof(double) * Nv * Nq);
    if (Ahq) memset(Ahq, 0, sizeof(double) * Nt * Nq);
    if (Aqq) memset(Aqq, 0, sizeof(double) * Nq * Nq);
    if (Aqv) memset(Aqv, 0, sizeof(double) * Nq * Nv);
    if (Aqh) memset(Aqh, 0, sizeof(double) * Nq * Nt);
    vpt_t P;
    for (int e3 = 0; e3 < m; ++e3) for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g3 = 0; g3 < ng; ++g3) for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        vol_basis(&g, e1, e2, e3, g1, g2, g3, &P);
        double vx[5], vsx[5], qx[15];
        vol_values(&g, &P, v, vs, q, vx, vsx, qx);
        double dU[5][5], dFG[15][5], dFGq[15][15];
        for (int l = 0; l < 5; ++l) {
            cplx cv[5], cvs[5], cq[15], U[5], FG[15];
            to_c(vx, cv, 5); to_c(vsx, cvs, 5); to_c(qx, cq, 15);
            cv[l] += I * hcs;
            vol_point(pr, cv, cvs, cq, U, FG);
            for (int k = 0; k < 5; ++k) dU[k][l] = cimag(U[k]) / hcs;
            for (int i = 0; i < 15; ++i) dFG[i][l] = cimag(FG[i]) / hcs;
        }
        if (pr->viscous) for (int l = 0; l < 15; ++l) {
            cplx cv[5], cvs[5], cq[15], U[5], FG[15];
            to_c(vx, cv, 5); to_c(vsx, cvs, 5); to_c(qx, cq, 15);
            cq[l] += I * hcs;
            vol_point(pr, cv, cvs, cq, U, FG);
            for (int i = 0; i < 15; ++i) dFGq[i][l] = cimag(FG[i]) / hcs;
        }
        for (int ta = 0; ta < P.nl; ++ta) {
            int A = P.A[ta];
            for (int tb = 0; tb < P.nl; ++tb) {
                int B = P.A[tb];
                double pp = P.W * P.phi[ta] * P.phi[tb];
                double gp[3];
                for (int j = 0; j < 3; ++j) gp[j] = P.W * P.dphi[ta][j] * P.phi[tb];
                for (int k = 0; k < 5; ++k) {
                    if (Avv) for (int l = 0; l < 5; ++l) {
                        double s = pp * dU[k][l];
                        for (int j = 0; j < 3; ++j) s -= gp[j] * dFG[k * 3 + j][l];
                        Avv[(k * Nn + A) * Nv + l * Nn + B] += s;
                    }
                    if (Avq && pr->viscous) for (int l = 0; l < 15; ++l) {
                        double s = 0;
                        for (int j = 0; j < 3; ++j) s -= gp[j] * dFGq[k * 3 + j][l];
                        Avq[(k * Nn + A) * Nq + (long)l * Nn + B] += s;
                    }
                    for (int d = 0; d < 3; ++d) {
                        long row = (long)(k * 3 + d) * Nn + A;
                        if (Aqq) Aqq[row * Nq + row - A + B] += pp;
                        if (Aqv) Aqv[row * Nv + k * Nn + B] += gp[d];
                    }
                }
            }
        }
    }
    fpt_t F;
    for (int f = 0; f < 6; ++f)
    for (int e2 = 0; e2 < m; ++e2) for (int e1 = 0; e1 < m; ++e1)
    for (int g2 = 0; g2 < ng; ++g2) for (int g1 = 0; g1 < ng; ++g1) {
        face_basis(&g, f, e1, e2, g1, g2, &F);
        double vx[5], vhx[5], qx[15];
        face_values(&g, f, &F, v, vh, q, vx, vhx, qx);
        double dH[5][5], dV[5][5], dQ[5][15];
        for (int l = 0; l < 5; ++l) {
            cplx cv[5], cvh[5], cq[15], Fh[5];
            to_c(vx, cv, 5); to_c(vhx, cvh, 5); to_c(qx, cq, 15);
            cvh[l] += I * hcs;
            face_point(pr, cvh, cv, cq, F.nrm, Fh);
            for (int k = 0; k < 5; ++k) dH[k][l] = cimag(Fh[k]) / hcs;
            to_c(vhx, cvh, 5); cv[l] += I * hcs;
            face_point(pr, cvh, cv, cq, F.nrm, Fh);
            for (int k = 0; k < 5; ++k) dV[k][l] = cimag(Fh[k]) / hcs;
        }
        if (pr->viscous) for (int l = 0; l < 15; ++l) {
            cplx cv[5], cvh[5], cq[15], Fh[5];
            to_c(vx, cv, 5); to_c(vhx, cvh, 5); to_c(qx, cq, 15);
            cq[l] += I * hcs;
            face_point(pr, cvh, cv, cq, F.nrm, Fh);
            for (int k = 0; k < 5; ++k) dQ[k][l] = cimag(Fh[k]) / hcs;
        }
        int d = f / 2;
        for (int ta = 0; ta < F.nl; ++ta) {
            int A = F.A[ta], ca = F.c[ta];
            for (int tb = 0; tb < F.nl; ++tb) {
                int B = F.A[tb], cb = F.c[tb];
                double mm = F.w * F.mu[ta] * F.mu[tb];
                for (int k = 0; k < 5; ++k) {
                    long rv = (long)k * Nn + A, rh = (long)(f * 5 + k) * n2 + ca;
                    for (int l = 0; l < 5; ++l) {
                        long cvv = (long)l * Nn + B, chh = (long)(f * 5 + l) * n2 + cb;
                        if (Avv) Avv[rv * Nv + cvv] += mm * dV[k][l];
                        if (Avh) Avh[rv * Nt + chh] += mm * dH[k][l];
                        if (Ahv) Ahv[rh * Nv + cvv] += mm * dV[k][l];
                        if (Ahh) Ahh[rh * Nt + chh] += mm * dH[k][l];
                    }
                    if (pr->viscous) for (int l = 0; l < 15; ++l) {
                        long cq = (long)l * Nn + B;
                        if (Avq) Avq[rv * Nq + cq] += mm * dQ[k][l];
                        if (Ahq) Ahq[rh * Nq + cq] += mm * dQ[k][l];
                    }
                    if (Aqh) Aqh[((long)(k * 3 + d) * Nn + A) * Nt + (long)(f * 5 + k) * n2 + cb]
                                -= mm * F.nrm[d];
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dense LU with partial pivoting (largest |.|, ties -> lowest index)    */
/* row-major, in place; piv[k] = row swapped with row k at step k.       */
/* ------------------------------------------------------------------ */
int orc_getrf(int N, double *A, int *piv)
{
    for (int k = 0; k < N; ++k) {
        int r = k; double best = fabs(A[(long)k * N + k]);
        for (int i = k + 1; i < N; ++i) {
            double a = fabs(A[(long)i * N + k]);
            if (a > best) { best = a; r = i; }
        }
        piv[k] = r;
        if (best == 0.0) return k + 1;
        if (r != k) {
            double *x = A + (long)k * N, *y = A + (long)r * N;
            for (int j = 0; j < N; ++j) { double t = x[j]; x[j] = y[j]; y[j] = t; }
        }
        double inv = 1.0 / A[(long)k * N + k];
        const double *rk = A + (long)k * N;
        for (int i = k + 1; i < N; ++i) {
            double *ri = A + (long)i * N;
            double l = ri[k] * inv;
            ri[k] = l;
            if (l != 0.0) for (int j = k + 1; j < N; ++j) ri[j] -= l * rk[j];
        }
    }
    return 0;
}

/* solve with the factors for nrhs right-hand sides B[N][nrhs] (row-major) */
void orc_getrs(int N, const double *LU, const int *piv, int nrhs, double *B)
{
    for (int k = 0; k < N; ++k) {
        if (piv[k] != k) {
            double *x = B + (long)k * nrhs, *y = B + (long)piv[k] * nrhs;
            for (int j = 0; j < nrhs; ++j) { double t = x[j]; x[j] = y[j]; y[j] = t; }
        }
    }
    for (int i = 0; i < N; ++i) {
        double *bi = B + (long)i * nrhs;
        for (int k = 0; k < i; ++k) {
            double l = LU[(long)i * N + k];
            if (l != 0.0) { const double *bk = B + (long)k * nrhs; for (int j = 0; j < nrhs; ++j) bi[j] -= l * bk[j]; }
        }
    }
    for (int i = N - 1; i >= 0; --i) {
        double *bi = B + (long)i * nrhs;
        for (int k = i + 1; k < N; ++k) {
            double u = LU[(long)i * N + k];
            if (u != 0.0) { const double *bk = B + (long)k * nrhs; for (int j = 0; j < nrhs; ++j) bi[j] -= u * bk[j]; }
        }
        double inv = 1.0 / LU[(long)i * N + i];
        for (int j = 0; j < nrhs; ++j) bi[j] *= inv;
    }
}

/* C[M][N] += alpha A[M][K] B[K][N] (plain triple loop, row-major) */
static void gemm_acc(long M, long N, long K, double alpha, const double *A, const double *B, double *C)
{
    for (long i = 0; i < M; ++i)
        for (long k = 0; k < K; ++k) {
            double a = alpha * A[i * K + k];
            if (a == 0.0) continue;
            const double *bk = B + k * N; double *ci = C + i * N;
            for (long j = 0; j < N; ++j) ci[j] += a * bk[j];
        }
}

/* ------------------------------------------------------------------ */
/* Static condensation of one macro-element (eqs. R1-R6), literal.     */
/* Inputs are the residuals and blocks of this element; A_qq^{-1} is    */
/* applied through a dense LU of A_qq.                                   */
/* Outputs: bhat[Nt] (eq. R5b); Ahat[Nt*Nt] (eq. R5a, may be NULL);       */
/* if dvh != NULL also the recovery dV[Nv] (eq. R2), dQ[Nq] (eq. R6).    */
/* ------------------------------------------------------------------ */
int orc_condense_blocks(int viscous, long Nv, long Nq, long Nt,
                        const double *RV, const double *RQ, const double *RH,
                        const double *Avv, const double *Avh, const double *Ahv, const double *Ahh,
                        const double *Avq, const double *Ahq, const double *Aqq, const double *Aqv,
                        const double *Aqh,
                        double *bhat, double *Ahat, const double *dvh, double *dV, double *dQ)
{
    /* S, Avh' = Avh - Avq Aqq^-1 Aqh, Ahv' = Ahv - Ahq Aqq^-1 Aqv,
     * Ahh' = Ahh - Ahq Aqq^-1 Aqh, rV = -RV + Avq Aqq^-1 RQ,
     * rH = -RH + Ahq Aqq^-1 RQ                                              */
    double *S = malloc(sizeof(double) * Nv * Nv);
    double *Avh2 = malloc(sizeof(double) * Nv * Nt);
    double *Ahv2 = malloc(sizeof(double) * Nt * Nv);
    double *Ahh2 = malloc(sizeof(double) * Nt * Nt);
    double *rV = malloc(sizeof(double) * Nv);
    double *rH = malloc(sizeof(double) * Nt);
    int *piv = malloc(sizeof(int) * Nv);
    if (!S || !Avh2 || !Ahv2 || !Ahh2 || !rV || !rH || !piv) return -2;
    memcpy(S, Avv, sizeof(double) * Nv * Nv);
    memcpy(Avh2, Avh, sizeof(double) * Nv * Nt);
    memcpy(Ahv2, Ahv, sizeof(double) * Nt * Nv);
    memcpy(Ahh2, Ahh, sizeof(double) * Nt * Nt);
    for (long i = 0; i < Nv; ++i) rV[i] = -RV[i];
    for (long i = 0; i < Nt; ++i) rH[i] = -RH[i];
    double *X = NULL, *Y = NULL, *z = NULL, *LUq = NULL; int *pq = NULL;
    if (viscous) {
        /* Aqq^{-1} [Aqv | Aqh | RQ] */
        long nc = Nv + Nt + 1;
        LUq = malloc(sizeof(double) * Nq * Nq);
        pq = malloc(sizeof(int) * Nq);
        X = malloc(sizeof(double) * Nq * nc);
        if (!LUq || !pq || !X) return -2;
        memcpy(LUq, Aqq, sizeof(double) * Nq * Nq);
        if (orc_getrf((int)Nq, LUq, pq)) return -3;
        for (long i = 0; i < Nq; ++i) {
            for (long j = 0; j < Nv; ++j) X[i * nc + j] = Aqv[i * Nv + j];
            for (long j = 0; j < Nt; ++j) X[i * nc + Nv + j] = Aqh[i * Nt + j];
            X[i * nc + Nv + Nt] = RQ[i];
        }
        orc_getrs((int)Nq, LUq, pq, (int)nc, X);
        /* split into C = Aqq^-1 Aqv, Ct = Aqq^-1 Aqh, z = Aqq^-1 RQ */
        double *C = malloc(sizeof(double) * Nq * Nv), *Ct = malloc(sizeof(double) * Nq * Nt);
        z = malloc(sizeof(double) * Nq);
        for (long i = 0; i < Nq; ++i) {
            for (long j = 0; j < Nv; ++j) C[i * Nv + j] = X[i * nc + j];
            for (long j = 0; j < Nt; ++j) Ct[i * Nt + j] = X[i * nc + Nv + j];
            z[i] = X[i * nc + Nv + Nt];
        }
        gemm_acc(Nv, Nv, Nq, -1.0, Avq, C, S);
        gemm_acc(Nv, Nt, Nq, -1.0, Avq, Ct, Avh2);
        gemm_acc(Nt, Nv, Nq, -1.0, Ahq, C, Ahv2);
        gemm_acc(Nt, Nt, Nq, -1.0, Ahq, Ct, Ahh2);
        gemm_acc(Nv, 1, Nq, 1.0, Avq, z, rV);
        gemm_acc(Nt, 1, Nq, 1.0, Ahq, z, rH);
        free(C); Y = Ct;   /* keep Ct for the recovery */
    }
    if (orc_getrf((int)Nv, S, piv)) return -3;
    /* b-hat = rH - Ahv' S^-1 rV  (eq. R5b: -RH + AhqAqq^-1RQ + (-Ahv')S^-1(-RV+...)) */
    double *y = malloc(sizeof(double) * Nv);
    memcpy(y, rV, sizeof(double) * Nv);
    orc_getrs((int)Nv, S, piv, 1, y);
    for (long i = 0; i < Nt; ++i) {
        double s = rH[i];
        for (long j = 0; j < Nv; ++j) s -= Ahv2[i * Nv + j] * y[j];
        bhat[i] = s;
    }
    if (Ahat) {
        /* Ahat = Ahh' + Ahv' S^-1 (-Avh')  (eq. R5a) */
        double *W = malloc(sizeof(double) * Nv * Nt);
        for (long i = 0; i < Nv * Nt; ++i) W[i] = -Avh2[i];
        orc_getrs((int)Nv, S, piv, (int)Nt, W);
        memcpy(Ahat, Ahh2, sizeof(double) * Nt * Nt);
        gemm_acc(Nt, Nt, Nv, 1.0, Ahv2, W, Ahat);
        free(W);
    }
    if (dvh) {
        /* eq. R2: S dV = rV - Avh' dvh ;  eq. R6: dQ = Aqq^-1(-RQ - Aqv dV - Aqh dvh) */
        for (long i = 0; i < Nv; ++i) {
            double s = rV[i];
            for (long j = 0; j < Nt; ++j) s -= Avh2[i * Nt + j] * dvh[j];
            dV[i] = s;
        }
        orc_getrs((int)Nv, S, piv, 1, dV);
        if (viscous && dQ) {
            /* dQ = -z - C dV - Ct dvh, with C = Aqq^-1 Aqv recomputed from X */
            long nc = Nv + Nt + 1;
            for (long i = 0; i < Nq; ++i) {
                double s = -z[i];
                for (long j = 0; j < Nv; ++j) s -= X[i * nc + j] * dV[j];
                for (long j = 0; j < Nt; ++j) s -= Y[i * Nt + j] * dvh[j];
                dQ[i] = s;
            }
        }
    }
    free(S); free(Avh2); free(Ahv2); free(Ahh2); free(rV); free(rH); free(piv); free(y);
    free(X); free(Y); free(z); free(LUq); free(pq);
    return 0;
}

/* y = A x (row-major M x N) -- used by the tests for residual checks */
void orc_matvec(long M, long N, const double *A, const double *x, double *y)
{
    for (long i = 0; i < M; ++i) {
        double s = 0; const double *a = A + i * N;
        for (long j = 0; j < N; ++j) s += a[j] * x[j];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Degree-of-freedom counting (Tables Inv_TGV_DOF and TGV_DOF):          */
/* tetrahedral macro-elements made of m^3 congruent tetrahedra (m=2: 8),  */
/* P_p on each; the macro-element's C0 space is the P_{mp} lattice of the */
/* refined tetrahedron; local unknowns v (5) and q (15) per node; global   */
/* unknowns: 5 per node of the P_{mp} face lattice, each face shared by 2. */
/* n_tet counts the tetrahedra of the whole mesh.                        */
/* ------------------------------------------------------------------ */
void orc_dof_counts_tet(int p, int m, long n_tet, long *dof_local, long *dof_global)
{
    long q = (long)m * p;
    long nodes_vol = (q + 1) * (q + 2) * (q + 3) / 6;
    long nodes_face = (q + 1) * (q + 2) / 2;
    long n_macro = n_tet / ((long)m * m * m);
    *dof_local = n_macro * nodes_vol * 20;
    *dof_global = n_macro * 4 / 2 * nodes_face * 5;
}

/* hexahedral analogue: hex micro-elements, the six faces of K independent */
void orc_dof_counts_hex(int p, int m, long n_macro, int viscous, long *dof_local, long *dof_global)
{
    long n = (long)m * p + 1;
    *dof_local = n_macro * n * n * n * (viscous ? 20 : 5);
    *dof_global = n_macro * 3 * n * n * 5;
}
