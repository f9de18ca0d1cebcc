// physics.cuh -- point-wise physics of the entropy-variable formulation,
// templated on the scalar (double, or a forward-mode dual for tangents and
// Jacobians).  Faces are axis-aligned: the outward normal is s e_d.
#pragma once
#include "common.cuh"

template <class T>
struct Prim {
    T rho, V[3], P, beta, rE;
};

// Inverse of eq. s222: beta = -v5, V = v_{2..4}/beta,
// s = gamma - (gamma-1)(v1 + beta |V|^2 / 2), rho = (beta e^s)^{1/(1-gamma)},
// P = rho/beta, rho E = P/(gamma-1) + rho |V|^2/2.
template <class T>
__device__ __forceinline__ bool entropy_to_prim(const T* v, double g, Prim<T>& w) {
    w.beta = -v[4];
    T ib = 1.0 / w.beta;
    w.V[0] = v[1] * ib; w.V[1] = v[2] * ib; w.V[2] = v[3] * ib;
    T V2 = w.V[0] * w.V[0] + w.V[1] * w.V[1] + w.V[2] * w.V[2];
    T s = g - (g - 1.0) * (v[0] + 0.5 * (w.beta * V2));
    w.rho = dexp((dlog(w.beta) + s) * (1.0 / (1.0 - g)));
    w.P = w.rho * ib;
    w.rE = w.P * (1.0 / (g - 1.0)) + 0.5 * (w.rho * V2);
    double b = val(w.beta), r = val(w.rho);
    return b > 0.0 && r > 0.0 && isfinite(r) && isfinite(b);
}

// inviscid flux in direction j (eq. C5)
template <class T>
__device__ __forceinline__ void euler_flux(const Prim<T>& w, int j, T* F) {
    T m = w.rho * w.V[j];
    F[0] = m;
    F[1] = m * w.V[0]; F[2] = m * w.V[1]; F[3] = m * w.V[2];
    F[1 + j] = F[1 + j] + w.P;
    F[4] = w.V[j] * (w.rE + w.P);
}

// A0 x, A0 = du/dv in closed form (symmetric positive definite)
template <class T>
__device__ __forceinline__ void A0_times(const Prim<T>& w, double g, const T* x, T* y) {
    T Et = w.rE, EP = w.rE + w.P;
    T H = EP / w.rho;
    T a2 = g * w.P / w.rho;
    T Vx = w.V[0] * x[1] + w.V[1] * x[2] + w.V[2] * x[3];
    y[0] = w.rho * x[0] + w.rho * Vx + Et * x[4];
    for (int i = 0; i < 3; ++i)
        y[1 + i] = w.rho * w.V[i] * x[0] + w.rho * w.V[i] * Vx + w.P * x[1 + i] + EP * w.V[i] * x[4];
    y[4] = Et * x[0] + EP * Vx + (w.rho * H * H - a2 * w.P * (1.0 / (g - 1.0))) * x[4];
}

// Ismail-Roe logarithmic mean (eq. avg): zeta = b/a, f = (zeta-1)/(zeta+1),
// u = f^2; F = 1 + u/3 + u^2/5 + u^3/7 if u < 1e-4 else ln(zeta)/(2 f);
// mean = (a + b) / (2 F).
template <class T>
__device__ __forceinline__ T log_mean(const T& a, const T& b) {
    T zeta = b / a;
    T f = (zeta - 1.0) / (zeta + 1.0);
    T u = f * f;
    T F;
    if (val(u) < 1e-4) F = 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0)));
    else F = dlog(zeta) / (2.0 * f);
    return (a + b) / (2.0 * F);
}

// Numerical inviscid flux F-hat(vh, v; n), n = s e_d (eqs. Flux_En_Inv, EC, ES).
template <class T>
__device__ __forceinline__ void num_flux(int kind, const Prim<T>& a /*interior*/, const Prim<T>& b /*hat*/,
                                         const T* v, const T* vh, int d, double s, double g, T* out) {
    if (kind == MEHDG_FLUX_ES) {
        // 1/2 (F(vh) + F(v)).n - 1/2 sigma(vh) A0(vh) [[v]], sigma = |Vh.n| + c_h
        T Fa[5], Fb[5], dv[5], A0dv[5];
        euler_flux(a, d, Fa); euler_flux(b, d, Fb);
        for (int k = 0; k < 5; ++k) dv[k] = vh[k] - v[k];
        A0_times(b, g, dv, A0dv);
        T sig = dabs(b.V[d]) + dsqrt(g * b.P / b.rho);
        for (int k = 0; k < 5; ++k) out[k] = 0.5 * s * (Fa[k] + Fb[k]) - 0.5 * (sig * A0dv[k]);
        return;
    }
    // averages of eq. avg / eq. EC
    T rln = log_mean(a.rho, b.rho);
    T bln = log_mean(a.beta, b.beta);
    T Vb[3];
    for (int i = 0; i < 3; ++i) Vb[i] = 0.5 * (a.V[i] + b.V[i]);
    T Pb = (a.rho + b.rho) / (a.beta + b.beta);          // rho-bar / beta-bar
    T VV = 0.5 * (a.V[0] * a.V[0] + a.V[1] * a.V[1] + a.V[2] * a.V[2] +
                  b.V[0] * b.V[0] + b.V[1] * b.V[1] + b.V[2] * b.V[2]);
    T vn = s * Vb[d];
    T f1 = rln * vn;
    T f2[3];
    for (int i = 0; i < 3; ++i) f2[i] = Vb[i] * f1;
    f2[d] = f2[d] + s * Pb;
    T f3 = (1.0 / (bln * (g - 1.0)) - 0.5 * VV) * f1 + Vb[0] * f2[0] + Vb[1] * f2[1] + Vb[2] * f2[2];
    out[0] = f1; out[1] = f2[0]; out[2] = f2[1]; out[3] = f2[2]; out[4] = f3;
    if (kind != MEHDG_FLUX_KEPES) return;
    // KEPES dissipation R |Lambda| T R^T [[v]] (eqs. KEPES3-KEPES5): averaged
    // eigenvectors rotated to n; tangents t1, t2 = the other two axes.
    int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    T c = dsqrt(g * Pb / rln);
    T hb = g / (bln * (g - 1.0)) + 0.5 * VV;
    T dv[5];
    for (int k = 0; k < 5; ++k) dv[k] = vh[k] - v[k];
    T Vdv = Vb[0] * dv[1] + Vb[1] * dv[2] + Vb[2] * dv[3];
    T cn = c * s;                                       // c n_d
    T w1 = dv[0] + Vdv - cn * dv[1 + d] + (hb - c * vn) * dv[4];
    T w2 = dv[0] + Vdv + 0.5 * VV * dv[4];
    T w3 = dv[1 + t1] + Vb[t1] * dv[4];
    T w4 = dv[1 + t2] + Vb[t2] * dv[4];
    T w5 = dv[0] + Vdv + cn * dv[1 + d] + (hb + c * vn) * dv[4];
    // |Lambda| = (1-theta)|lambda| + theta lambda_max, |lambda_1,5| = |vn| + c
    T avn = dabs(vn);
    T lmax = avn + c;
    T x = (a.P - b.P) / (a.P + b.P);
    T theta = (val(x) == 0.0) ? cst<T>(0.0) : dsqrt(dabs(x));
    T lmid = avn + theta * c;                            // (1-theta)|vn| + theta (|vn|+c)
    T T15 = rln * (1.0 / (2.0 * g));
    T T2 = rln * ((g - 1.0) / g);
    T z1 = w1 * lmax * T15, z5 = w5 * lmax * T15;
    T z2 = w2 * lmid * T2, z3 = w3 * lmid * Pb, z4 = w4 * lmid * Pb;
    T dis[5];
    dis[0] = z1 + z2 + z5;
    for (int i = 0; i < 3; ++i) dis[1 + i] = (z1 + z2 + z5) * Vb[i];
    dis[1 + d] = dis[1 + d] + (z5 - z1) * cn;
    dis[1 + t1] = dis[1 + t1] + z3;
    dis[1 + t2] = dis[1 + t2] + z4;
    dis[4] = (z1 + z5) * hb + (z5 - z1) * (c * vn) + z2 * (0.5 * VV) + z3 * Vb[t1] + z4 * Vb[t2];
    for (int k = 0; k < 5; ++k) out[k] = out[k] - 0.5 * dis[k];
}

// Viscous flux column j, G = -[0, tau, tau V - phi] (eqs. C5, C6), from
// q = grad v: V_i = -v_{i+1}/v5, T = -gamma/v5, grad by the chain rule.
template <class T>
__device__ __forceinline__ void visc_flux(const T* v, const T* q /*[5][3]*/, const Phys& ph, T G[5][3]) {
    T i5 = 1.0 / v[4];
    T i55 = i5 * i5;
    T V[3], dV[3][3], dT[3];
    for (int i = 0; i < 3; ++i) V[i] = -(v[1 + i] * i5);
    for (int i = 0; i < 3; ++i)
        for (int dd = 0; dd < 3; ++dd) dV[i][dd] = -(q[(1 + i) * 3 + dd] * i5) + v[1 + i] * q[12 + dd] * i55;
    for (int dd = 0; dd < 3; ++dd) dT[dd] = ph.gamma * (q[12 + dd] * i55);
    T div = dV[0][0] + dV[1][1] + dV[2][2];
    for (int j = 0; j < 3; ++j) {
        T tcol[3];
        for (int i = 0; i < 3; ++i) tcol[i] = ph.mu * (dV[i][j] + dV[j][i]);
        tcol[j] = tcol[j] - ph.mu * (2.0 / 3.0) * div;
        G[0][j] = cst<T>(0.0);
        for (int i = 0; i < 3; ++i) G[1 + i][j] = -tcol[i];
        // (tau V)_j - phi_j, phi = -kappa grad T
        G[4][j] = -(tcol[0] * V[0] + tcol[1] * V[1] + tcol[2] * V[2] + ph.kappa * dT[j]);
    }
}

// face integrand F-hat + G-hat (eq. Flux_En_Vis for the viscous part)
template <class T>
__device__ __forceinline__ bool face_integrand(const Phys& ph, const T* v, const T* vh, const T* q,
                                               int d, double s, T* out) {
    Prim<T> a, b;
    bool ok = entropy_to_prim(v, ph.gamma, a);
    ok = entropy_to_prim(vh, ph.gamma, b) && ok;
    num_flux(ph.flux, a, b, v, vh, d, s, ph.gamma, out);
    if (ph.viscous) {
        T G[5][3];
        visc_flux(vh, q, ph, G);
        for (int k = 0; k < 5; ++k) out[k] = out[k] + s * G[k][d];
        for (int k = 1; k < 4; ++k) out[k] = out[k] - 0.5 * ph.sv_mom * (vh[k] - v[k]);
        out[4] = out[4] - 0.5 * ph.sv_en * (vh[4] - v[4]);
    }
    return ok;
}

// volume integrand: U = (u(v) - u(v*))/dt and FG = F + G
template <class T>
__device__ __forceinline__ bool vol_integrand(const Phys& ph, const T* v, const T* vs, const T* q,
                                              T* U, T FG[5][3]) {
    Prim<T> w;
    bool ok = entropy_to_prim(v, ph.gamma, w);
    if (ph.time_term) {
        Prim<T> ws;
        ok = entropy_to_prim(vs, ph.gamma, ws) && ok;
        U[0] = (w.rho - ws.rho) * ph.inv_dt;
        for (int i = 0; i < 3; ++i) U[1 + i] = (w.rho * w.V[i] - ws.rho * ws.V[i]) * ph.inv_dt;
        U[4] = (w.rE - ws.rE) * ph.inv_dt;
    } else {
        for (int k = 0; k < 5; ++k) U[k] = cst<T>(0.0);
    }
    for (int j = 0; j < 3; ++j) {
        T F[5];
        euler_flux(w, j, F);
        for (int k = 0; k < 5; ++k) FG[k][j] = F[k];
    }
    if (ph.viscous) {
        T G[5][3];
        visc_flux(v, q, ph, G);
        for (int k = 0; k < 5; ++k)
            for (int j = 0; j < 3; ++j) FG[k][j] = FG[k][j] + G[k][j];
    }
    return ok;
}
