// residual.cu -- FP64 residual of eq. s32 (with the stage term of eq. C242)
// for every macro-element, and its forward-mode tangent.
//
// Volume pass: one CTA per (micro-element, macro-element).  The CTA stages
// the local nodal state in shared memory, evaluates the state and the point
// physics at the (p+2)^3 Gauss points (one thread per point), stores the
// weighted integrands in shared memory, tests them against the local basis
// (one thread per local node and component) and adds the result into the
// element's rows of R_V / R_Q with FP64 atomics (micro-elements share nodes).
// Face pass: one CTA per (micro-face, macro-element) with the two-point
// fluxes; it adds into R_V and into the element's side of the trace residual.
// A third kernel sums the two sides of every global face (eq. s32c).
//
// With T = Dual<1> the same code returns R and dR[dv, dvh, dq], the
// directional derivative used by the refinement residual r - S x, the
// right-hand side b-hat and the reduced mat-vec (all matrix-free, FP64).
#include <algorithm>
#include <type_traits>
#include "physics.cuh"
#include "kernels.cuh"

namespace {

template <class T> __device__ __forceinline__ T load_t(const double* a, const double* da, int64_t i);
template <> __device__ __forceinline__ double load_t<double>(const double* a, const double*, int64_t i) { return a[i]; }
template <> __device__ __forceinline__ Dual<1> load_t<Dual<1>>(const double* a, const double* da, int64_t i) {
    Dual<1> r; r.v = a[i]; r.d[0] = da ? da[i] : 0.0; return r;
}
__device__ __forceinline__ double tan0(double) { return 0.0; }
__device__ __forceinline__ double tan0(const Dual<1>& x) { return x.d[0]; }

template <class T>
__device__ __forceinline__ void acc_out(double* out, double* tout, int64_t i, const T& x) {
    if (out) atomicAdd(out + i, val(x));
    if (tout) atomicAdd(tout + i, tan0(x));
}

__device__ __forceinline__ void load_tables(const Tab& tb, double* sL, double* sD, double* sW) {
    const int p1 = tb.p + 1;
    for (int i = threadIdx.x; i < tb.ng * p1; i += blockDim.x) {
        sL[i] = tb.L[i / p1][i % p1];
        sD[i] = tb.dL[i / p1][i % p1];
    }
    if (threadIdx.x < tb.ng) sW[threadIdx.x] = tb.w[threadIdx.x];
}

}  // namespace

template <class T, bool VISC>
__global__ void __launch_bounds__(128)
residual_volume_kernel(ResidualArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    if (a.skip && a.skip[K]) return;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn;
    const int nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);         // [ng][p1]
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);          // [ng][p1]
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);          // [ng]
    T* base = reinterpret_cast<T*>(sW + 8);
    T* vl = base;                 // [5][nl]
    T* vsl = vl + 5 * nl;         // [5][nl]
    T* ql = vsl + 5 * nl;         // [15][nl]
    T* pu = ql + (VISC ? 15 * nl : 0);   // [5][npt]
    T* pf = pu + 5 * npt;         // [15][npt]  (k*3+j)
    T* pq = pf + 15 * npt;        // [15][npt]
    T* pv = pq + (VISC ? 15 * npt : 0);  // [5][npt]
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    const Phys& ph = a.ph;
    const double* box = a.box + 6 * K;
    double sc[3], hw[3];
    for (int d = 0; d < 3; ++d) { double h = (box[3 + d] - box[d]) / m; sc[d] = 2.0 / h; hw[d] = 0.5 * h; }
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn;

    for (int i = tid; i < nl; i += nth) {
        int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
        int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
        for (int k = 0; k < 5; ++k) {
            vl[k * nl + i] = load_t<T>(a.v, a.dv, oV + k * Nn + A);
            if (ph.time_term) vsl[k * nl + i] = load_t<T>(a.vs, nullptr, oV + k * Nn + A);
        }
        if (VISC)
            for (int c = 0; c < 15; ++c) ql[c * nl + i] = load_t<T>(a.q, a.dq, oQ + c * Nn + A);
    }
    __syncthreads();
    bool ok = true;
    for (int x = tid; x < npt; x += nth) {
        int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
        T vx[5], vsx[5], qx[15];
        for (int k = 0; k < 5; ++k) { vx[k] = cst<T>(0.0); vsx[k] = cst<T>(0.0); }
        if (VISC) for (int c = 0; c < 15; ++c) qx[c] = cst<T>(0.0);
        for (int i = 0; i < nl; ++i) {
            int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
            double f = sL[g1 * p1 + l1] * sL[g2 * p1 + l2] * sL[g3 * p1 + l3];
            for (int k = 0; k < 5; ++k) {
                vx[k] += vl[k * nl + i] * f;
                if (ph.time_term) vsx[k] += vsl[k * nl + i] * f;
            }
            if (VISC) for (int c = 0; c < 15; ++c) qx[c] += ql[c * nl + i] * f;
        }
        T U[5], FG[5][3];
        ok = vol_integrand(ph, vx, vsx, qx, U, FG) && ok;
        double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
        for (int k = 0; k < 5; ++k) {
            pu[k * npt + x] = U[k] * W;
            for (int j = 0; j < 3; ++j) pf[(k * 3 + j) * npt + x] = FG[k][j] * W;
        }
        if (VISC) {
            for (int c = 0; c < 15; ++c) pq[c * npt + x] = qx[c] * W;
            for (int k = 0; k < 5; ++k) pv[k * npt + x] = vx[k] * W;
        }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
    const int nrow = VISC ? nl * 20 : nl * 5;
    for (int r = tid; r < nrow; r += nth) {
        int i = r % nl, kk = r / nl;          // kk < 5: R_V row; else R_Q row (k,d) = kk-5
        int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
        int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
        T s = cst<T>(0.0);
        if (kk < 5) {
            for (int x = 0; x < npt; ++x) {
                int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
                double a1 = sL[g1 * p1 + l1], a2 = sL[g2 * p1 + l2], a3 = sL[g3 * p1 + l3];
                double d1 = sD[g1 * p1 + l1] * sc[0], d2 = sD[g2 * p1 + l2] * sc[1], d3 = sD[g3 * p1 + l3] * sc[2];
                s += pu[kk * npt + x] * (a1 * a2 * a3);
                s -= pf[(kk * 3 + 0) * npt + x] * (d1 * a2 * a3);
                s -= pf[(kk * 3 + 1) * npt + x] * (a1 * d2 * a3);
                s -= pf[(kk * 3 + 2) * npt + x] * (a1 * a2 * d3);
            }
            acc_out(a.RV, a.tRV, oV + kk * Nn + A, s);
        } else if (VISC) {
            int c = kk - 5, k = c / 3, d = c % 3;
            for (int x = 0; x < npt; ++x) {
                int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
                double a1 = sL[g1 * p1 + l1], a2 = sL[g2 * p1 + l2], a3 = sL[g3 * p1 + l3];
                double dd = d == 0 ? sD[g1 * p1 + l1] * sc[0] * a2 * a3
                          : d == 1 ? a1 * sD[g2 * p1 + l2] * sc[1] * a3
                                   : a1 * a2 * sD[g3 * p1 + l3] * sc[2];
                s += pq[c * npt + x] * (a1 * a2 * a3) + pv[k * npt + x] * dd;
            }
            acc_out(a.RQ, a.tRQ, oQ + c * Nn + A, s);
        }
    }
}

// Sum-factorised volume pass (same result as residual_volume_kernel up to
// rounding order).  Interpolation to the Gauss points and testing against the
// basis are each three one-dimensional contractions over the tensor indices:
//   interpolation  nodes (l1,l2,l3) -> (g1,l2,l3) -> (g1,g2,l3) -> (g1,g2,g3)
//   testing        points (g1,g2,g3) -> (l1,g2,g3) -> (l1,l2,g3) -> (l1,l2,l3)
// The derivative factors of the weak form ride along as separate partial sums
// (H after the g1 contraction, J after g2).  Two shared regions alternate:
//   A: nodal state -> T2 -> H        B: T1 -> point values / integrands -> J
//
// LIN = true: the tangent dR_V[dv] of the volume pass from the stored weighted
// point Jacobians a.pj (written by the Jacobian kernels at the same state):
// only dv is interpolated, the point step is a 20 x 5 product per Gauss point
// instead of the dual-number physics, and the result goes to tRV.  On the
// viscous path (a.pq and a.dq set) dq is interpolated as well and the stored
// W dG/dq blocks add their 15 x 15 product per point: G is linear in q and its
// v-derivative at fixed q is part of the stored flux blocks.
template <class T, bool VISC, bool LIN>
__global__ void __launch_bounds__(128)
residual_volume_sf_kernel(ResidualArgs a, int nA) {
    static_assert(!LIN || (!VISC && std::is_same<T, double>::value), "linear pass: inviscid FP64 only");
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    if (a.skip && a.skip[K]) return;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn;
    const int nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    const Phys& ph = a.ph;
    const bool tt = !LIN && ph.time_term;
    const bool lq = LIN && a.pq && a.dq;                     // linear pass with the q-direction
    const int NIN = 5 + (tt ? 5 : 0) + (VISC || lq ? 15 : 0);     // v, v* (time term), q
    const int cq = tt ? 10 : 5;
    constexpr int NHK = VISC ? 7 : 3, NJK = VISC ? 6 : 2;   // partial sums per component k
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);         // [ng][p1]
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);          // [ng][p1]
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);          // [ng]
    T* RA = reinterpret_cast<T*>(sW + 8);
    T* RB = RA + nA;
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    const double* box = a.box + 6 * K;
    double sc[3], hw[3];
    for (int d = 0; d < 3; ++d) { double h = (box[3 + d] - box[d]) / m; sc[d] = 2.0 / h; hw[d] = 0.5 * h; }
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn;

    // nodal state of the micro-element -> A [NIN][nl]
    for (int i = tid; i < nl; i += nth) {
        int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
        int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
        for (int k = 0; k < 5; ++k) {
            if constexpr (LIN) RA[k * nl + i] = a.dv ? a.dv[oV + k * Nn + A] : 0.0;
            else RA[k * nl + i] = load_t<T>(a.v, a.dv, oV + k * Nn + A);
            if (tt) RA[(5 + k) * nl + i] = load_t<T>(a.vs, nullptr, oV + k * Nn + A);
        }
        if (VISC)
            for (int c = 0; c < 15; ++c) RA[(cq + c) * nl + i] = load_t<T>(a.q, a.dq, oQ + c * Nn + A);
        if constexpr (LIN)
            if (lq) for (int c = 0; c < 15; ++c) RA[(cq + c) * nl + i] = a.dq[oQ + c * Nn + A];
    }
    __syncthreads();
    // interpolation, g1: B[c][g1 + ng (l2 + p1 l3)]
    {
        const int s1 = ng * p1 * p1;
        for (int it = tid; it < NIN * s1; it += nth) {
            const int c = it / s1, o = it % s1, g1 = o % ng, r = o / ng;
            const T* src = RA + c * nl + r * p1;
            T s = cst<T>(0.0);
            for (int l = 0; l < p1; ++l) s += src[l] * sL[g1 * p1 + l];
            RB[it] = s;
        }
    }
    __syncthreads();
    // g2: A[c][g1 + ng (g2 + ng l3)]
    {
        const int s1 = ng * p1 * p1, s2 = ng * ng * p1;
        for (int it = tid; it < NIN * s2; it += nth) {
            const int c = it / s2, o = it % s2, g1 = o % ng, g2 = (o / ng) % ng, l3 = o / (ng * ng);
            const T* src = RB + c * s1 + g1 + ng * p1 * l3;
            T s = cst<T>(0.0);
            for (int l = 0; l < p1; ++l) s += src[ng * l] * sL[g2 * p1 + l];
            RA[it] = s;
        }
    }
    __syncthreads();
    // g3: B[c][x], x = g1 + ng (g2 + ng g3)
    {
        const int s2 = ng * ng * p1;
        for (int it = tid; it < NIN * npt; it += nth) {
            const int c = it / npt, x = it % npt, g12 = x % (ng * ng), g3 = x / (ng * ng);
            const T* src = RA + c * s2 + g12;
            T s = cst<T>(0.0);
            for (int l = 0; l < p1; ++l) s += src[ng * ng * l] * sL[g3 * p1 + l];
            RB[it] = s;
        }
    }
    __syncthreads();
    // point physics, in place in B (each thread touches only its own column x):
    // rows 0-4 W U, 5-19 W F/G (k*3+j), 20-34 W q (k*3+d), 35-39 W v
    bool ok = true;
    if constexpr (LIN) {
        // rows 0-4: W dU/dv dv; rows 5-19: W dFG/dv dv (the stored blocks carry -W)
        const double* Gb = a.pj + ((size_t)K * m * m * m + e) * 100 * npt;   // [100][npt]
        // viscous: W dG_kj/dq_(l,d) at [d*75 + j*25 + k*5 + l][npt], q component l*3 + d
        const double* Qb = lq ? a.pq + ((size_t)K * m * m * m + e) * 225 * npt : nullptr;
        for (int x = tid; x < npt; x += nth) {
            double dvx[5], dqx[15];
            for (int l = 0; l < 5; ++l) dvx[l] = RB[l * npt + x];
            if (lq) for (int c = 0; c < 15; ++c) dqx[c] = RB[(cq + c) * npt + x];
            const double* Gx = Gb + x;
            for (int k = 0; k < 5; ++k) {
                double u = 0.0, f[3] = {0.0, 0.0, 0.0};
                for (int l = 0; l < 5; ++l) {
                    u += Gx[(size_t)(k * 5 + l) * npt] * dvx[l];
                    f[0] += Gx[(size_t)(25 + k * 5 + l) * npt] * dvx[l];
                    f[1] += Gx[(size_t)(50 + k * 5 + l) * npt] * dvx[l];
                    f[2] += Gx[(size_t)(75 + k * 5 + l) * npt] * dvx[l];
                }
                RB[k * npt + x] = u;
                for (int j = 0; j < 3; ++j) {
                    double g = 0.0;
                    if (lq) {
                        const double* Qx = Qb + (size_t)(j * 25 + k * 5) * npt + x;
                        for (int d = 0; d < 3; ++d)
                            for (int l = 0; l < 5; ++l) g += Qx[(size_t)(d * 75 + l) * npt] * dqx[l * 3 + d];
                    }
                    RB[(5 + k * 3 + j) * npt + x] = g - f[j];
                }
            }
        }
    } else
    for (int x = tid; x < npt; x += nth) {
        const int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
        T vx[5], vsx[5], qx[15];
        for (int k = 0; k < 5; ++k) { vx[k] = RB[k * npt + x]; vsx[k] = tt ? RB[(5 + k) * npt + x] : cst<T>(0.0); }
        if (VISC) for (int c = 0; c < 15; ++c) qx[c] = RB[(cq + c) * npt + x];
        T U[5], FG[5][3];
        ok = vol_integrand(ph, vx, vsx, qx, U, FG) && ok;
        const double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
        for (int k = 0; k < 5; ++k) {
            RB[k * npt + x] = U[k] * W;
            for (int j = 0; j < 3; ++j) RB[(5 + k * 3 + j) * npt + x] = FG[k][j] * W;
        }
        if (VISC) {
            for (int c = 0; c < 15; ++c) RB[(20 + c) * npt + x] = qx[c] * W;
            for (int k = 0; k < 5; ++k) RB[(35 + k) * npt + x] = vx[k] * W;
        }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
    // testing, g1: A[k*NHK + j][l1 + p1 (g2 + ng g3)]
    {
        const int h1 = p1 * ng * ng;
        for (int it = tid; it < 5 * h1; it += nth) {
            const int k = it / h1, o = it % h1, l1 = o % p1, g23 = o / p1;
            const T* pu = RB + k * npt + g23 * ng;
            const T* pf = RB + (5 + 3 * k) * npt + g23 * ng;
            T h[NHK];
            for (int j = 0; j < NHK; ++j) h[j] = cst<T>(0.0);
            for (int g = 0; g < ng; ++g) {
                const double Lg = sL[g * p1 + l1], Dg = sD[g * p1 + l1] * sc[0];
                h[0] += pu[g] * Lg - pf[g] * Dg;
                h[1] += pf[npt + g] * Lg;
                h[2] += pf[2 * npt + g] * Lg;
                if (VISC) {
                    const T* pq = RB + (20 + 3 * k) * npt + g23 * ng;
                    const T pv = RB[(35 + k) * npt + g23 * ng + g];
                    h[3] += pq[g] * Lg + pv * Dg;
                    h[4] += pq[npt + g] * Lg;
                    h[5] += pq[2 * npt + g] * Lg;
                    h[6] += pv * Lg;
                }
            }
            for (int j = 0; j < NHK; ++j) RA[(k * NHK + j) * h1 + o] = h[j];
        }
    }
    __syncthreads();
    // g2: B[k*NJK + j][l1 + p1 (l2 + p1 g3)]
    {
        const int h1 = p1 * ng * ng, j1 = p1 * p1 * ng;
        for (int it = tid; it < 5 * j1; it += nth) {
            const int k = it / j1, o = it % j1, l1 = o % p1, l2 = (o / p1) % p1, g3 = o / (p1 * p1);
            const T* H = RA + k * NHK * h1 + l1 + p1 * ng * g3;
            T jv[NJK];
            for (int j = 0; j < NJK; ++j) jv[j] = cst<T>(0.0);
            for (int g = 0; g < ng; ++g) {
                const double Lg = sL[g * p1 + l2], Dg = sD[g * p1 + l2] * sc[1];
                const int o2 = p1 * g;
                jv[0] += H[o2] * Lg - H[h1 + o2] * Dg;
                jv[1] += H[2 * h1 + o2] * Lg;
                if (VISC) {
                    jv[2] += H[3 * h1 + o2] * Lg;
                    jv[3] += H[4 * h1 + o2] * Lg + H[6 * h1 + o2] * Dg;
                    jv[4] += H[5 * h1 + o2] * Lg;
                    jv[5] += H[6 * h1 + o2] * Lg;
                }
            }
            for (int j = 0; j < NJK; ++j) RB[(k * NJK + j) * j1 + o] = jv[j];
        }
    }
    __syncthreads();
    // g3: nodal rows of R_V (and R_Q), added into the element's rows
    {
        const int j1 = p1 * p1 * ng;
        for (int it = tid; it < 5 * nl; it += nth) {
            const int k = it / nl, i = it % nl, l12 = i % (p1 * p1), l3 = i / (p1 * p1);
            const int l1 = l12 % p1, l2 = l12 / p1;
            const T* J = RB + k * NJK * j1 + l12;
            T rv = cst<T>(0.0), rq0 = cst<T>(0.0), rq1 = cst<T>(0.0), rq2 = cst<T>(0.0);
            for (int g = 0; g < ng; ++g) {
                const double Lg = sL[g * p1 + l3], Dg = sD[g * p1 + l3] * sc[2];
                const int o3 = p1 * p1 * g;
                rv += J[o3] * Lg - J[j1 + o3] * Dg;
                if (VISC) {
                    rq0 += J[2 * j1 + o3] * Lg;
                    rq1 += J[3 * j1 + o3] * Lg;
                    rq2 += J[4 * j1 + o3] * Lg + J[5 * j1 + o3] * Dg;
                }
            }
            const int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
            if constexpr (LIN) { if (a.tRV) atomicAdd(a.tRV + oV + k * Nn + A, (double)rv); }
            else acc_out(a.RV, a.tRV, oV + k * Nn + A, rv);
            if (VISC) {
                acc_out(a.RQ, a.tRQ, oQ + (k * 3 + 0) * Nn + A, rq0);
                acc_out(a.RQ, a.tRQ, oQ + (k * 3 + 1) * Nn + A, rq1);
                acc_out(a.RQ, a.tRQ, oQ + (k * 3 + 2) * Nn + A, rq2);
            }
        }
    }
}

template <class T, bool VISC>
__global__ void __launch_bounds__(128)
residual_face_kernel(ResidualArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y;
    if (a.skip && a.skip[K]) return;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, n2 = tb.n2, p1 = p + 1;
    const int f = blockIdx.x / (m * m), e = blockIdx.x % (m * m);
    const int e1 = e % m, e2 = e / m;
    const int d = f / 2;
    const double sgn = (f & 1) ? 1.0 : -1.0;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int fl = p1 * p1, fpt = ng * ng;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    T* fv = reinterpret_cast<T*>(sW + 8);   // [5][fl]
    T* fh = fv + 5 * fl;           // [5][fl]
    T* fq = fh + 5 * fl;           // [15][fl]
    T* pF = fq + (VISC ? 15 * fl : 0);    // [5][fpt]
    T* pH = pF + 5 * fpt;          // [5][fpt]  W n_d vh (for R_Q)
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    const Phys& ph = a.ph;
    const double* box = a.box + 6 * K;
    const double hw1 = 0.5 * (box[3 + t1] - box[t1]) / m, hw2 = 0.5 * (box[3 + t2] - box[t2]) / m;
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn, oH = (int64_t)K * 30 * n2;
    const int64_t og = a.gid[6 * K + f] * 5 * n2;
    for (int i = tid; i < fl; i += nth) {
        int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        int A = idx[0] + n * (idx[1] + n * idx[2]);
        for (int k = 0; k < 5; ++k) {
            fv[k * fl + i] = load_t<T>(a.v, a.dv, oV + k * Nn + A);
            fh[k * fl + i] = load_t<T>(a.vh, a.dvh, og + k * n2 + c1 + n * c2);
        }
        if (VISC)
            for (int cc = 0; cc < 15; ++cc) fq[cc * fl + i] = load_t<T>(a.q, a.dq, oQ + cc * Nn + A);
    }
    __syncthreads();
    bool ok = true;
    for (int x = tid; x < fpt; x += nth) {
        int g1 = x % ng, g2 = x / ng;
        T vx[5], hx[5], qx[15];
        for (int k = 0; k < 5; ++k) { vx[k] = cst<T>(0.0); hx[k] = cst<T>(0.0); }
        if (VISC) for (int cc = 0; cc < 15; ++cc) qx[cc] = cst<T>(0.0);
        for (int i = 0; i < fl; ++i) {
            double mu = sL[g1 * p1 + (i % p1)] * sL[g2 * p1 + (i / p1)];
            for (int k = 0; k < 5; ++k) { vx[k] += fv[k * fl + i] * mu; hx[k] += fh[k * fl + i] * mu; }
            if (VISC) for (int cc = 0; cc < 15; ++cc) qx[cc] += fq[cc * fl + i] * mu;
        }
        T Fh[5];
        ok = face_integrand(ph, vx, hx, qx, d, sgn, Fh) && ok;
        double W = sW[g1] * hw1 * sW[g2] * hw2;
        for (int k = 0; k < 5; ++k) {
            pF[k * fpt + x] = Fh[k] * W;
            if (VISC) pH[k * fpt + x] = hx[k] * (W * sgn);
        }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
    for (int r = tid; r < fl * 5; r += nth) {
        int i = r % fl, k = r / fl;
        int l1 = i % p1, l2 = i / p1;
        int c1 = e1 * p + l1, c2 = e2 * p + l2;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        int A = idx[0] + n * (idx[1] + n * idx[2]);
        T s = cst<T>(0.0), sq = cst<T>(0.0);
        for (int x = 0; x < fpt; ++x) {
            double mu = sL[(x % ng) * p1 + l1] * sL[(x / ng) * p1 + l2];
            s += pF[k * fpt + x] * mu;
            if (VISC) sq += pH[k * fpt + x] * mu;
        }
        acc_out(a.RV, a.tRV, oV + k * Nn + A, s);
        acc_out(a.RH, a.tRH, oH + (f * 5 + k) * n2 + c1 + n * c2, s);
        if (VISC) acc_out(a.RQ, a.tRQ, oQ + (k * 3 + d) * Nn + A, -sq);
    }
}

// Linear face pass of the tangent with dvhat = 0: the stored weighted face
// blocks W d(Fhat + Ghat)/dv of the Jacobian kernel, applied to dv
// interpolated to the face points, plus on the viscous path the blocks
// W dGhat/dq applied to the interior dq; tested against the face nodes, added
// into tRV and into the element's side of the trace tangent tRH.
__global__ void __launch_bounds__(128)
residual_face_lin_kernel(ResidualArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y;
    if (a.skip && a.skip[K]) return;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, n2 = tb.n2, p1 = p + 1;
    const int f = blockIdx.x / (m * m), e = blockIdx.x % (m * m);
    const int e1 = e % m, e2 = e / m;
    const int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int fl = p1 * p1, fpt = ng * ng;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);          // [ng][p1]
    const bool lq = a.pqf && a.dq;
    double* fd = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);           // [5][fl] dv on the face nodes
    double* fdq = fd + 5 * fl;                                 // [15][fl] dq on the face nodes (viscous)
    double* pF = fdq + (lq ? 15 * fl : 0);                     // [5][fpt]
    int* nodeA = reinterpret_cast<int*>(pF + 5 * fpt);         // [fl]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    const int64_t oV = (int64_t)K * 5 * Nn, oH = (int64_t)K * 30 * n2;
    for (int i = tid; i < fl; i += nth) {
        const int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        const int A = idx[0] + n * (idx[1] + n * idx[2]);
        nodeA[i] = A;
        for (int k = 0; k < 5; ++k) fd[k * fl + i] = a.dv ? a.dv[oV + k * Nn + A] : 0.0;
        if (lq) for (int c = 0; c < 15; ++c) fdq[c * fl + i] = a.dq[(int64_t)K * 15 * Nn + c * Nn + A];
    }
    __syncthreads();
    const double* Gb = a.pjf + ((size_t)K * 6 * m * m + blockIdx.x) * 25 * fpt;   // [25][fpt]
    // viscous: W dGhat_k/dq_(l,d) at [d*25 + k*5 + l][fpt], q component l*3 + d
    const double* Qb = lq ? a.pqf + ((size_t)K * 6 * m * m + blockIdx.x) * 75 * fpt : nullptr;
    for (int x = tid; x < fpt; x += nth) {
        const int g1 = x % ng, g2 = x / ng;
        double dvx[5] = {0, 0, 0, 0, 0}, dqx[15];
        for (int c = 0; c < 15; ++c) dqx[c] = 0.0;
        for (int i = 0; i < fl; ++i) {
            const double mu = sL[g1 * p1 + i % p1] * sL[g2 * p1 + i / p1];
            for (int k = 0; k < 5; ++k) dvx[k] += fd[k * fl + i] * mu;
            if (lq) for (int c = 0; c < 15; ++c) dqx[c] += fdq[c * fl + i] * mu;
        }
        const double* Gx = Gb + x;
        for (int k = 0; k < 5; ++k) {
            double s = 0.0;
            for (int l = 0; l < 5; ++l) s += Gx[(size_t)(k * 5 + l) * fpt] * dvx[l];
            if (lq)
                for (int d = 0; d < 3; ++d)
                    for (int l = 0; l < 5; ++l) s += Qb[(size_t)(d * 25 + k * 5 + l) * fpt + x] * dqx[l * 3 + d];
            pF[k * fpt + x] = s;
        }
    }
    __syncthreads();
    for (int r = tid; r < fl * 5; r += nth) {
        const int i = r % fl, k = r / fl;
        const int l1 = i % p1, l2 = i / p1;
        double s = 0.0;
        for (int x = 0; x < fpt; ++x) s += pF[k * fpt + x] * sL[(x % ng) * p1 + l1] * sL[(x / ng) * p1 + l2];
        if (a.tRV) atomicAdd(a.tRV + oV + k * Nn + nodeA[i], s);
        if (a.tRH) atomicAdd(a.tRH + oH + (f * 5 + k) * n2 + (e1 * p + l1) + n * (e2 * p + l2), s);
    }
}

// sum the (one or two) element sides of every global face
__global__ void trace_gather_kernel(const double* __restrict__ loc, const int64_t* __restrict__ g2l,
                                    int64_t G, int n2, double* __restrict__ out, double alpha,
                                    const double* __restrict__ add, double beta) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per = 5 * (int64_t)n2;
    if (i >= G * per) return;
    int64_t g = i / per, r = i % per;
    double s = 0.0;
    for (int side = 0; side < 2; ++side) {
        int64_t kf = g2l[2 * g + side];
        if (kf >= 0) s += loc[kf * per + r];
    }
    double o = alpha * s;
    if (add) o += beta * add[i];
    out[i] = o;
}

// zero the outputs of the elements that are not skipped
__global__ void zero_outputs_kernel(double* a, double* b, int64_t per, const int32_t* skip) {
    const int K = blockIdx.y;
    if (skip && skip[K]) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
        if (a) a[(size_t)K * per + i] = 0.0;
        if (b) b[(size_t)K * per + i] = 0.0;
    }
}

namespace {

size_t head_bytes() { return sizeof(double) * (2 * MEHDG_MAXG * (MEHDG_MAXP + 1) + 8); }

size_t volume_smem_bytes(const Tab& t, bool visc, size_t ts) {
    size_t n = (size_t)(10 + (visc ? 15 : 0)) * t.nl + (size_t)(20 + (visc ? 20 : 0)) * t.npt;
    return head_bytes() + ts * n;
}

// region sizes (entries) of the sum-factorised volume kernel
void volume_sf_regions(const Tab& t, bool visc, int& nA, int& nB) {
    const int p1 = t.p + 1, ng = t.ng;
    const int nin = 10 + (visc ? 15 : 0);       // v, v* (counted whether or not the time term is on), q
    const int nout = visc ? 40 : 20, nh = 5 * (visc ? 7 : 3), nj = 5 * (visc ? 6 : 2);
    nA = std::max(std::max(nin * t.nl, nin * ng * ng * p1), nh * p1 * ng * ng);
    nB = std::max(std::max(nin * ng * p1 * p1, std::max(nin, nout) * t.npt), nj * p1 * p1 * ng);
}

size_t volume_sf_smem_bytes(const Tab& t, bool visc, size_t ts) {
    int nA, nB;
    volume_sf_regions(t, visc, nA, nB);
    return head_bytes() + ts * (size_t)(nA + nB);
}

size_t face_smem_bytes(const Tab& t, bool visc, size_t ts) {
    int fl = (t.p + 1) * (t.p + 1), fpt = t.ng * t.ng;
    size_t n = (size_t)(10 + (visc ? 15 : 0)) * fl + 10 * (size_t)fpt;
    return head_bytes() + ts * n;
}

cudaError_t zero(double* a, double* b, int64_t per, int64_t nK, const int32_t* skip, cudaStream_t st) {
    if (!a && !b) return cudaSuccess;
    dim3 g((unsigned)((per + 255) / 256 < 64 ? (per + 255) / 256 : 64), (unsigned)nK);
    zero_outputs_kernel<<<g, 256, 0, st>>>(a, b, per, skip);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_residual(const ResidualArgs& a, int64_t nK, bool visc, bool tangent, cudaStream_t st) {
    const Tab& t = a.tab;
    cudaError_t e;
    if ((e = zero(a.RV, a.tRV, 5LL * t.Nn, nK, a.skip, st)) != cudaSuccess) return e;
    if (visc && (e = zero(a.RQ, a.tRQ, 15LL * t.Nn, nK, a.skip, st)) != cudaSuccess) return e;
    if ((e = zero(a.RH, a.tRH, 30LL * t.n2, nK, a.skip, st)) != cudaSuccess) return e;
    size_t ts = tangent ? sizeof(Dual<1>) : sizeof(double);
    size_t sv = volume_smem_bytes(t, visc, ts), sf = face_smem_bytes(t, visc, ts);
    // the sum-factorised volume pass wherever its two regions fit in shared memory
    int nA, nB;
    volume_sf_regions(t, visc, nA, nB);
    const size_t ssf = volume_sf_smem_bytes(t, visc, ts);
    const bool sf_vol = ssf <= 220 * 1024;
    dim3 gv((unsigned)(t.m * t.m * t.m), (unsigned)nK), gf((unsigned)(6 * t.m * t.m), (unsigned)nK), b(128);
#define LAUNCH_RES(T, V)                                                                                 \
    do { if (sf_vol) {                                                                                   \
             cudaFuncSetAttribute(residual_volume_sf_kernel<T, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssf); \
             residual_volume_sf_kernel<T, V, false><<<gv, b, ssf, st>>>(a, nA);                                  \
         } else {                                                                                        \
             cudaFuncSetAttribute(residual_volume_kernel<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv); \
             residual_volume_kernel<T, V><<<gv, b, sv, st>>>(a);                                         \
         }                                                                                               \
         cudaFuncSetAttribute(residual_face_kernel<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);   \
         residual_face_kernel<T, V><<<gf, b, sf, st>>>(a); } while (0)
    if (tangent && a.pj && sf_vol && (!visc || (a.pq && !a.RQ && !a.tRQ))) {
        // linear volume pass from the stored point Jacobians (none when dv = 0
        // and dq = 0: the volume integrand does not depend on the traces; on the
        // viscous path only when the R_Q rows are not asked for), then the face
        // pass: linear when the trace direction is 0, else dual numbers
        if (a.dv || (visc && a.dq)) {
            const size_t sl = volume_sf_smem_bytes(t, visc, sizeof(double));
            cudaFuncSetAttribute(residual_volume_sf_kernel<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
            residual_volume_sf_kernel<double, false, true><<<gv, b, sl, st>>>(a, nA);
        }
        if (a.pjf && !a.dvh && (!visc || a.pqf)) {
            // linear face pass (viscous: with the dGhat/dq blocks); nothing to add
            // when neither dv nor dq is set
            if (a.dv || (visc && a.dq)) {
                const int fl = (t.p + 1) * (t.p + 1), fpt = t.ng * t.ng;
                const size_t sfl = sizeof(double) * (MEHDG_MAXG * (MEHDG_MAXP + 1) + (visc ? 20 : 5) * (size_t)fl +
                                                     5 * (size_t)fpt)
                                 + sizeof(int) * fl + 16;
                residual_face_lin_kernel<<<gf, b, sfl, st>>>(a);
            }
        } else if (visc) {
            cudaFuncSetAttribute(residual_face_kernel<Dual<1>, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
            residual_face_kernel<Dual<1>, true><<<gf, b, sf, st>>>(a);
        } else {
            cudaFuncSetAttribute(residual_face_kernel<Dual<1>, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
            residual_face_kernel<Dual<1>, false><<<gf, b, sf, st>>>(a);
        }
    } else if (tangent) { if (visc) LAUNCH_RES(Dual<1>, true); else LAUNCH_RES(Dual<1>, false); }
    else { if (visc) LAUNCH_RES(double, true); else LAUNCH_RES(double, false); }
#undef LAUNCH_RES
    MEHDG_COUNT(2);
    return cudaGetLastError();
}

cudaError_t launch_trace_gather(const double* loc, const int64_t* g2l, int64_t G, int n2, double* out,
                                double alpha, const double* add, double beta, cudaStream_t st) {
    int64_t N = G * 5 * n2;
    int bs = 256;
    trace_gather_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(loc, g2l, G, n2, out, alpha, add, beta);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}
