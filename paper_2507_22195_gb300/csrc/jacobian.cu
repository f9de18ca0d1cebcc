// jacobian.cu -- assembly of the dense Schur matrix S^K = A_vv (eqs. R1, R3)
// of every macro-element, in FP32 (mixed path) or FP64.
//
// The point-wise Jacobians of the integrands (5x5 blocks dU/dv and
// dFG_j/dv at every Gauss point, dF-hat/dv at every face point) come from
// forward-mode duals with 5 tangent directions (FP64 log/exp of the
// entropy-to-conservative map and of the logarithmic means).  They are
// weighted and contracted with the basis of the micro-element:
//   S[(k,A),(l,B)] += sum_x W [ phi_A phi_B dU_k/dv_l - sum_j d_j phi_A phi_B dFG_kj/dv_l ]
//                   + sum_faces sum_x w mu_A mu_B dFhat_k/dv_l.
// Volume contraction by sum factorisation over the three tensor directions
// (test/trial pair tables per direction; about 2.9M FMA per micro-element at
// p = 3 instead of 51M pair by pair), per trial component l; the pair-by-pair form
// remains for the case whose staging does not fit in shared memory (FP64,
// p = 4).  Results are added into S with atomics (micro-elements share
// nodes).  Unknowns are ordered node-major, row (A, k) = 5 A + k, so the
// partial pivoting (which mostly exchanges components of one node) stays
// inside a block of rows.  S is column-major with a padded leading
// dimension; the padding is an identity block.
#include "physics.cuh"
#include "kernels.cuh"

namespace {

__device__ __forceinline__ void atomic_add_t(float* p, double x) { atomicAdd(p, (float)x); }
__device__ __forceinline__ void atomic_add_t(double* p, double x) { atomicAdd(p, x); }

constexpr int HEAD_DOUBLES = 2 * MEHDG_MAXG * (MEHDG_MAXP + 1) + 8;

// Stage the local state of micro-element (e1,e2,e3) of element K and write
// the weighted point Jacobians P[x][alpha][k*5+l] (alpha 0: W dU/dv; alpha
// 1..3: -W dFG_j/dv).  vl/vsl/ql: shared scratch.
template <class TS, bool VISC>
__device__ void volume_point_jacobians(const JacobianArgs& a, int K, int e1, int e2, int e3, const double* sL,
                                       const double* sW, const double* hw, double* vl, double* vsl, double* ql,
                                       TS* P) {
    const Tab& tb = a.tab;
    const int p = tb.p, n = tb.n, ng = tb.ng, Nn = tb.Nn, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn;
    for (int i = tid; i < nl; i += nth) {
        int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
        int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
        for (int k = 0; k < 5; ++k) {
            vl[k * nl + i] = a.v[oV + k * Nn + A];
            vsl[k * nl + i] = a.ph.time_term ? a.vs[oV + k * Nn + A] : 0.0;
        }
        if (VISC) for (int c = 0; c < 15; ++c) ql[c * nl + i] = a.q[oQ + c * Nn + A];
    }
    __syncthreads();
    bool ok = true;
    for (int x = tid; x < npt; x += nth) {
        int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
        double vx[5] = {0, 0, 0, 0, 0}, vsx[5] = {0, 0, 0, 0, 0}, qx[15];
        for (int c = 0; c < 15; ++c) qx[c] = 0.0;
        for (int i = 0; i < nl; ++i) {
            double f = sL[g1 * p1 + i % p1] * sL[g2 * p1 + (i / p1) % p1] * sL[g3 * p1 + i / (p1 * p1)];
            for (int k = 0; k < 5; ++k) { vx[k] += f * vl[k * nl + i]; vsx[k] += f * vsl[k * nl + i]; }
            if (VISC) for (int c = 0; c < 15; ++c) qx[c] += f * ql[c * nl + i];
        }
        Dual<5> dv[5], dvs[5], dq[15];
        for (int k = 0; k < 5; ++k) {
            dv[k] = mkdual<5>(vx[k]); dv[k].d[k] = 1.0;
            dvs[k] = mkdual<5>(vsx[k]);
        }
        for (int c = 0; c < 15; ++c) dq[c] = mkdual<5>(qx[c]);
        Dual<5> U[5], FG[5][3];
        ok = vol_integrand(a.ph, dv, dvs, dq, U, FG) && ok;
        double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
        TS* Px = P ? P + (size_t)x * 100 : nullptr;
        // stored point-fastest, [K][micro-element][100][npt]: coalesced over the points
        double* Gx = a.pj ? a.pj + ((size_t)K * tb.m * tb.m * tb.m + e1 + tb.m * (e2 + tb.m * e3)) * 100 * npt + x
                          : nullptr;
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l) {
                const double u = W * U[k].d[l];
                if (Px) Px[k * 5 + l] = (TS)u;
                if (Gx) Gx[(size_t)(k * 5 + l) * npt] = u;
                for (int j = 0; j < 3; ++j) {
                    const double f = -W * FG[k][j].d[l];
                    if (Px) Px[25 * (1 + j) + k * 5 + l] = (TS)f;
                    if (Gx) Gx[(size_t)(25 * (1 + j) + k * 5 + l) * npt] = f;
                }
            }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
}

__device__ __forceinline__ void geometry(const JacobianArgs& a, int K, double* sc, double* hw) {
    const double* box = a.box + 6 * K;
    for (int d = 0; d < 3; ++d) { double h = (box[3 + d] - box[d]) / a.tab.m; sc[d] = 2.0 / h; hw[d] = 0.5 * h; }
}

__device__ __forceinline__ void load_tables(const Tab& tb, double* sL, double* sD, double* sW) {
    const int p1 = tb.p + 1;
    for (int i = threadIdx.x; i < tb.ng * p1; i += blockDim.x) { sL[i] = tb.L[i / p1][i % p1]; sD[i] = tb.dL[i / p1][i % p1]; }
    if (threadIdx.x < tb.ng) sW[threadIdx.x] = tb.w[threadIdx.x];
}

// The contraction of the stored point blocks P into S for one micro-element,
// with p + 1 = P1 known at compile time (ng = p + 2 = P1 + 1): every index
// division is by a constant, the loops over the quadrature points unroll, and
// stage 3 keeps the P1 sums of a row a3 of an item as independent
// accumulators, reading that row of the z-table once per (alpha, g3) (as a
// float4 when P1 = 4).
// Every sum runs over its quadrature index in increasing order.  Mt:
// [3 dir][2 tau][NG][PP] pair tables, P: [NG^3][100],
// H1: [4 alpha][G2][P1 b1][P1 a1][5 k], O: the node index of the
// micro-element's first node in the macro-element.
template <int P1, class TS>
__device__ __forceinline__ void vol_contract(const TS* __restrict__ Mt, const TS* __restrict__ P, TS* __restrict__ H1,
                                             TS* S, int64_t ld, int n, int O) {
    constexpr int NG = P1 + 1, PP = P1 * P1, G2 = NG * NG, NH = 5 * 4 * PP * G2;
    const TS* M1 = Mt;
    const TS* M2 = Mt + 2 * NG * PP;
    const TS* M3 = Mt + 4 * NG * PP;
    const int tid = threadIdx.x, nth = blockDim.x;
    const size_t sa = (size_t)5 * n * n, sb = sa * (size_t)ld;
    for (int l = 0; l < 5; ++l) {
        // stage 1: contract g1 (alpha = 1 takes the x derivative of the test function)
        for (int i = tid; i < NH; i += nth) {
            const int k = i % 5, a1 = (i / 5) % P1, b1 = (i / (5 * P1)) % P1;
            const int g23 = (i / (5 * PP)) % G2, al = i / (5 * PP * G2);
            const TS* Mx = M1 + (al == 1 ? NG * PP : 0) + a1 * P1 + b1;
            const TS* Pc = P + (size_t)NG * g23 * 100 + 25 * al + 5 * k + l;
            TS s = 0;
#pragma unroll
            for (int g1 = 0; g1 < NG; ++g1) s += Mx[g1 * PP] * Pc[g1 * 100];
            H1[i] = s;
        }
        __syncthreads();
        // stages 2 and 3 per item (k, a1, a2, b1, b2)
        for (int it = tid; it < 5 * PP * PP; it += nth) {
            int r = it;
            const int k = r % 5; r /= 5;
            const int a1 = r % P1; r /= P1;
            const int a2 = r % P1; r /= P1;
            const int b1 = r % P1; const int b2 = r / P1;
            TS h2[4][NG];
#pragma unroll
            for (int al = 0; al < 4; ++al) {
                const TS* My = M2 + (al == 2 ? NG * PP : 0) + a2 * P1 + b2;
                const TS* h = H1 + al * G2 * 5 * PP + (b1 * P1 + a1) * 5 + k;
#pragma unroll
                for (int g3 = 0; g3 < NG; ++g3) {
                    TS s = 0;
#pragma unroll
                    for (int g2 = 0; g2 < NG; ++g2) s += My[g2 * PP] * h[(g2 + NG * g3) * 5 * PP];
                    h2[al][g3] = s;
                }
            }
            TS* Sb = S + (size_t)((O + a1 + n * a2) * 5 + k) + (size_t)((O + b1 + n * b2) * 5 + l) * ld;
#pragma unroll 1
            for (int a3 = 0; a3 < P1; ++a3) {
                TS acc[P1];
#pragma unroll
                for (int q = 0; q < P1; ++q) acc[q] = 0;
#pragma unroll
                for (int al = 0; al < 4; ++al) {
                    const TS* Mz = M3 + (al == 3 ? NG * PP : 0) + a3 * P1;
#pragma unroll
                    for (int g3 = 0; g3 < NG; ++g3) {
                        const TS hv = h2[al][g3];
                        const TS* row = Mz + g3 * PP;
                        if constexpr (P1 == 4 && sizeof(TS) == 4) {
                            const float4 v = *reinterpret_cast<const float4*>(row);
                            acc[0] += v.x * hv;
                            acc[1] += v.y * hv;
                            acc[2] += v.z * hv;
                            acc[3] += v.w * hv;
                        } else {
#pragma unroll
                            for (int q = 0; q < P1; ++q) acc[q] += row[q] * hv;
                        }
                    }
                }
#pragma unroll
                for (int b3 = 0; b3 < P1; ++b3) atomic_add_t(Sb + a3 * sa + b3 * sb, (double)acc[b3]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- sum factorised
// Per trial component l: stage 1 contracts g1 for all five test components k
// into H1[alpha][g2 g3][b1][a1][k]; then every thread takes items
// (k, a1, a2, b1, b2), contracts g2 into registers (4 x ng values) and g3 for
// all (a3, b3), and adds the p1^2 results into S.  Items are ordered k
// fastest, then a1, so a warp's atomics fall on runs of 5 p1 consecutive rows
// 5 A + k of one column, and its reads of H1 on consecutive words (with k or
// a1 slowest in H1, the 20 lanes would read one shared-memory bank).
// Point pass alone (inviscid, with a.pj): the dual-number physics at the
// Gauss points of one micro-element, written to a.pj.  Its 255 registers no
// longer hold the contraction below to one CTA per SM.
__global__ void __launch_bounds__(128)
jac_points_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int m = tb.m, nl = tb.nl;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* vl = sW + 8;
    double* vsl = vl + 5 * nl;
    double* ql = vsl + 5 * nl;
    load_tables(tb, sL, sD, sW);
    double sc[3], hw[3];
    geometry(a, K, sc, hw);
    __syncthreads();
    volume_point_jacobians<float, false>(a, K, e1, e2, e3, sL, sW, hw, vl, vsl, ql, (float*)nullptr);
}

// PRE: the point blocks come from a.pj (written by jac_points_kernel) instead
// of being computed here.
template <class TS, bool VISC, bool PRE = false>
__global__ void __launch_bounds__(256, PRE ? 2 : 1)
jac_volume_sf_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int PP = p1 * p1;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    TS* Mt = reinterpret_cast<TS*>(sW + 8);                 // [3][2][ng][PP] pair tables
    TS* P = Mt + 6 * MEHDG_MAXG * (MEHDG_MAXP + 1) * (MEHDG_MAXP + 1);   // [npt][100]
    unsigned char* uni = reinterpret_cast<unsigned char*>(P + (size_t)npt * 100);
    double* vl = reinterpret_cast<double*>(uni);            // phase 1: nodal state
    double* vsl = vl + 5 * nl;
    double* ql = vsl + 5 * nl;
    // phase 2: H1[al][g23][b1][a1][k], so that the lanes of a warp (k fastest,
    // then a1) read consecutive words in stage 2
    TS* H1 = reinterpret_cast<TS*>(uni);
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    double sc[3], hw[3];
    geometry(a, K, sc, hw);
    __syncthreads();
    // pair tables: Mt[d][tau][g][a*p1+b] = (tau ? dphi_a : phi_a)(g) phi_b(g), direction d
    for (int i = tid; i < 6 * ng * PP; i += nth) {
        int ab = i % PP, g = (i / PP) % ng, dt = i / (PP * ng), d = dt >> 1, tau = dt & 1;
        int aa = ab / p1, bb = ab % p1;
        double t = tau ? sD[g * p1 + aa] * sc[d] : sL[g * p1 + aa];
        Mt[i] = (TS)(t * sL[g * p1 + bb]);
    }
    if constexpr (PRE) {
        const double* Gb = a.pj + ((size_t)K * m * m * m + e) * 100 * npt;    // [100][npt]
        for (int i = tid; i < 100 * npt; i += nth) {
            const int idx = i / npt, x = i % npt;
            P[(size_t)x * 100 + idx] = (TS)Gb[i];
        }
        __syncthreads();
    } else {
        volume_point_jacobians<TS, VISC>(a, K, e1, e2, e3, sL, sW, hw, vl, vsl, ql, P);
    }
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    const int O = e1 * p + n * (e2 * p + n * e3 * p);
    switch (p1) {
    case 2: vol_contract<2, TS>(Mt, P, H1, S, a.ld, n, O); break;
    case 3: vol_contract<3, TS>(Mt, P, H1, S, a.ld, n, O); break;
    case 4: vol_contract<4, TS>(Mt, P, H1, S, a.ld, n, O); break;
    default: vol_contract<5, TS>(Mt, P, H1, S, a.ld, n, O); break;    // p = MEHDG_MAXP
    }
}

// ---------------------------------------------------------------- pair by pair
template <class TS, bool VISC>
__global__ void __launch_bounds__(256)
jac_volume_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* vl = sW + 8;                  // [5][nl]
    double* vsl = vl + 5 * nl;            // [5][nl]
    double* ql = vsl + 5 * nl;            // [15][nl]
    TS* P = reinterpret_cast<TS*>(ql + (VISC ? 15 * nl : 0));   // [npt][4][25]
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    double sc[3], hw[3];
    geometry(a, K, sc, hw);
    __syncthreads();
    volume_point_jacobians<TS, VISC>(a, K, e1, e2, e3, sL, sW, hw, vl, vsl, ql, P);
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    const int npair = nl * nl;
    for (int r = tid; r < npair; r += nth) {
        int ia = r / nl, ib = r % nl;
        int la[3] = {ia % p1, (ia / p1) % p1, ia / (p1 * p1)};
        int lb[3] = {ib % p1, (ib / p1) % p1, ib / (p1 * p1)};
        TS acc[25];
        for (int i = 0; i < 25; ++i) acc[i] = 0;
        for (int x = 0; x < npt; ++x) {
            int g[3] = {x % ng, (x / ng) % ng, x / (ng * ng)};
            double Aa[3], Ad[3], Bb = 1.0;
            for (int d = 0; d < 3; ++d) {
                Aa[d] = sL[g[d] * p1 + la[d]];
                Ad[d] = sD[g[d] * p1 + la[d]] * sc[d];
                Bb *= sL[g[d] * p1 + lb[d]];
            }
            TS c0 = (TS)(Aa[0] * Aa[1] * Aa[2] * Bb), c1 = (TS)(Ad[0] * Aa[1] * Aa[2] * Bb);
            TS c2 = (TS)(Aa[0] * Ad[1] * Aa[2] * Bb), c3 = (TS)(Aa[0] * Aa[1] * Ad[2] * Bb);
            const TS* Px = P + (size_t)x * 100;
            for (int kl = 0; kl < 25; ++kl)
                acc[kl] += c0 * Px[kl] + c1 * Px[25 + kl] + c2 * Px[50 + kl] + c3 * Px[75 + kl];
        }
        int A = (e1 * p + la[0]) + n * ((e2 * p + la[1]) + n * (e3 * p + la[2]));
        int B = (e1 * p + lb[0]) + n * ((e2 * p + lb[1]) + n * (e3 * p + lb[2]));
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l)
                atomic_add_t(&S[(size_t)(A * 5 + k) + (size_t)(B * 5 + l) * a.ld], (double)acc[k * 5 + l]);
    }
}

// ---------------------------------------------------------------- faces
template <class TS, bool VISC>
__global__ void __launch_bounds__(256)
jac_face_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, n2 = tb.n2, p1 = p + 1;
    const int f = blockIdx.x / (m * m), e = blockIdx.x % (m * m);
    const int e1 = e % m, e2 = e / m;
    const int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const double sgn = (f & 1) ? 1.0 : -1.0;
    const int fl = p1 * p1, fpt = ng * ng;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sW = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* fv = sW + 8;              // [5][fl]
    double* fh = fv + 5 * fl;         // [5][fl]
    double* fq = fh + 5 * fl;         // [15][fl]
    int* nodeA = reinterpret_cast<int*>(fq + 15 * fl);   // [fl]
    TS* P = reinterpret_cast<TS*>(reinterpret_cast<double*>(nodeA) + ((fl + 1) / 2 + 1));  // [fpt][25]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    if (tid < ng) sW[tid] = tb.w[tid];
    const double* box = a.box + 6 * K;
    double hw1 = 0.5 * (box[3 + t1] - box[t1]) / m, hw2 = 0.5 * (box[3 + t2] - box[t2]) / m;
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn, og = a.gid[6 * K + f] * 5 * n2;
    for (int i = tid; i < fl; i += nth) {
        int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        int A = idx[0] + n * (idx[1] + n * idx[2]);
        nodeA[i] = A;
        for (int k = 0; k < 5; ++k) {
            fv[k * fl + i] = a.v[oV + k * Nn + A];
            fh[k * fl + i] = a.vh[og + k * n2 + c1 + n * c2];
        }
        if (VISC) for (int c = 0; c < 15; ++c) fq[c * fl + i] = a.q[oQ + c * Nn + A];
    }
    __syncthreads();
    for (int x = tid; x < fpt; x += nth) {
        int g1 = x % ng, g2 = x / ng;
        double vx[5] = {0, 0, 0, 0, 0}, hx[5] = {0, 0, 0, 0, 0}, qx[15];
        for (int c = 0; c < 15; ++c) qx[c] = 0.0;
        for (int i = 0; i < fl; ++i) {
            double mu = sL[g1 * p1 + i % p1] * sL[g2 * p1 + i / p1];
            for (int k = 0; k < 5; ++k) { vx[k] += mu * fv[k * fl + i]; hx[k] += mu * fh[k * fl + i]; }
            if (VISC) for (int c = 0; c < 15; ++c) qx[c] += mu * fq[c * fl + i];
        }
        Dual<5> dv[5], dh[5], dq[15];
        for (int k = 0; k < 5; ++k) { dv[k] = mkdual<5>(vx[k]); dv[k].d[k] = 1.0; dh[k] = mkdual<5>(hx[k]); }
        for (int c = 0; c < 15; ++c) dq[c] = mkdual<5>(qx[c]);
        Dual<5> Fh[5];
        face_integrand(a.ph, dv, dh, dq, d, sgn, Fh);
        double W = sW[g1] * hw1 * sW[g2] * hw2;
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l) {
                P[x * 25 + k * 5 + l] = (TS)(W * Fh[k].d[l]);
                if (a.pjf) a.pjf[(((size_t)K * 6 * m * m + blockIdx.x) * 25 + k * 5 + l) * fpt + x] = W * Fh[k].d[l];
            }
    }
    __syncthreads();
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    // pairs (ia, ib), ia fastest: a warp's atomics for one (k, l) fall on a few
    // rows of one or two columns
    for (int r = tid; r < fl * fl; r += nth) {
        int ia = r % fl, ib = r / fl;
        TS acc[25];
        for (int i = 0; i < 25; ++i) acc[i] = 0;
        for (int x = 0; x < fpt; ++x) {
            int g1 = x % ng, g2 = x / ng;
            TS c = (TS)(sL[g1 * p1 + ia % p1] * sL[g2 * p1 + ia / p1] * sL[g1 * p1 + ib % p1] * sL[g2 * p1 + ib / p1]);
            for (int kl = 0; kl < 25; ++kl) acc[kl] += c * P[x * 25 + kl];
        }
        int A = nodeA[ia], B = nodeA[ib];
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l)
                atomic_add_t(&S[(size_t)(A * 5 + k) + (size_t)(B * 5 + l) * a.ld], (double)acc[k * 5 + l]);
    }
}

// Face point pass alone (with a.pjf): the dual-number two-point flux at every
// Gauss point of one macro-face (all its micro-faces, one thread per point),
// written as the weighted FP64 blocks W d(Fhat+Ghat)/dv (the layout of the
// fused kernel above).  It adds nothing into S, so it can run beside the
// zeroing of S; jac_face_contract_kernel then reads the blocks.
template <bool VISC>
__global__ void __launch_bounds__(256)
jac_face_points_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, f = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, n2 = tb.n2, p1 = p + 1;
    const int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const double sgn = (f & 1) ? 1.0 : -1.0;
    const int fl = p1 * p1, fpt = ng * ng, mm = m * m;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sW = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* fv = sW + 8;              // [5][n2] element values on the face
    double* fh = fv + 5 * n2;         // [5][n2] trace values
    double* fq = fh + 5 * n2;         // [15][n2] (viscous)
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    if (tid < ng) sW[tid] = tb.w[tid];
    const double* box = a.box + 6 * K;
    const double hw1 = 0.5 * (box[3 + t1] - box[t1]) / m, hw2 = 0.5 * (box[3 + t2] - box[t2]) / m;
    const int64_t oV = (int64_t)K * 5 * Nn, oQ = (int64_t)K * 15 * Nn, og = a.gid[6 * K + f] * 5 * n2;
    for (int c = tid; c < n2; c += nth) {
        const int c1 = c % n, c2 = c / n;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        const int A = idx[0] + n * (idx[1] + n * idx[2]);
        for (int k = 0; k < 5; ++k) {
            fv[k * n2 + c] = a.v[oV + k * Nn + A];
            fh[k * n2 + c] = a.vh[og + k * n2 + c];
        }
        if (VISC) for (int q = 0; q < 15; ++q) fq[q * n2 + c] = a.q[oQ + q * Nn + A];
    }
    __syncthreads();
    for (int t = tid; t < mm * fpt; t += nth) {
        const int e = t / fpt, x = t % fpt;
        const int e1 = e % m, e2 = e / m, g1 = x % ng, g2 = x / ng;
        double vx[5] = {0, 0, 0, 0, 0}, hx[5] = {0, 0, 0, 0, 0}, qx[15];
        for (int q = 0; q < 15; ++q) qx[q] = 0.0;
        for (int i = 0; i < fl; ++i) {
            const double mu = sL[g1 * p1 + i % p1] * sL[g2 * p1 + i / p1];
            const int c = (e1 * p + i % p1) + n * (e2 * p + i / p1);
            for (int k = 0; k < 5; ++k) { vx[k] += mu * fv[k * n2 + c]; hx[k] += mu * fh[k * n2 + c]; }
            if (VISC) for (int q = 0; q < 15; ++q) qx[q] += mu * fq[q * n2 + c];
        }
        Dual<5> dv[5], dh[5], dq[15];
        for (int k = 0; k < 5; ++k) { dv[k] = mkdual<5>(vx[k]); dv[k].d[k] = 1.0; dh[k] = mkdual<5>(hx[k]); }
        for (int q = 0; q < 15; ++q) dq[q] = mkdual<5>(qx[q]);
        Dual<5> Fh[5];
        face_integrand(a.ph, dv, dh, dq, d, sgn, Fh);
        const double W = sW[g1] * hw1 * sW[g2] * hw2;
        double* out = a.pjf + (((size_t)K * 6 * mm + (size_t)f * mm + e) * 25) * fpt + x;
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l) out[(size_t)(k * 5 + l) * fpt] = W * Fh[k].d[l];
    }
}

// Contraction of the stored face blocks into S, one CTA per (micro-face,
// element): the pair loop of the fused kernel, at several CTAs per SM.
template <class TS>
__global__ void __launch_bounds__(256)
jac_face_contract_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, p1 = p + 1;
    const int f = blockIdx.x / (m * m), e = blockIdx.x % (m * m);
    const int e1 = e % m, e2 = e / m;
    const int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int fl = p1 * p1, fpt = ng * ng;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    int* nodeA = reinterpret_cast<int*>(sL + MEHDG_MAXG * (MEHDG_MAXP + 1));       // [fl]
    TS* P = reinterpret_cast<TS*>(sL + MEHDG_MAXG * (MEHDG_MAXP + 1) + (fl + 1) / 2 + 1);   // [fpt][25]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    for (int i = tid; i < fl; i += nth) {
        const int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        nodeA[i] = idx[0] + n * (idx[1] + n * idx[2]);
    }
    const double* blk = a.pjf + (((size_t)K * 6 * m * m + blockIdx.x) * 25) * fpt;
    for (int i = tid; i < 25 * fpt; i += nth) {
        const int kl = i / fpt, x = i % fpt;          // reads run over the points (coalesced)
        P[x * 25 + kl] = (TS)blk[i];
    }
    __syncthreads();
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    for (int r = tid; r < fl * fl; r += nth) {
        const int ia = r % fl, ib = r / fl;
        TS acc[25];
        for (int i = 0; i < 25; ++i) acc[i] = 0;
        for (int x = 0; x < fpt; ++x) {
            const int g1 = x % ng, g2 = x / ng;
            const TS c = (TS)(sL[g1 * p1 + ia % p1] * sL[g2 * p1 + ia / p1] * sL[g1 * p1 + ib % p1] *
                              sL[g2 * p1 + ib / p1]);
            for (int kl = 0; kl < 25; ++kl) acc[kl] += c * P[x * 25 + kl];
        }
        const int A = nodeA[ia], B = nodeA[ib];
        for (int k = 0; k < 5; ++k)
            for (int l = 0; l < 5; ++l)
                atomic_add_t(&S[(size_t)(A * 5 + k) + (size_t)(B * 5 + l) * a.ld], (double)acc[k * 5 + l]);
    }
}

// ---------------------------------------------------------------- viscous: -A_vq C
// The contraction of the point blocks P (direction d of q) into S for one
// micro-element, with p + 1 = P1 known at compile time (ng = P1 + 1): the
// quadrature loops unroll and the index divisions are by constants, except
// those by n (the line direction's trial count) and by kn.  Stage 1 gives a
// thread one (a1, g23, j, b1) and all kn components (the T1 values loaded
// once); stage 3 keeps four b3 sums of a row a3 as independent accumulators.
// Every sum runs over its quadrature index in increasing order, as in the
// formulas of the comment below.  T: [3 dir][2 tau][NG][TW] line tables
// (TW = P1 n), P: [NG^3][3 j][25 kl], H1: [3 j][G2][nb0 b1][P1 a1][kn kk].
template <int P1, class TS>
__device__ __forceinline__ void q_contract(const TS* __restrict__ T, const TS* __restrict__ P, TS* __restrict__ H1,
                                           TS* S, int64_t ld, int n, const int (&eo)[3], int d, int kg) {
    constexpr int NG = P1 + 1, G2 = NG * NG, PP = P1 * P1;
    const int TW = P1 * n;
    const int nb0 = d == 0 ? n : P1, nb1 = d == 1 ? n : P1, nb2 = d == 2 ? n : P1;
    const int PB = P1 * nb0;                        // (a1, b1) pairs
    const TS* T1 = T;                               // direction x (tau at + NG * TW)
    const TS* T2 = T + 2 * NG * TW;
    const TS* T3 = T + 4 * NG * TW;
    const int tid = threadIdx.x, nth = blockDim.x;
    const size_t sa = (size_t)5 * n * n, sb = sa * (size_t)ld;
    for (int l = 0; l < 5; ++l)
        for (int k0 = 0; k0 < 5; k0 += kg) {
            const int kn = 5 - k0 < kg ? 5 - k0 : kg;
            // stage 1: H1[j][g23][b1][a1][kk] = sum_g1 T1_(j==0)[g1][a1 b1] P[x][j][k l]
            for (int i = tid; i < P1 * G2 * 3 * nb0; i += nth) {
                const int a1 = i % P1, g23 = (i / P1) % G2, j = (i / (P1 * G2)) % 3, b1 = i / (3 * P1 * G2);
                const TS* Tx = T1 + (j == 0 ? NG * TW : 0) + a1 * nb0 + b1;
                const TS* Pc = P + (size_t)NG * g23 * 75 + 25 * j + 5 * k0 + l;
                TS tx[NG];
#pragma unroll
                for (int g1 = 0; g1 < NG; ++g1) tx[g1] = Tx[g1 * TW];
                TS* out = H1 + ((size_t)(j * G2 + g23) * PB + b1 * P1 + a1) * kn;
                for (int kk = 0; kk < kn; ++kk) {
                    TS s = 0;
#pragma unroll
                    for (int g1 = 0; g1 < NG; ++g1) s += tx[g1] * Pc[g1 * 75 + 5 * kk];
                    out[kk] = s;
                }
            }
            __syncthreads();
            // stages 2 and 3 per item (kk, a1, a2, b1, b2), kk fastest
            const int nitem = kn * PP * nb0 * nb1;
            for (int it = tid; it < nitem; it += nth) {
                int r = it;
                const int kk = r % kn; r /= kn;
                const int a1 = r % P1; r /= P1;
                const int a2 = r % P1; r /= P1;
                const int b1 = r % nb0; const int b2 = r / nb0;
                TS h2[3][NG];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const TS* Ty = T2 + (j == 1 ? NG * TW : 0) + a2 * nb1 + b2;
                    const TS* h = H1 + (size_t)j * G2 * PB * kn + (b1 * P1 + a1) * kn + kk;
#pragma unroll
                    for (int g3 = 0; g3 < NG; ++g3) {
                        TS s = 0;
#pragma unroll
                        for (int g2 = 0; g2 < NG; ++g2) s += Ty[g2 * TW] * h[(size_t)(g2 + NG * g3) * PB * kn];
                        h2[j][g3] = s;
                    }
                }
                const int k = k0 + kk;
                // S row (A, k) with A = (eo0 + a1) + n (eo1 + a2) + n^2 (eo2 + a3); column (B, l) with
                // B = B1 + n B2 + n^2 B3, B3 = b3 on the line direction d = 2, else eo2 + b3
                const int B1 = d == 0 ? b1 : eo[0] + b1, B2 = d == 1 ? b2 : eo[1] + b2;
                TS* Sb = S + (size_t)(((eo[0] + a1) + n * (eo[1] + a2) + n * n * eo[2]) * 5 + k) +
                         (size_t)((B1 + n * (B2 + n * (d == 2 ? 0 : eo[2]))) * 5 + l) * ld;
#pragma unroll 1
                for (int a3 = 0; a3 < P1; ++a3)
                    for (int b30 = 0; b30 < nb2; b30 += 4) {
                        TS acc[4] = {0, 0, 0, 0};
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const TS* Tz = T3 + (j == 2 ? NG * TW : 0) + a3 * nb2 + b30;
#pragma unroll
                            for (int g3 = 0; g3 < NG; ++g3) {
                                const TS hv = h2[j][g3];
                                const TS* row = Tz + g3 * TW;
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    if (b30 + q < nb2) acc[q] += row[q] * hv;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (b30 + q < nb2) atomic_add_t(Sb + a3 * sa + (b30 + q) * sb, (double)acc[q]);
                    }
            }
            __syncthreads();
        }
}

// Q-elimination term of S = A_vv - A_vq A_qq^-1 A_qv (eq. R3).  A_qq = I x M
// with M a tensor product of 1-D mass matrices, so C = A_qq^-1 A_qv acts on
// the q-component (l, d) along the d-lines only: C = (2/h_d) C1_ref (x) I.
// Composed with the interpolation of q, the q-trial function of direction d
// is again a tensor product: the micro-element basis in the two other
// directions and, along d,
//   chi_b(x_d) = sum_c phi_c(x_d) (2/h_d) C1_ref[c][b]
// for every node b of the macro-element's d-line (n of them).  So
//   S[(a,k),(b,l)] += sum_x W sum_j dG_kj/dq_ld d_j phi_a  psi_{b,d}
// is sum-factorised like A_vv, with n instead of p+1 trial functions along d:
// stage 1 contracts g1 into H1[j][g2 g3][b1][a1][k]; items (k, a1, a2, b1, b2)
// contract g2 into registers and g3 for every (a3, b3).  Items run k fastest,
// then a1, so a warp's atomics fall on runs of consecutive rows 5 A + k and its
// reads of H1 on consecutive words.
// The five test components k are processed kg at a time (kg = 5 unless the
// stage-1 buffer would not fit in shared memory).
// Point pass of the Q-elimination term: dG/dq at every Gauss point of one
// micro-element from one 15-direction dual evaluation (G is linear in q),
// stored weighted and point-fastest: a.pq[K][e][d*75 + j*25 + k*5 + l][npt] =
// W dG_kj/dq_ld.
__global__ void __launch_bounds__(128)
jac_visc_q_points_kernel(JacobianArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int eo[3] = {(e % m) * p, ((e / m) % m) * p, (e / (m * m)) * p};
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* vl = sW + 8;                                     // [5][nl]
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    double sc[3], hw[3];
    geometry(a, K, sc, hw);
    const int64_t oV = (int64_t)K * 5 * Nn;
    for (int i = tid; i < nl; i += nth) {
        int A = (eo[0] + i % p1) + n * ((eo[1] + (i / p1) % p1) + n * (eo[2] + i / (p1 * p1)));
        for (int k = 0; k < 5; ++k) vl[k * nl + i] = a.v[oV + k * Nn + A];
    }
    __syncthreads();
    double* Gb = a.pq + ((size_t)K * m * m * m + e) * 225 * npt;
    for (int x = tid; x < npt; x += nth) {
        const int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
        Dual<15> v15[5], q15[15], G[5][3];
        for (int k = 0; k < 5; ++k) {
            double s5 = 0.0;
            for (int i = 0; i < nl; ++i)
                s5 += sL[g1 * p1 + i % p1] * sL[g2 * p1 + (i / p1) % p1] * sL[g3 * p1 + i / (p1 * p1)] * vl[k * nl + i];
            v15[k] = mkdual<15>(s5);
        }
        for (int c = 0; c < 15; ++c) { q15[c] = mkdual<15>(0.0); q15[c].d[c] = 1.0; }
        visc_flux(v15, q15, a.ph, G);
        const double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 5; ++k)
                    for (int l = 0; l < 5; ++l)
                        Gb[(size_t)(d * 75 + j * 25 + k * 5 + l) * npt + x] = W * G[k][j].d[l * 3 + d];
    }
}

// PRE: the point blocks come from a.pq (jac_visc_q_points_kernel) instead of
// three dual evaluations per point here
template <class TS, bool PRE = false>
__global__ void __launch_bounds__(256, PRE ? 2 : 1)
jac_visc_q_volume_kernel(JacobianArgs a, const double* __restrict__ C1, int kg) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int TW = p1 * n;
    const int eo[3] = {(e % m) * p, ((e / m) % m) * p, (e / (m * m)) * p};
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* C1s = sW + 8;                                    // [n][n]
    double* vl = C1s + n * n;                                // [5][nl]
    double* vx = vl + 5 * nl;                                // [npt][5]
    TS* T = reinterpret_cast<TS*>(vx + 5 * npt);             // [3 dir][2 tau][ng][TW]
    TS* P = T + 6 * ng * TW;                                 // [npt][3 j][25 kl]
    // H1[j][g23][b1][a1][kk] (kk < kn <= kg), so that the lanes of a warp (kk
    // fastest, then a1) read consecutive words in stage 2
    TS* H1 = P + (size_t)npt * 75;
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    double sc[3], hw[3];
    geometry(a, K, sc, hw);
    for (int i = tid; i < n * n; i += nth) C1s[i] = C1[i];
    const int64_t oV = (int64_t)K * 5 * Nn;
    if constexpr (!PRE) {
        for (int i = tid; i < nl; i += nth) {
            int A = (eo[0] + i % p1) + n * ((eo[1] + (i / p1) % p1) + n * (eo[2] + i / (p1 * p1)));
            for (int k = 0; k < 5; ++k) vl[k * nl + i] = a.v[oV + k * Nn + A];
        }
        __syncthreads();
        for (int x = tid; x < npt; x += nth) {
            int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
            double s5[5] = {0, 0, 0, 0, 0};
            for (int i = 0; i < nl; ++i) {
                double f = sL[g1 * p1 + i % p1] * sL[g2 * p1 + (i / p1) % p1] * sL[g3 * p1 + i / (p1 * p1)];
                for (int k = 0; k < 5; ++k) s5[k] += f * vl[k * nl + i];
            }
            for (int k = 0; k < 5; ++k) vx[x * 5 + k] = s5[k];
        }
    }
    __syncthreads();
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    for (int d = 0; d < 3; ++d) {
        int nb[3];
        for (int q = 0; q < 3; ++q) nb[q] = q == d ? n : p1;
        // tables T[dir][tau][g][a * nb + b]: (tau ? dphi_a : phi_a)(g) times phi_b(g),
        // or chi_b(g) along the line direction d
        for (int i = tid; i < 6 * ng * TW; i += nth) {
            const int col = i % TW, g = (i / TW) % ng, dt = i / (TW * ng), dir = dt >> 1, tau = dt & 1;
            const int w = nb[dir];
            TS val = 0;
            if (col < p1 * w) {
                const int aa = col / w, bb = col % w;
                const double t = tau ? sD[g * p1 + aa] * sc[dir] : sL[g * p1 + aa];
                double trial;
                if (dir == d) {
                    trial = 0.0;
                    for (int c = 0; c < p1; ++c) trial += sL[g * p1 + c] * C1s[(eo[d] + c) * n + bb];
                    trial *= sc[d];
                } else {
                    trial = sL[g * p1 + bb];
                }
                val = (TS)(t * trial);
            }
            T[i] = val;
        }
        // point blocks P[x][j][k*5+l] = W dG_kj/dq_ld (G is linear in q)
        if constexpr (PRE) {
            const double* Gb = a.pq + ((size_t)K * m * m * m + e) * 225 * npt + (size_t)d * 75 * npt;
            for (int i = tid; i < 75 * npt; i += nth) P[(size_t)(i % npt) * 75 + i / npt] = (TS)Gb[i];
        } else
        for (int x = tid; x < npt; x += nth) {
            int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
            Dual<15> v15[5], q15[15], G[5][3];
            for (int k = 0; k < 5; ++k) v15[k] = mkdual<15>(vx[x * 5 + k]);
            for (int c = 0; c < 15; ++c) { q15[c] = mkdual<15>(0.0); q15[c].d[c] = 1.0; }
            visc_flux(v15, q15, a.ph, G);
            double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
            TS* Px = P + (size_t)x * 75;
            double* Gq = a.pq ? a.pq + ((size_t)K * m * m * m + e) * 225 * npt + (size_t)d * 75 * npt + x : nullptr;
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 5; ++k)
                    for (int l = 0; l < 5; ++l) {
                        const double gv = W * G[k][j].d[l * 3 + d];
                        Px[25 * j + k * 5 + l] = (TS)gv;
                        if (Gq) Gq[(size_t)(25 * j + k * 5 + l) * npt] = gv;   // also kept for the tangents
                    }
        }
        __syncthreads();
        switch (p1) {
        case 2: q_contract<2, TS>(T, P, H1, S, a.ld, n, eo, d, kg); break;
        case 3: q_contract<3, TS>(T, P, H1, S, a.ld, n, eo, d, kg); break;
        case 4: q_contract<4, TS>(T, P, H1, S, a.ld, n, eo, d, kg); break;
        default: q_contract<5, TS>(T, P, H1, S, a.ld, n, eo, d, kg); break;   // p = MEHDG_MAXP
        }
    }
}

// face part of -A_vq C: G-hat = G(vhat, q).n depends on the interior q at the
// face points, with the same q-trial functions restricted to the face: along
// the normal direction (d = face direction) chi_b at the face end is the
// constant (2/h) C1_ref[end][b]; along a tangential direction it is chi_b of
// that direction.  Per face and q-direction d: stage 1 contracts g1 into
// H1[g2][b1][a1][k] (a warp's lanes, k fastest and then a1, read consecutive
// words), items (k, a1, a2, b1, b2) contract g2 and add the result (times the
// normal factor for every b on the normal line when d is normal).
template <class TS>
__global__ void __launch_bounds__(256)
jac_visc_q_face_kernel(JacobianArgs a, const double* __restrict__ C1) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, n2 = tb.n2, p1 = p + 1;
    const int f = blockIdx.x / (m * m), e = blockIdx.x % (m * m);
    const int e1 = e % m, e2 = e / m;
    const int df = f / 2, t1 = df == 0 ? 1 : 0, t2 = df == 2 ? 1 : 2;
    const double sgn = (f & 1) ? 1.0 : -1.0;
    const int iface = (f & 1) ? n - 1 : 0;
    const int fl = p1 * p1, fpt = ng * ng, TW = p1 * n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sW = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* C1s = sW + 8;             // [n][n]
    double* fh = C1s + n * n;         // [5][fl]
    TS* PF = reinterpret_cast<TS*>(fh + 5 * fl);   // [fpt][3 d][25 kl]
    TS* T = PF + (size_t)fpt * 75;                  // [2 tangential][ng][TW]
    TS* H1 = T + 2 * ng * TW;                       // [ng][nb1][p1][5] (at most 5 TW ng)
    TS* cn = H1 + 5 * TW * ng;                      // [n] normal factors
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    if (tid < ng) sW[tid] = tb.w[tid];
    for (int i = tid; i < n * n; i += nth) C1s[i] = C1[i];
    const double* box = a.box + 6 * K;
    double h[3];
    for (int d = 0; d < 3; ++d) h[d] = (box[3 + d] - box[d]) / m;
    const double hw1 = 0.5 * h[t1], hw2 = 0.5 * h[t2];
    const int64_t og = a.gid[6 * K + f] * 5 * n2;
    for (int i = tid; i < fl; i += nth) {
        int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        for (int k = 0; k < 5; ++k) fh[k * fl + i] = a.vh[og + k * n2 + c1 + n * c2];
    }
    __syncthreads();
    for (int x = tid; x < fpt; x += nth) {
        int g1 = x % ng, g2 = x / ng;
        Dual<15> v15[5], q15[15], G[5][3];
        for (int k = 0; k < 5; ++k) {
            double s = 0.0;
            for (int i = 0; i < fl; ++i) s += sL[g1 * p1 + i % p1] * sL[g2 * p1 + i / p1] * fh[k * fl + i];
            v15[k] = mkdual<15>(s);
        }
        for (int c = 0; c < 15; ++c) { q15[c] = mkdual<15>(0.0); q15[c].d[c] = 1.0; }
        visc_flux(v15, q15, a.ph, G);
        const double W = sW[g1] * hw1 * sW[g2] * hw2 * sgn;
        double* Gq = a.pqf ? a.pqf + ((size_t)K * 6 * m * m + blockIdx.x) * 75 * fpt + x : nullptr;
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < 5; ++k)
                for (int l = 0; l < 5; ++l) {
                    const double gv = W * G[k][df].d[l * 3 + d];
                    PF[(size_t)x * 75 + d * 25 + k * 5 + l] = (TS)gv;
                    if (Gq) Gq[(size_t)(d * 25 + k * 5 + l) * fpt] = gv;   // also kept for the tangents
                }
    }
    TS* S = reinterpret_cast<TS*>(a.S) + (size_t)K * a.ld * a.ld;
    const int eo1 = e1 * p, eo2 = e2 * p;
    for (int d = 0; d < 3; ++d) {
        const int nb1 = d == t1 ? n : p1, nb2 = d == t2 ? n : p1, nn = d == df ? n : 1;
        __syncthreads();
        // tables T[u][g][a * nb_u + b] for the tangential directions u = t1, t2
        for (int i = tid; i < 2 * ng * TW; i += nth) {
            const int col = i % TW, g = (i / TW) % ng, u = i / (TW * ng);
            const int dir = u == 0 ? t1 : t2, w = u == 0 ? nb1 : nb2, eo = u == 0 ? eo1 : eo2;
            TS val = 0;
            if (col < p1 * w) {
                const int aa = col / w, bb = col % w;
                double trial;
                if (dir == d) {
                    trial = 0.0;
                    for (int c = 0; c < p1; ++c) trial += sL[g * p1 + c] * C1s[(eo + c) * n + bb];
                    trial *= 2.0 / h[d];
                } else {
                    trial = sL[g * p1 + bb];
                }
                val = (TS)(sL[g * p1 + aa] * trial);
            }
            T[i] = val;
        }
        for (int i = tid; i < n; i += nth) cn[i] = d == df ? (TS)(C1s[iface * n + i] * 2.0 / h[d]) : (TS)1;
        __syncthreads();
        for (int l = 0; l < 5; ++l) {
            for (int i = tid; i < 5 * p1 * nb1 * ng; i += nth) {
                const int k = i % 5, a1 = (i / 5) % p1, b1 = (i / (5 * p1)) % nb1, g2 = i / (5 * p1 * nb1);
                const int ab1 = a1 * nb1 + b1;
                TS s = 0;
                for (int g1 = 0; g1 < ng; ++g1)
                    s += T[g1 * TW + ab1] * PF[(size_t)(g1 + ng * g2) * 75 + d * 25 + k * 5 + l];
                H1[i] = s;
            }
            __syncthreads();
            const int nitem = 5 * p1 * p1 * nb1 * nb2;
            for (int it = tid; it < nitem; it += nth) {
                int r = it;
                const int k = r % 5; r /= 5;
                const int a1 = r % p1; r /= p1;
                const int a2 = r % p1; r /= p1;
                const int b1 = r % nb1; const int b2 = r / nb1;
                const TS* hk = H1 + (b1 * p1 + a1) * 5 + k;
                const TS* Ty = T + ng * TW + a2 * nb2 + b2;
                TS s = 0;
                for (int g2 = 0; g2 < ng; ++g2) s += Ty[g2 * TW] * hk[(size_t)g2 * 5 * p1 * nb1];
                int ca[3], cb[3];
                ca[df] = iface; ca[t1] = eo1 + a1; ca[t2] = eo2 + a2;
                cb[df] = iface; cb[t1] = d == t1 ? b1 : eo1 + b1; cb[t2] = d == t2 ? b2 : eo2 + b2;
                const int A = ca[0] + n * (ca[1] + n * ca[2]);
                for (int bd = 0; bd < nn; ++bd) {
                    if (d == df) cb[df] = bd;
                    const int B = cb[0] + n * (cb[1] + n * cb[2]);
                    atomic_add_t(&S[(size_t)(A * 5 + k) + (size_t)(B * 5 + l) * a.ld], -(double)(s * cn[bd]));
                }
            }
            __syncthreads();
        }
    }
}

template <class TS>
__global__ void pad_identity_kernel(TS* S, int64_t ld, int Nv) {
    int K = blockIdx.y;
    int64_t i = Nv + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ld) S[(size_t)K * ld * ld + i + i * ld] = (TS)1;
}

size_t sf_smem_bytes(const Tab& t, bool visc, size_t ts) {
    const size_t PP = (size_t)(t.p + 1) * (t.p + 1), G2 = (size_t)t.ng * t.ng;
    size_t head = sizeof(double) * HEAD_DOUBLES;
    size_t tables = ts * 6 * MEHDG_MAXG * (MEHDG_MAXP + 1) * (MEHDG_MAXP + 1);
    size_t P = ts * 100 * (size_t)t.npt;
    size_t state = sizeof(double) * (size_t)(10 + (visc ? 15 : 0)) * t.nl;
    size_t hbuf = ts * 5 * 4 * PP * G2;
    return head + tables + P + (state > hbuf ? state : hbuf) + 16;
}

}  // namespace

cudaError_t launch_jacobian(const JacobianArgs& a, int64_t nK, bool fp64, cudaStream_t st, int phase) {
    const Tab& t = a.tab;
    bool visc = a.ph.viscous != 0;
    size_t ts = fp64 ? 8 : 4;
    size_t ssf = sf_smem_bytes(t, visc, ts);
    const bool use_sf = ssf <= 220 * 1024;
    size_t sv = use_sf ? ssf
                       : sizeof(double) * (HEAD_DOUBLES + (size_t)(10 + (visc ? 15 : 0)) * t.nl)
                             + ts * 100 * (size_t)t.npt;
    int fl = (t.p + 1) * (t.p + 1), fpt = t.ng * t.ng;
    size_t sf = sizeof(double) * (MEHDG_MAXG * (MEHDG_MAXP + 1) + 8 + 25 * (size_t)fl + (fl + 1) / 2 + 1)
              + ts * 25 * (size_t)fpt + 64;
    dim3 gv(t.m * t.m * t.m, (unsigned)nK), gf(6 * t.m * t.m, (unsigned)nK), b(256);
    // split face pass: the point pass stages the macro-face's nodal values, the contraction its blocks
    const size_t sfp = sizeof(double) * (MEHDG_MAXG * (MEHDG_MAXP + 1) + 8 + (size_t)(10 + (visc ? 15 : 0)) * t.n2);
    const size_t sfc = sizeof(double) * (MEHDG_MAXG * (MEHDG_MAXP + 1) + (fl + 1) / 2 + 1) + ts * 25 * (size_t)fpt + 64;
    // phase 1: the point passes (they write the stored point Jacobians, not S);
    // phase 2: everything that adds into S
#define LJ(TS, V)                                                                                        \
    do { if (use_sf && !V && a.pj) {                                                                     \
             if (phase & 1) {                                                                            \
                 const size_t sp = sizeof(double) * (HEAD_DOUBLES + 10 * (size_t)t.nl) + 16;             \
                 cudaFuncSetAttribute(jac_points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp); \
                 jac_points_kernel<<<gv, 128, sp, st>>>(a);                                              \
                 MEHDG_COUNT(1);                                                                         \
             }                                                                                           \
             if (phase & 2) {                                                                            \
                 cudaFuncSetAttribute(jac_volume_sf_kernel<TS, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv); \
                 jac_volume_sf_kernel<TS, V, true><<<gv, b, sv, st>>>(a);                                \
                 MEHDG_COUNT(1);                                                                         \
             }                                                                                           \
         } else if (phase & 2) {                                                                         \
             if (use_sf) {                                                                               \
                 cudaFuncSetAttribute(jac_volume_sf_kernel<TS, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv); \
                 jac_volume_sf_kernel<TS, V><<<gv, b, sv, st>>>(a);                                      \
             } else {                                                                                    \
                 cudaFuncSetAttribute(jac_volume_kernel<TS, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv); \
                 jac_volume_kernel<TS, V><<<gv, b, sv, st>>>(a);                                         \
             }                                                                                           \
             MEHDG_COUNT(1);                                                                             \
         }                                                                                               \
         if (a.pjf) {                                                                                    \
             if (phase & 1) {                                                                            \
                 cudaFuncSetAttribute(jac_face_points_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sfp); \
                 jac_face_points_kernel<V><<<dim3(6, (unsigned)nK), b, sfp, st>>>(a);                    \
                 MEHDG_COUNT(1);                                                                         \
             }                                                                                           \
             if (phase & 2) {                                                                            \
                 cudaFuncSetAttribute(jac_face_contract_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sfc); \
                 jac_face_contract_kernel<TS><<<gf, b, sfc, st>>>(a);                                    \
                 MEHDG_COUNT(1);                                                                         \
             }                                                                                           \
         } else if (phase & 2) {                                                                         \
             cudaFuncSetAttribute(jac_face_kernel<TS, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf); \
             jac_face_kernel<TS, V><<<gf, b, sf, st>>>(a);                                               \
             MEHDG_COUNT(1);                                                                             \
         } } while (0)
    if (fp64) { if (visc) LJ(double, true); else LJ(double, false); }
    else { if (visc) LJ(float, true); else LJ(float, false); }
#undef LJ
    if (visc) {
        const size_t G2 = (size_t)t.ng * t.ng, TW = (size_t)(t.p + 1) * t.n;
        const size_t base = sizeof(double) * (HEAD_DOUBLES + (size_t)t.n * t.n + 5 * (size_t)t.nl + 5 * (size_t)t.npt)
                          + ts * (6 * (size_t)t.ng * TW + 75 * (size_t)t.npt) + 16;
        // with the point pass separate (a.pq) the contraction runs two CTAs per SM
        // if its shared memory fits in half an SM's; otherwise one, with the
        // largest k group that fits
        const size_t per_k = ts * 3 * TW * G2;
        const bool pre = a.pq && base + per_k <= 110 * 1024;
        const size_t limit = pre ? 110 * 1024 : 220 * 1024;
        int kg = 5;
        while (kg > 1 && base + (size_t)kg * per_k > limit) --kg;
        const size_t sq = base + (size_t)kg * per_k;
        size_t sqf = sizeof(double) * (MEHDG_MAXG * (MEHDG_MAXP + 1) + 8 + (size_t)t.n * t.n + 5 * (size_t)fl)
                   + ts * (75 * (size_t)fpt + 2 * (size_t)t.ng * TW + 5 * TW * t.ng + t.n) + 16;
        if (sq > 227 * 1024) return cudaErrorInvalidValue;      // FP64 at p = 4: not supported
#define LQ(TS)                                                                                          \
        do { if (pre) {                                                                                 \
                 if (phase & 1) {                                                                       \
                     const size_t sp = sizeof(double) * (HEAD_DOUBLES + 5 * (size_t)t.nl) + 16;         \
                     jac_visc_q_points_kernel<<<gv, 128, sp, st>>>(a);                                  \
                     MEHDG_COUNT(1);                                                                    \
                 }                                                                                      \
                 if (phase & 2) {                                                                       \
                     cudaFuncSetAttribute(jac_visc_q_volume_kernel<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sq); \
                     jac_visc_q_volume_kernel<TS, true><<<gv, b, sq, st>>>(a, a.C1, kg);                \
                     MEHDG_COUNT(1);                                                                    \
                 }                                                                                      \
             } else if (phase & 2) {                                                                    \
                 cudaFuncSetAttribute(jac_visc_q_volume_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sq); \
                 jac_visc_q_volume_kernel<TS><<<gv, b, sq, st>>>(a, a.C1, kg);                          \
                 MEHDG_COUNT(1);                                                                        \
             }                                                                                          \
             if (phase & 2) {                                                                           \
                 cudaFuncSetAttribute(jac_visc_q_face_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sqf); \
                 jac_visc_q_face_kernel<TS><<<gf, b, sqf, st>>>(a, a.C1);                               \
                 MEHDG_COUNT(1);                                                                        \
             } } while (0)
        if (fp64) LQ(double); else LQ(float);
#undef LQ
    }
    return cudaGetLastError();
}

cudaError_t launch_pad_identity(void* S, int64_t nK, int64_t ld, int Nv, bool fp64, cudaStream_t st) {
    int64_t np = ld - Nv;
    if (np <= 0) return cudaSuccess;
    dim3 g((unsigned)((np + 127) / 128), (unsigned)nK);
    if (fp64) pad_identity_kernel<double><<<g, 128, 0, st>>>((double*)S, ld, Nv);
    else pad_identity_kernel<float><<<g, 128, 0, st>>>((float*)S, ld, Nv);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}
