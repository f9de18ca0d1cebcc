// vjp.cu -- vector-Jacobian product of the residual of eq. s32 (Euler):
//   g_v    = (dR_V/dv)^T lam_V    + (dR_Vhat/dv)^T lam_Vhat
//   g_vhat = (dR_V/dvhat)^T lam_V + (dR_Vhat/dvhat)^T lam_Vhat
// for cotangents lam_V [nK][5][Nn] and lam_Vhat [G][5][n^2] (the global trace
// residual, summed over both sides of every face).  Nothing is stored between
// the forward residual and this pass: the quadrature-point states are
// recomputed from the nodal state, and the point Jacobians come from
// forward-mode duals at each point (5 directions in the volume, 10 at the
// faces: v and vhat).
//
// Volume, per micro-element: with R_V[k,A] = sum_x W (U_k phi_A - sum_j FG_kj
// d_j phi_A), the cotangent is carried to the Gauss points through the test
// functions, Lam0_k = sum_A lam[k,A] phi_A and Lamj_k = sum_A lam[k,A] d_j phi_A,
// multiplied by the point Jacobians, and tested against phi_B:
//   g_v[l,B] += sum_x phi_B W (sum_k Lam0_k dU_k/dv_l - sum_kj Lamj_k dFG_kj/dv_l).
// Faces: R_V and R_Vhat take the same flux W Fhat_k at each face point, so the
// point cotangent is W (Lam_k + Lamhat_k) and it multiplies dFhat/dv (tested
// with the element's face nodes) and dFhat/dvhat (tested with the trace nodes).
#include "physics.cuh"
#include "kernels.cuh"

namespace {

struct VjpArgs {
    Tab tab;
    Phys ph;
    const double* box;
    const int64_t* gid;
    const double *v, *vs, *vh;
    const double *lamV, *lamH;
    double *gv, *gh;
    int32_t* status;
};

__device__ __forceinline__ void load_tables(const Tab& tb, double* sL, double* sD, double* sW) {
    const int p1 = tb.p + 1;
    for (int i = threadIdx.x; i < tb.ng * p1; i += blockDim.x) { sL[i] = tb.L[i / p1][i % p1]; sD[i] = tb.dL[i / p1][i % p1]; }
    if (threadIdx.x < tb.ng) sW[threadIdx.x] = tb.w[threadIdx.x];
}

__global__ void __launch_bounds__(128) vjp_volume_kernel(VjpArgs a) {
    const Tab& tb = a.tab;
    const int K = blockIdx.y, e = blockIdx.x;
    const int p = tb.p, m = tb.m, n = tb.n, ng = tb.ng, Nn = tb.Nn, nl = tb.nl, npt = tb.npt, p1 = p + 1;
    const int e1 = e % m, e2 = (e / m) % m, e3 = e / (m * m);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sL = reinterpret_cast<double*>(smem_raw);
    double* sD = sL + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* sW = sD + MEHDG_MAXG * (MEHDG_MAXP + 1);
    double* vl = sW + 8;              // [5][nl]
    double* vsl = vl + 5 * nl;        // [5][nl]
    double* ll = vsl + 5 * nl;        // [5][nl] cotangent at the nodes
    double* mu = ll + 5 * nl;         // [5][npt] point cotangent of v
    const int tid = threadIdx.x, nth = blockDim.x;
    load_tables(tb, sL, sD, sW);
    const double* box = a.box + 6 * K;
    double sc[3], hw[3];
    for (int d = 0; d < 3; ++d) { double h = (box[3 + d] - box[d]) / m; sc[d] = 2.0 / h; hw[d] = 0.5 * h; }
    const int64_t oV = (int64_t)K * 5 * Nn;
    for (int i = tid; i < nl; i += nth) {
        const int A = (e1 * p + i % p1) + n * ((e2 * p + (i / p1) % p1) + n * (e3 * p + i / (p1 * p1)));
        for (int k = 0; k < 5; ++k) {
            vl[k * nl + i] = a.v[oV + k * Nn + A];
            vsl[k * nl + i] = a.ph.time_term ? a.vs[oV + k * Nn + A] : 0.0;
            ll[k * nl + i] = a.lamV ? a.lamV[oV + k * Nn + A] : 0.0;
        }
    }
    __syncthreads();
    bool ok = true;
    for (int x = tid; x < npt; x += nth) {
        const int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
        double vx[5] = {0, 0, 0, 0, 0}, vsx[5] = {0, 0, 0, 0, 0}, L0[5] = {0, 0, 0, 0, 0}, Lj[3][5] = {};
        for (int i = 0; i < nl; ++i) {
            const int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
            const double a1 = sL[g1 * p1 + l1], a2 = sL[g2 * p1 + l2], a3 = sL[g3 * p1 + l3];
            const double f = a1 * a2 * a3;
            const double d1 = sD[g1 * p1 + l1] * sc[0] * a2 * a3, d2 = a1 * sD[g2 * p1 + l2] * sc[1] * a3,
                         d3 = a1 * a2 * sD[g3 * p1 + l3] * sc[2];
            for (int k = 0; k < 5; ++k) {
                vx[k] += vl[k * nl + i] * f;
                vsx[k] += vsl[k * nl + i] * f;
                const double lk = ll[k * nl + i];
                L0[k] += lk * f; Lj[0][k] += lk * d1; Lj[1][k] += lk * d2; Lj[2][k] += lk * d3;
            }
        }
        Dual<5> dv[5], dvs[5], dq[15], U[5], FG[5][3];
        for (int k = 0; k < 5; ++k) { dv[k] = mkdual<5>(vx[k]); dv[k].d[k] = 1.0; dvs[k] = mkdual<5>(vsx[k]); }
        for (int c = 0; c < 15; ++c) dq[c] = mkdual<5>(0.0);
        ok = vol_integrand(a.ph, dv, dvs, dq, U, FG) && ok;
        const double W = sW[g1] * hw[0] * sW[g2] * hw[1] * sW[g3] * hw[2];
        for (int l = 0; l < 5; ++l) {
            double s = 0.0;
            for (int k = 0; k < 5; ++k) {
                s += L0[k] * U[k].d[l];
                for (int j = 0; j < 3; ++j) s -= Lj[j][k] * FG[k][j].d[l];
            }
            mu[l * npt + x] = W * s;
        }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
    for (int r = tid; r < 5 * nl; r += nth) {
        const int i = r % nl, l = r / nl;
        const int l1 = i % p1, l2 = (i / p1) % p1, l3 = i / (p1 * p1);
        double s = 0.0;
        for (int x = 0; x < npt; ++x) {
            const int g1 = x % ng, g2 = (x / ng) % ng, g3 = x / (ng * ng);
            s += mu[l * npt + x] * sL[g1 * p1 + l1] * sL[g2 * p1 + l2] * sL[g3 * p1 + l3];
        }
        const int A = (e1 * p + l1) + n * ((e2 * p + l2) + n * (e3 * p + l3));
        atomicAdd(a.gv + oV + l * Nn + A, s);
    }
}

__global__ void __launch_bounds__(128) vjp_face_kernel(VjpArgs a) {
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
    double* fv = sW + 8;              // [5][fl] element state on the face
    double* fh = fv + 5 * fl;         // [5][fl] trace
    double* lv = fh + 5 * fl;         // [5][fl] lam_V on the face nodes
    double* lh = lv + 5 * fl;         // [5][fl] lam_Vhat on the trace nodes
    double* gvx = lh + 5 * fl;        // [5][fpt]
    double* ghx = gvx + 5 * fpt;      // [5][fpt]
    int* nodeA = reinterpret_cast<int*>(ghx + 5 * fpt);
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < ng * p1; i += nth) sL[i] = tb.L[i / p1][i % p1];
    if (tid < ng) sW[tid] = tb.w[tid];
    const double* box = a.box + 6 * K;
    const double hw1 = 0.5 * (box[3 + t1] - box[t1]) / m, hw2 = 0.5 * (box[3 + t2] - box[t2]) / m;
    const int64_t oV = (int64_t)K * 5 * Nn, og = a.gid[6 * K + f] * 5 * n2;
    for (int i = tid; i < fl; i += nth) {
        const int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        int idx[3]; idx[d] = (f & 1) ? n - 1 : 0; idx[t1] = c1; idx[t2] = c2;
        const int A = idx[0] + n * (idx[1] + n * idx[2]);
        nodeA[i] = A;
        for (int k = 0; k < 5; ++k) {
            fv[k * fl + i] = a.v[oV + k * Nn + A];
            fh[k * fl + i] = a.vh[og + k * n2 + c1 + n * c2];
            lv[k * fl + i] = a.lamV ? a.lamV[oV + k * Nn + A] : 0.0;
            lh[k * fl + i] = a.lamH ? a.lamH[og + k * n2 + c1 + n * c2] : 0.0;
        }
    }
    __syncthreads();
    bool ok = true;
    for (int x = tid; x < fpt; x += nth) {
        const int g1 = x % ng, g2 = x / ng;
        double vx[5] = {0, 0, 0, 0, 0}, hx[5] = {0, 0, 0, 0, 0}, nu[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < fl; ++i) {
            const double mw = sL[g1 * p1 + i % p1] * sL[g2 * p1 + i / p1];
            for (int k = 0; k < 5; ++k) {
                vx[k] += fv[k * fl + i] * mw;
                hx[k] += fh[k * fl + i] * mw;
                nu[k] += (lv[k * fl + i] + lh[k * fl + i]) * mw;
            }
        }
        Dual<10> dv[5], dh[5], dq[15], Fh[5];
        for (int k = 0; k < 5; ++k) {
            dv[k] = mkdual<10>(vx[k]); dv[k].d[k] = 1.0;
            dh[k] = mkdual<10>(hx[k]); dh[k].d[5 + k] = 1.0;
        }
        for (int c = 0; c < 15; ++c) dq[c] = mkdual<10>(0.0);
        ok = face_integrand(a.ph, dv, dh, dq, d, sgn, Fh) && ok;
        const double W = sW[g1] * hw1 * sW[g2] * hw2;
        for (int l = 0; l < 5; ++l) {
            double sv = 0.0, sh = 0.0;
            for (int k = 0; k < 5; ++k) { sv += nu[k] * Fh[k].d[l]; sh += nu[k] * Fh[k].d[5 + l]; }
            gvx[l * fpt + x] = W * sv;
            ghx[l * fpt + x] = W * sh;
        }
    }
    if (!ok && a.status) a.status[K] = MEHDG_ENONPHYS;
    __syncthreads();
    for (int r = tid; r < 5 * fl; r += nth) {
        const int i = r % fl, l = r / fl;
        double sv = 0.0, sh = 0.0;
        for (int x = 0; x < fpt; ++x) {
            const double mw = sL[(x % ng) * p1 + i % p1] * sL[(x / ng) * p1 + i / p1];
            sv += gvx[l * fpt + x] * mw;
            sh += ghx[l * fpt + x] * mw;
        }
        const int c1 = e1 * p + i % p1, c2 = e2 * p + i / p1;
        atomicAdd(a.gv + oV + l * Nn + nodeA[i], sv);
        atomicAdd(a.gh + og + l * n2 + c1 + n * c2, sh);
    }
}

}  // namespace

// the two VJP passes at the context's state (no status reset, no checks):
// g_v, g_vhat overwritten
cudaError_t launch_vjp(mehdg_ctx* c, const double* lam_V, const double* lam_Vhat, double* g_v, double* g_vhat,
                       cudaStream_t st) {
    const Tab& t = c->tab;
    VjpArgs a;
    a.tab = t; a.ph = c->ph; a.box = c->d_box; a.gid = c->d_gid;
    a.v = c->v; a.vs = c->vs; a.vh = c->vh; a.lamV = lam_V; a.lamH = lam_Vhat; a.gv = g_v; a.gh = g_vhat;
    a.status = c->d_status;
    cudaError_t e;
    if ((e = cudaMemsetAsync(g_v, 0, sizeof(double) * c->nK * 5 * t.Nn, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(g_vhat, 0, sizeof(double) * c->G * 5 * t.n2, st)) != cudaSuccess)
        return e;
    const size_t head = sizeof(double) * (2 * MEHDG_MAXG * (MEHDG_MAXP + 1) + 8);
    const size_t sv = head + sizeof(double) * (15 * (size_t)t.nl + 5 * (size_t)t.npt);
    const int fl = (t.p + 1) * (t.p + 1), fpt = t.ng * t.ng;
    const size_t sf = head + sizeof(double) * (20 * (size_t)fl + 10 * (size_t)fpt) + sizeof(int) * fl + 16;
    cudaFuncSetAttribute(vjp_volume_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv);
    cudaFuncSetAttribute(vjp_face_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
    vjp_volume_kernel<<<dim3((unsigned)(t.m * t.m * t.m), (unsigned)c->nK), 128, sv, st>>>(a);
    vjp_face_kernel<<<dim3((unsigned)(6 * t.m * t.m), (unsigned)c->nK), 128, sf, st>>>(a);
    MEHDG_COUNT(2);
    return cudaGetLastError();
}

extern "C" int mehdg_residual_vjp(mehdg_ctx* c, const double* lam_V, const double* lam_Vhat, double* g_v,
                                  double* g_vhat, void* stream) {
    if (c && c->batch) { set_err(c, "residual_vjp: not available for elements of uneven p, m"); return MEHDG_EINVAL; }
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0 || !c->v || !c->vh) { set_err(c, "residual_vjp before set_mesh/set_state"); return MEHDG_ESTATE; }
    if (c->ph.viscous) { set_err(c, "residual_vjp: the Euler residual only"); return MEHDG_EINVAL; }
    if (!lam_V || !g_v || !g_vhat) return MEHDG_EINVAL;
    if (c->ph.time_term && !c->vs) { set_err(c, "residual_vjp: the time term needs vstar"); return MEHDG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * c->nK, st) != cudaSuccess) {
        set_err(c, "residual_vjp: memset failed"); return MEHDG_ECUDA;
    }
    if (launch_vjp(c, lam_V, lam_Vhat, g_v, g_vhat, st) != cudaSuccess) { set_err(c, "residual_vjp: launch failed"); return MEHDG_ECUDA; }
    return MEHDG_OK;
}
