// adjoint.cu -- the adjoint (transposed) condensed solve, for Euler contexts.
//
// A vector-Jacobian product through one Newton step needs lambda = J^-T g
// for the linearised system J = [[A_vv, A_v,vhat], [A_vhat,v, A_vhat,vhat]]
// of eq. R1 (Euler: no Q).  Its transpose condenses the same way (eqs.
// R2-R5 with every block transposed):
//   bhat_a  = g_vhat - A_v,vhat^T S^-T g_v                     (adjoint R5b)
//   A-hat^T x = A_vhat,vhat^T x - A_v,vhat^T S^-T A_vhat,v^T x  (adjoint of the four stages)
//   lambda_v = S^-T (g_v - A_vhat,v^T lambda_vhat)              (adjoint R2)
// with S = A_vv.  S^-T uses the stored LU factors of the condensation
// (lu_solve_T) and FP64 refinement against the exact transposed product
// S^T x, which is the residual's VJP with cotangent (x, 0); every other
// transposed block product is a VJP as well: (lam_V, lam_Vhat) -> (g_v,
// g_vhat) = (A_vv^T lam_V + A_vhat,v^T lam_Vhat, A_v,vhat^T lam_V +
// A_vhat,vhat^T lam_Vhat).
#include <cstdio>
#include <cstring>
#include "common.cuh"
#include "kernels.cuh"

cudaError_t launch_axpy(int64_t nK, int64_t ld, const double* dx, double* x, const int32_t* conv, cudaStream_t st);

namespace {

#define ATRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return MEHDG_ECUDA; } } while (0)

struct AdjWork {
    double *gv, *gh, *gv2, *gh2, *ya;
};

int adj_work(mehdg_ctx* c, AdjWork* w) {
    const size_t nv = (size_t)c->nK * c->Nv, nt = (size_t)c->G * 5 * c->tab.n2;
    const size_t need = sizeof(double) * (3 * nv + 2 * nt) + 5 * 256;
    if (c->adj_bytes < need) {
        if (c->d_adj) cudaFree(c->d_adj);
        c->d_adj = nullptr; c->adj_bytes = 0;
        if (cudaMalloc(&c->d_adj, need) != cudaSuccess) { set_err(c, "adjoint: out of memory"); return MEHDG_ENOMEM; }
        c->adj_bytes = need;
    }
    unsigned char* b = reinterpret_cast<unsigned char*>(c->d_adj);
    size_t off = 0;
    auto take = [&](double*& p, size_t n) { p = reinterpret_cast<double*>(b + off); off += (n * 8 + 255) & ~(size_t)255; };
    take(w->gv, nv); take(w->gh, nt); take(w->gv2, nv); take(w->gh2, nt); take(w->ya, nv);
    return MEHDG_OK;
}

int checks(mehdg_ctx* c, const char* what) {
    if (!c) return MEHDG_EINVAL;
    if (c->batch || c->ph.viscous) { set_err(c, "%s: Euler contexts of one element type only", what); return MEHDG_EINVAL; }
    if (!c->condensed) { set_err(c, "%s before condense", what); return MEHDG_ESTATE; }
    return MEHDG_OK;
}

// x (unpadded [nK][5][Nn]) = S^-T r (unpadded), FP64-refined: padded node-major
// solves with the transposed factors, r - S^T x from the VJP
int refine_solve_T(mehdg_ctx* c, const double* r_u, double* x_u, AdjWork& w, cudaStream_t st) {
    LUPlan P;
    P.nK = c->nK; P.ld = c->Npad; P.N = c->Nv; P.fp64 = c->prm.prec == MEHDG_FP64; P.prec = c->prm.prec;
    P.S = c->d_S; P.piv = c->d_piv; P.status = c->d_status; P.work = c->d_work; P.work_bytes = c->work_bytes;
    P.prof = &c->prof;
    const int64_t nK = c->nK, ld = c->Npad;
    ATRY(launch_set_rhs(nK, c->Nv, ld, c->tab.Nn, r_u, 1.0, nullptr, 0.0, c->d_r, st));
    ATRY(cudaMemsetAsync(c->d_x, 0, sizeof(double) * nK * ld, st));
    ATRY(cudaMemcpyAsync(c->d_res, c->d_r, sizeof(double) * nK * ld, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemsetAsync(c->d_conv, 0, sizeof(int32_t) * nK, st));
    const int maxit = c->prm.refine_max_iter > 0 ? c->prm.refine_max_iter : 1;
    for (int it = 0; it < maxit; ++it) {
        ATRY(lu_solve_T(P, c->d_res, c->d_dx, c->d_conv, st));
        ATRY(launch_axpy(nK, ld, c->d_dx, c->d_x, c->d_conv, st));
        ATRY(launch_copy_unpad(nK, c->Nv, ld, c->d_x, x_u, 1.0, st));
        ATRY(launch_vjp(c, x_u, nullptr, w.gv2, w.gh2, st));                 // S^T x = A_vv^T x
        ATRY(cudaMemsetAsync(c->d_cnt, 0, sizeof(int32_t), st));
        ATRY(launch_refine_update(nK, c->Nv, ld, c->d_r, w.gv2, c->d_res, c->d_nrm, c->d_conv, c->d_iters,
                                  c->d_status, c->prm.refine_tol, it, it == maxit - 1, nullptr, nullptr, c->d_cnt, st));
        ATRY(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        ATRY(cudaStreamSynchronize(st));
        if (*c->h_cnt == 0) break;
    }
    ATRY(launch_copy_unpad(nK, c->Nv, ld, c->d_x, x_u, 1.0, st));
    return MEHDG_OK;
}

__global__ void axpby2_kernel(double a, const double* x, double b, const double* y, double* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * (x ? x[i] : 0.0) + b * y[i];
}

unsigned grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

extern "C" int mehdg_condense_adjoint(mehdg_ctx* c, const double* g_V, const double* g_Vhat, double* bhat_a,
                                      void* stream) {
    int rc = checks(c, "condense_adjoint");
    if (rc) return rc;
    if (!g_V || !bhat_a) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    AdjWork w;
    if ((rc = adj_work(c, &w))) return rc;
    ATRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * c->nK, st));
    ATRY(cudaMemsetAsync(c->d_iters, 0, sizeof(int32_t) * c->nK, st));
    if ((rc = refine_solve_T(c, g_V, w.ya, w, st))) return rc;           // ya = S^-T g_V
    ATRY(launch_vjp(c, w.ya, nullptr, w.gv, w.gh, st));                   // gh = A_v,vhat^T ya
    const int64_t nt = c->G * 5 * (int64_t)c->tab.n2;
    axpby2_kernel<<<grid_of(nt), 256, 0, st>>>(1.0, g_Vhat, -1.0, w.gh, bhat_a, nt);
    MEHDG_COUNT(1);
    ATRY(cudaGetLastError());
    return MEHDG_OK;
}

extern "C" int mehdg_apply_condensed_adjoint(mehdg_ctx* c, const double* x, double* y, void* stream) {
    int rc = checks(c, "apply_condensed_adjoint");
    if (rc) return rc;
    if (!x || !y) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    AdjWork w;
    if ((rc = adj_work(c, &w))) return rc;
    ATRY(launch_vjp(c, nullptr, x, w.gv, w.gh, st));                      // A_vhat,v^T x, A_vhat,vhat^T x
    if ((rc = refine_solve_T(c, w.gv, w.ya, w, st))) return rc;           // S^-T A_vhat,v^T x
    ATRY(launch_vjp(c, w.ya, nullptr, w.gv, w.gh2, st));                  // A_v,vhat^T (...)
    const int64_t nt = c->G * 5 * (int64_t)c->tab.n2;
    axpby2_kernel<<<grid_of(nt), 256, 0, st>>>(1.0, w.gh, -1.0, w.gh2, y, nt);
    MEHDG_COUNT(1);
    ATRY(cudaGetLastError());
    return MEHDG_OK;
}

extern "C" int mehdg_recover_adjoint(mehdg_ctx* c, const double* g_V, const double* lam_Vhat, double* lam_V,
                                     void* stream) {
    int rc = checks(c, "recover_adjoint");
    if (rc) return rc;
    if (!g_V || !lam_Vhat || !lam_V) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    AdjWork w;
    if ((rc = adj_work(c, &w))) return rc;
    ATRY(launch_vjp(c, nullptr, lam_Vhat, w.gv, w.gh, st));               // A_vhat,v^T lam_Vhat
    const int64_t nv = c->nK * (int64_t)c->Nv;
    axpby2_kernel<<<grid_of(nv), 256, 0, st>>>(1.0, g_V, -1.0, w.gv, w.gv2, nv);
    MEHDG_COUNT(1);
    ATRY(cudaGetLastError());
    ATRY(cudaMemcpyAsync(w.ya, w.gv2, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    return refine_solve_T(c, w.ya, lam_V, w, st);
}

extern "C" int mehdg_solve_condensed_adjoint(mehdg_ctx* c, const double* bhat_a, double* x, double rtol, int restart,
                                             int max_iter, int* iters, double* relres, void* stream) {
    int rc = checks(c, "solve_condensed_adjoint");
    if (rc) return rc;
    if (!bhat_a || !x || restart < 1 || max_iter < 1 || !(rtol > 0.0)) return MEHDG_EINVAL;
    return gmres_trace(c, mehdg_apply_condensed_adjoint, bhat_a, x, rtol, restart, max_iter, iters, relres, stream);
}

// ---------------------------------------------------------------- VJP through Newton steps
namespace {

__global__ void lin3_kernel(double* out, const double* a, double sb, const double* b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + sb * b[i];
}
// g -= a + (p - m) / (2 h)
__global__ void gbar_update_kernel(double* g, const double* a, const double* p, const double* m, double inv2h,
                                   int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] -= a[i] + (p[i] - m[i]) * inv2h;
}
__global__ void maxabs_kernel(const double* x, int64_t n, unsigned long long* out) {
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(x[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __double_as_longlong(mx));   // non-negative doubles order as integers
}

}  // namespace

extern "C" int mehdg_pseudo_time_newton_vjp(mehdg_ctx* c, double* v, double* vhat, int nsteps, double tau,
                                            double lin_rtol, int restart, int max_iter, const double* gbar_v,
                                            const double* gbar_vhat, double* g_v0, double* g_vhat0, double fd_step,
                                            void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (c->batch || c->ph.viscous || !c->prm.time_term) {
        set_err(c, "pseudo_time_newton_vjp: Euler contexts of one element type with the stage term");
        return MEHDG_EINVAL;
    }
    if (c->nK == 0) return MEHDG_ESTATE;
    if (!v || !vhat || !gbar_v || !g_v0 || !g_vhat0 || nsteps < 1 || !(tau > 0.0) || !(fd_step > 0.0) ||
        !(lin_rtol > 0.0) || restart < 1 || max_iter < 1) {
        set_err(c, "pseudo_time_newton_vjp: bad arguments");
        return MEHDG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nv = c->nK * (int64_t)c->Nv, nt = c->G * 5 * (int64_t)c->tab.n2;
    // trajectory: states s_k and increments d_k (k < nsteps), and work vectors
    const size_t per = (size_t)(nv + nt);
    double* traj = nullptr;
    const size_t tbytes = sizeof(double) * (2 * (size_t)nsteps * per + 8 * per) + 64;
    if (cudaMalloc((void**)&traj, tbytes) != cudaSuccess) { set_err(c, "pseudo_time_newton_vjp: out of memory"); return MEHDG_ENOMEM; }
    auto S = [&](int k) { return traj + (size_t)k * per; };                 // [v | vhat] of state k
    auto D = [&](int k) { return traj + (size_t)(nsteps + k) * per; };      // [dV | dVhat] of step k
    double* W = traj + 2 * (size_t)nsteps * per;
    double *vs = W, *bh = W + per, *lam = W + 2 * per, *a = W + 3 * per, *pp = W + 4 * per, *mm = W + 5 * per,
           *gb = W + 6 * per, *sp = W + 7 * per;
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(W + 8 * per);
    const double dt0 = c->prm.dt;
    int rc = MEHDG_OK;
    const unsigned gn = grid_of(per);
    auto fail = [&](int r) { cudaFree(traj); if (dt0 > 0) mehdg_set_dt(c, dt0); return r; };
#define VTRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return fail(MEHDG_ECUDA); } } while (0)
#define VRC(x) do { int r_ = (x); if (r_) return fail(r_); } while (0)
    VRC(mehdg_set_dt(c, tau));
    // forward: s_{k+1} = s_k + d_k, J(s_k; v* = v_k) d_k = -R(s_k; v* = v_k)
    for (int k = 0; k < nsteps; ++k) {
        VTRY(cudaMemcpyAsync(S(k), v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        VTRY(cudaMemcpyAsync(S(k) + nv, vhat, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
        VTRY(cudaMemcpyAsync(vs, v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        VRC(mehdg_set_state(c, v, vhat, nullptr, vs, stream));
        VRC(mehdg_condense(c, bh, nullptr, stream));
        VTRY(cudaMemsetAsync(D(k) + nv, 0, sizeof(double) * nt, st));
        VRC(mehdg_solve_condensed(c, bh, D(k) + nv, lin_rtol, restart, max_iter, nullptr, nullptr, stream));
        VRC(mehdg_recover(c, D(k) + nv, D(k), nullptr, stream));
        lin3_kernel<<<gn, 256, 0, st>>>(v, v, 1.0, D(k), nv);
        lin3_kernel<<<gn, 256, 0, st>>>(vhat, vhat, 1.0, D(k) + nv, nt);
        MEHDG_COUNT(2);
    }
    // reverse: gbar_k = gbar_{k+1} - J_steady^T lam - (d/de J(s_k + e d_k)^T lam)(0),
    // lam = J(s_k)^-T gbar_{k+1}
    VTRY(cudaMemcpyAsync(gb, gbar_v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    if (gbar_vhat) VTRY(cudaMemcpyAsync(gb + nv, gbar_vhat, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    else VTRY(cudaMemsetAsync(gb + nv, 0, sizeof(double) * nt, st));
    for (int k = nsteps - 1; k >= 0; --k) {
        VTRY(cudaMemcpyAsync(vs, S(k), sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        VRC(mehdg_set_state(c, S(k), S(k) + nv, nullptr, vs, stream));
        VRC(mehdg_condense(c, pp, nullptr, stream));               // the factors of J(s_k)
        VRC(mehdg_condense_adjoint(c, gb, gb + nv, bh, stream));
        VTRY(cudaMemsetAsync(lam + nv, 0, sizeof(double) * nt, st));
        VRC(mehdg_solve_condensed_adjoint(c, bh, lam + nv, lin_rtol, restart, max_iter, nullptr, nullptr, stream));
        VRC(mehdg_recover_adjoint(c, gb, lam + nv, lam, stream));
        // steady part: the stage term's derivatives in v and v* cancel when v* = v
        const double inv_dt = c->ph.inv_dt;
        c->ph.inv_dt = 0.0;
        const cudaError_t es = launch_vjp(c, lam, lam + nv, a, a + nv, st);
        c->ph.inv_dt = inv_dt;
        VTRY(es);
        // second-order term along d_k at fixed v* = v_k, by central differences of the VJP
        VTRY(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), st));
        maxabs_kernel<<<256, 256, 0, st>>>(D(k), (int64_t)per, dmax);
        maxabs_kernel<<<256, 256, 0, st>>>(S(k), (int64_t)per, dmax + 1);
        MEHDG_COUNT(2);
        unsigned long long hm[2];
        VTRY(cudaMemcpyAsync(hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, st));
        VTRY(cudaStreamSynchronize(st));
        double dm, sm;
        std::memcpy(&dm, &hm[0], sizeof(double));
        std::memcpy(&sm, &hm[1], sizeof(double));
        const double h = dm > 0.0 ? fd_step * (sm > 0.0 ? sm : 1.0) / dm : 0.0;
        if (h > 0.0) {
            lin3_kernel<<<gn, 256, 0, st>>>(sp, S(k), h, D(k), (int64_t)per);
            MEHDG_COUNT(1);
            VRC(mehdg_set_state(c, sp, sp + nv, nullptr, vs, stream));
            VTRY(launch_vjp(c, lam, lam + nv, pp, pp + nv, st));
            lin3_kernel<<<gn, 256, 0, st>>>(sp, S(k), -h, D(k), (int64_t)per);
            MEHDG_COUNT(1);
            VRC(mehdg_set_state(c, sp, sp + nv, nullptr, vs, stream));
            VTRY(launch_vjp(c, lam, lam + nv, mm, mm + nv, st));
        } else {
            VTRY(cudaMemsetAsync(pp, 0, sizeof(double) * per, st));
            VTRY(cudaMemsetAsync(mm, 0, sizeof(double) * per, st));
        }
        gbar_update_kernel<<<gn, 256, 0, st>>>(gb, a, pp, mm, h > 0.0 ? 0.5 / h : 0.0, (int64_t)per);
        MEHDG_COUNT(1);
        VTRY(cudaGetLastError());
    }
    VTRY(cudaMemcpyAsync(g_v0, gb, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    VTRY(cudaMemcpyAsync(g_vhat0, gb + nv, sizeof(double) * nt, cudaMemcpyDeviceToDevice, st));
    VTRY(cudaStreamSynchronize(st));
    // leave the context at the final state, with its own step size
    cudaFree(traj);
    if ((rc = mehdg_set_dt(c, dt0))) return rc;
    // the context's state pointed into the freed trajectory: a set_state comes next
    c->v = nullptr; c->vh = nullptr; c->vs = nullptr; c->condensed = false; c->pj_ready = false;
    return MEHDG_OK;
#undef VTRY
#undef VRC
}
