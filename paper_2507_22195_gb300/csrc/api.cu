// api.cu -- the C-ABI of include/mehdg.h and the orchestration of one Newton
// step per macro-element (Algorithm 1, local parts; eqs. R1-R6):
//   condense : R (eq. s32); z = A_qq^-1 R_Q; S^K = A_vv - A_vq A_qq^-1 A_qv
//              (eqs. R1, R3); LU(S^K); y = S^-1 (-R_V + A_vq z) refined in FP64;
//              bhat^K = -R_Vhat + A_vhat,q z + (-A_vhat,v + A_vhat,q C) y
//              (eq. R5b), summed over the two sides of every face;
//   apply    : y = (A_vhat,vhat - A_vhat,q C_t) x + (A_vhat,v - A_vhat,q C) S^-1
//              (-A_v,vhat + A_vq C_t) x  (Sec. 6.3 stages 1-4);
//   recover  : dV = S^-1 (-R_V + A_vq z - (A_v,vhat - A_vq C_t) dVhat)  (eq. R2),
//              dQ = -z - C dV - C_t dVhat  (eq. R6),
// with C = A_qq^-1 A_qv and C_t = A_qq^-1 A_qvhat (Euler: no q, no z, C, C_t).
// Every product with a Jacobian block other than the LU of S is matrix-free:
// a forward-mode tangent of the FP64 residual along (dv, dvhat, dq), with
// the q-direction built by the line operators of qproj.cu.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "kernels.cuh"
#include "prof.cuh"

cudaError_t launch_axpy(int64_t nK, int64_t ld, const double* dx, double* x, const int32_t* conv, cudaStream_t st);

std::atomic<long long> g_mehdg_launches{0};

void set_err(mehdg_ctx* ctx, const char* fmt, ...) {
    if (!ctx) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
}

namespace {

template <class T> void dfree(T*& p) { if (p) { cudaFree((void*)p); p = nullptr; } }

void free_mesh(mehdg_ctx* c) {
    dfree(c->d_box); dfree(c->d_gid); dfree(c->d_g2l); dfree(c->d_RV); dfree(c->d_RHloc);
    dfree(c->d_tRHloc); dfree(c->d_tRHloc2); dfree(c->d_tRV); dfree(c->d_xu); dfree(c->d_r); dfree(c->d_x);
    dfree(c->d_res); dfree(c->d_dx); dfree(c->d_nrm); dfree(c->d_status); dfree(c->d_iters); dfree(c->d_conv);
    dfree(c->d_cnt); dfree(c->d_S); dfree(c->d_piv); dfree(c->d_work);
    dfree(c->d_RQ); dfree(c->d_z); dfree(c->d_dq); dfree(c->d_qt1); dfree(c->d_qt2); dfree(c->d_Minv); dfree(c->d_C1);
    dfree(c->d_pj); dfree(c->d_pjf); dfree(c->d_pq); dfree(c->d_pqf); c->pj_ready = false;
    if (c->d_krylov) { cudaFree(c->d_krylov); c->d_krylov = nullptr; c->krylov_bytes = 0; }
    if (c->d_newton) { cudaFree(c->d_newton); c->d_newton = nullptr; c->newton_bytes = 0; }
    if (c->d_adj) { cudaFree(c->d_adj); c->d_adj = nullptr; c->adj_bytes = 0; }
    if (c->lu_graph) { cudaGraphExecDestroy(c->lu_graph); c->lu_graph = nullptr; }
    if (c->cond_graph) { cudaGraphExecDestroy(c->cond_graph); c->cond_graph = nullptr; }
    if (c->cap_in) { cudaEventDestroy(c->cap_in); c->cap_in = nullptr; }
    if (c->cap_out) { cudaEventDestroy(c->cap_out); c->cap_out = nullptr; }
    if (c->cap_stream) { cudaStreamDestroy(c->cap_stream); c->cap_stream = nullptr; }
    for (auto& k : c->cap_key) k = nullptr;
    if (c->lu_ev_in) { cudaEventDestroy(c->lu_ev_in); c->lu_ev_in = nullptr; }
    if (c->lu_ev_out) { cudaEventDestroy(c->lu_ev_out); c->lu_ev_out = nullptr; }
    if (c->zs_ev_in) { cudaEventDestroy(c->zs_ev_in); c->zs_ev_in = nullptr; }
    if (c->zs_ev_out) { cudaEventDestroy(c->zs_ev_out); c->zs_ev_out = nullptr; }
    if (c->lu_stream) { cudaStreamDestroy(c->lu_stream); c->lu_stream = nullptr; }
    if (c->h_cnt) { cudaFreeHost(c->h_cnt); c->h_cnt = nullptr; }
    batch_free(c);
    c->nK = 0; c->condensed = false; c->lu_graph_failed = false;
}

ResidualArgs base_args(mehdg_ctx* c) {
    ResidualArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tab = c->tab; a.ph = c->ph; a.box = c->d_box; a.gid = c->d_gid;
    a.v = c->v; a.vs = c->vs; a.vh = c->vh; a.q = c->q;
    a.status = c->d_status;
    return a;
}

QProjArgs qargs(mehdg_ctx* c) {
    QProjArgs q;
    q.tab = c->tab; q.box = c->d_box; q.gid = c->d_gid; q.Minv = c->d_Minv; q.C1 = c->d_C1;
    q.tmp1 = c->d_qt1; q.tmp2 = c->d_qt2;
    return q;
}

// LU of every S^K.  The sequence of launches depends only on the mesh and
// the precision, so it is captured into a CUDA graph on the first call and
// replayed afterwards (on the context's own stream, ordered after and before
// the caller's stream by events); with phase profiling on, the launches are
// issued directly so that the phase events sit between them.
cudaError_t factor_all(mehdg_ctx* c, const LUPlan& P, cudaStream_t st) {
    // MEHDG_NO_GRAPH=1: direct launches (e.g. under a kernel profiler that
    // replays launches one by one)
    static const bool no_graph = [] { const char* e = std::getenv("MEHDG_NO_GRAPH"); return e && e[0] == '1'; }();
    // (while the whole condensation is being recorded, its LU kernels go into that graph directly:
    // a graph launch cannot be part of a stream capture)
    if (c->prof.on || no_graph || c->lu_graph_failed || c->graph_refine) return lu_factor(P, st);
    cudaError_t e;
    if (!c->lu_graph) {
        if (!c->lu_stream && (e = cudaStreamCreateWithFlags(&c->lu_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if (!c->lu_ev_in && (e = cudaEventCreateWithFlags(&c->lu_ev_in, cudaEventDisableTiming)) != cudaSuccess) return e;
        if (!c->lu_ev_out && (e = cudaEventCreateWithFlags(&c->lu_ev_out, cudaEventDisableTiming)) != cudaSuccess) return e;
        const long long before = g_mehdg_launches.load();
        // A capture can fail or be invalidated from outside (a tool that
        // serialises launches, another thread's illegal call during the
        // capture).  Then the context stops capturing and launches the same
        // kernels directly, now and on later calls (lu_graph_failed).
        cudaGraph_t g = nullptr;
        cudaError_t ef = cudaStreamBeginCapture(c->lu_stream, cudaStreamCaptureModeRelaxed);
        if (ef == cudaSuccess) {
            ef = lu_factor(P, c->lu_stream);
            e = cudaStreamEndCapture(c->lu_stream, &g);
            if (ef == cudaSuccess) ef = e;
        }
        if (ef == cudaSuccess) {
            ef = cudaGraphInstantiate(&c->lu_graph, g, 0);
            if (ef != cudaSuccess) c->lu_graph = nullptr;
        }
        if (g) cudaGraphDestroy(g);
        if (ef != cudaSuccess) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(c->lu_stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g2 = nullptr;
                cudaStreamEndCapture(c->lu_stream, &g2);
                if (g2) cudaGraphDestroy(g2);
            }
            (void)cudaGetLastError();                   // capture errors are not sticky: clear the record
            g_mehdg_launches = before;                  // nothing of the failed capture ran
            c->lu_graph_failed = true;
            fprintf(stderr, "mehdg: LU graph capture failed (%s); launching its kernels directly\n",
                    cudaGetErrorString(ef));
            return lu_factor(P, st);
        }
        c->lu_graph_launches = g_mehdg_launches.load() - before;
        g_mehdg_launches -= c->lu_graph_launches;      // counted when they run
    }
    if ((e = cudaEventRecord(c->lu_ev_in, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->lu_stream, c->lu_ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(c->lu_graph, c->lu_stream)) != cudaSuccess ||
        (e = cudaEventRecord(c->lu_ev_out, c->lu_stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, c->lu_ev_out, 0)) != cudaSuccess)
        return e;
    g_mehdg_launches += c->lu_graph_launches;
    return cudaSuccess;
}

LUPlan plan(mehdg_ctx* c) {
    LUPlan P;
    P.nK = c->nK; P.ld = c->Npad; P.N = c->Nv;
    P.fp64 = c->prm.prec == MEHDG_FP64; P.prec = c->prm.prec;
    P.S = c->d_S; P.piv = c->d_piv; P.status = c->d_status;
    P.work = c->d_work; P.work_bytes = c->work_bytes;
    P.prof = &c->prof;
    P.leaf_ctas = c->tune_leaf_ctas;
    P.solve_ctas = c->tune_solve_ctas;
    return P;
}

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return MEHDG_ECUDA; } } while (0)

bool viscous(const mehdg_ctx* c) { return c->ph.viscous != 0; }

// q-direction: out = alpha A_qq^-1 R_Q + beta C x + gamma C_t xh (viscous only)
int qproj(mehdg_ctx* c, double alpha, const double* x, double beta, const double* xh, double gamma, double* out,
          const int32_t* skip, cudaStream_t st) {
    TRY(launch_qproj(qargs(c), c->nK, alpha != 0.0 ? c->d_RQ : nullptr, alpha, x, beta, xh, gamma, out, skip, st));
    return MEHDG_OK;
}

// tangent residual along (dv, dvh, dq): tRV ([nK][5][Nn]) and tRH (per-side trace)
int tangent(mehdg_ctx* c, const double* dv, const double* dvh, const double* dq, double* tRV, double* tRH,
            const int32_t* skip, cudaStream_t st) {
    ResidualArgs a = base_args(c);
    a.dv = dv; a.dvh = dvh; a.dq = viscous(c) ? dq : nullptr; a.tRV = tRV; a.tRH = tRH; a.skip = skip;
    a.pj = c->pj_ready ? c->d_pj : nullptr;      // linear volume pass from the stored point Jacobians
    a.pjf = c->pj_ready ? c->d_pjf : nullptr;    // linear face pass when the trace direction is 0
    a.pq = c->pj_ready ? c->d_pq : nullptr;      // viscous: dG/dq blocks for the linear volume pass
    a.pqf = c->pj_ready ? c->d_pqf : nullptr;    // viscous: dGhat/dq blocks for the linear face pass
    int ev = prof_begin(&c->prof, PH_TANGENT, st);
    TRY(launch_residual(a, c->nK, viscous(c), true, st));
    prof_end(&c->prof, ev, st, 0.0);
    return MEHDG_OK;
}

// S x = A_vv x - A_vq C x, matrix-free: tangent along (dv = x, dq = -C x)
int apply_S(mehdg_ctx* c, const double* xu, double* out, const int32_t* skip, cudaStream_t st) {
    if (viscous(c)) {
        int rc = qproj(c, 0.0, xu, -1.0, nullptr, 0.0, c->d_dq, skip, st);
        if (rc) return rc;
    }
    return tangent(c, xu, nullptr, c->d_dq, out, nullptr, skip, st);
}

// x (padded FP64) = S^-1 r by LU solves in the factor precision and FP64
// refinement with the matrix-free S x
int refine_solve(mehdg_ctx* c, const double* r, double* x, cudaStream_t st) {
    LUPlan P = plan(c);
    const int64_t nK = c->nK, ld = c->Npad;
    TRY(cudaMemsetAsync(x, 0, sizeof(double) * nK * ld, st));
    TRY(cudaMemcpyAsync(c->d_res, r, sizeof(double) * nK * ld, cudaMemcpyDeviceToDevice, st));
    TRY(cudaMemsetAsync(c->d_conv, 0, sizeof(int32_t) * nK, st));
    const int maxit = c->prm.refine_max_iter > 0 ? c->prm.refine_max_iter : 1;
    for (int it = 0; it < maxit; ++it) {
        int ev = prof_begin(&c->prof, PH_SOLVE, st);
        TRY(lu_solve(P, c->d_res, c->d_dx, c->d_conv, st));
        prof_end(&c->prof, ev, st, 0.0);
        TRY(launch_axpy(nK, ld, c->d_dx, x, c->d_conv, st));
        TRY(launch_copy_unpad(nK, c->Nv, ld, x, c->d_xu, 1.0, st));
        int rc = apply_S(c, c->d_xu, c->d_tRV, c->d_conv, st);
        if (rc) return rc;
        TRY(cudaMemsetAsync(c->d_cnt, 0, sizeof(int32_t), st));
        TRY(launch_refine_update(nK, c->Nv, ld, r, c->d_tRV, c->d_res, c->d_nrm, c->d_conv, c->d_iters,
                                 c->d_status, c->prm.refine_tol, it, it == maxit - 1, nullptr, nullptr,
                                 c->d_cnt, st));
        // graph capture: every sweep is recorded; converged elements skip their work on the device
        if (c->graph_refine) continue;
        TRY(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (*c->h_cnt == 0) break;
    }
    return MEHDG_OK;
}

}  // namespace

extern "C" {

void mehdg_default_params(mehdg_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gamma = 1.4; p->Re = 1600.0; p->Pr = 0.71; p->Mach = 0.1; p->dt = 1.0;
    p->viscous = 0; p->flux = MEHDG_FLUX_KEPES; p->prec = MEHDG_MIXED_TF32;
    p->refine_tol = 1e-12; p->refine_max_iter = 10; p->time_term = 1;
}

int mehdg_create(mehdg_ctx** out, const mehdg_params* prm) {
    if (!out || !prm) return MEHDG_EINVAL;
    *out = nullptr;
    if (!(prm->gamma > 1.0) || prm->flux < 0 || prm->flux > 2 || prm->prec < 0 || prm->prec > 4 ||
        (prm->time_term && !(prm->dt > 0.0)) || (prm->viscous && !(prm->Re > 0 && prm->Pr > 0 && prm->Mach > 0)))
        return MEHDG_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return MEHDG_ECUDA;
    mehdg_ctx* c = new mehdg_ctx();
    c->prm = *prm;
    c->err[0] = 0;
    Phys& ph = c->ph;
    ph.gamma = prm->gamma;
    ph.mu = prm->viscous ? prm->Mach / prm->Re : 0.0;
    ph.kappa = prm->viscous ? ph.mu / ((prm->gamma - 1.0) * prm->Pr) : 0.0;
    ph.sv_mom = prm->viscous ? 1.0 / prm->Re : 0.0;
    ph.sv_en = prm->viscous ? 1.0 / (prm->Re * (prm->gamma - 1.0) * prm->Mach * prm->Mach * prm->Pr) : 0.0;
    ph.inv_dt = prm->time_term ? 1.0 / prm->dt : 0.0;
    ph.viscous = prm->viscous; ph.flux = prm->flux; ph.time_term = prm->time_term;
    *out = c;
    return MEHDG_OK;
}

int mehdg_set_mesh(mehdg_ctx* c, int64_t nK, const int32_t* p, const int32_t* m, const double* box,
                   const int64_t* face_gid, int64_t G) {
    if (!c) return MEHDG_EINVAL;
    if (nK <= 0 || !p || !m || !box || !face_gid || G <= 0) { set_err(c, "set_mesh: bad arguments"); return MEHDG_EINVAL; }
    const int p0 = p[0], m0 = m[0];
    bool uneven = false;
    for (int64_t K = 0; K < nK; ++K)
        if (p[K] != p0 || m[K] != m0) uneven = true;
    // MEHDG_FORCE_BATCH=1 runs a uniform mesh through the batch path as well
    // (its waves, when the mesh exceeds the memory budget)
    if (const char* e = std::getenv("MEHDG_FORCE_BATCH")) uneven = uneven || e[0] == '1';
    if (uneven) {
        free_mesh(c);
        const int rc = batch_set_mesh(c, nK, p, m, box, face_gid, G);
        if (rc) free_mesh(c);
        return rc;
    }
    if (p0 < 1 || p0 > MEHDG_MAXP || m0 < 1 || m0 > 16) { set_err(c, "set_mesh: p in 1..4, m in 1..16"); return MEHDG_EINVAL; }
    if (c->prm.viscous && c->prm.prec == MEHDG_FP64 && p0 > 3) {
        set_err(c, "set_mesh: the FP64 viscous Jacobian supports p <= 3"); return MEHDG_EINVAL;
    }
    std::vector<int64_t> g2l(2 * G, -1);
    for (int64_t K = 0; K < nK; ++K) {
        for (int d = 0; d < 3; ++d)
            if (!(box[6 * K + 3 + d] > box[6 * K + d])) { set_err(c, "set_mesh: degenerate box %lld", (long long)K); return MEHDG_EINVAL; }
        for (int f = 0; f < 6; ++f) {
            int64_t g = face_gid[6 * K + f];
            if (g < 0 || g >= G) { set_err(c, "set_mesh: face id out of range"); return MEHDG_EINVAL; }
            if (g2l[2 * g] < 0) g2l[2 * g] = 6 * K + f;
            else if (g2l[2 * g + 1] < 0) g2l[2 * g + 1] = 6 * K + f;
            else { set_err(c, "set_mesh: global face %lld used more than twice", (long long)g); return MEHDG_EINVAL; }
        }
    }
    free_mesh(c);
    c->nK = nK; c->G = G; c->p = p0; c->m = m0;
    host_build_tables(p0, m0, &c->tab);
    const Tab& t = c->tab;
    c->Nv = 5 * t.Nn;
    c->Nt_loc = 30 * t.n2;
    c->Npad = (c->Nv + 255) / 256 * 256;
    const bool fp64 = c->prm.prec == MEHDG_FP64;
    const bool vis = c->prm.viscous != 0;
    const size_t ts = fp64 ? 8 : 4;
    const size_t Sbytes = (size_t)nK * c->Npad * c->Npad * ts;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    if (Sbytes > freeb * 0.9) {
        set_err(c, "set_mesh: %zu bytes of dense S^K do not fit (%zu free); use fewer elements per context", Sbytes, freeb);
        return MEHDG_ENOMEM;
    }
#define DALLOC(ptr, bytes) do { if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) { set_err(c, "cudaMalloc %s (%zu bytes) failed", #ptr, (size_t)(bytes)); free_mesh(c); return MEHDG_ENOMEM; } } while (0)
    DALLOC(c->d_box, sizeof(double) * 6 * nK);
    DALLOC(c->d_gid, sizeof(int64_t) * 6 * nK);
    DALLOC(c->d_g2l, sizeof(int64_t) * 2 * G);
    DALLOC(c->d_RV, sizeof(double) * nK * c->Nv);
    DALLOC(c->d_RHloc, sizeof(double) * nK * c->Nt_loc);
    DALLOC(c->d_tRHloc, sizeof(double) * nK * c->Nt_loc);
    DALLOC(c->d_tRHloc2, sizeof(double) * nK * c->Nt_loc);
    DALLOC(c->d_tRV, sizeof(double) * nK * c->Nv);
    DALLOC(c->d_xu, sizeof(double) * nK * c->Nv);
    DALLOC(c->d_r, sizeof(double) * nK * c->Npad);
    DALLOC(c->d_x, sizeof(double) * nK * c->Npad);
    DALLOC(c->d_res, sizeof(double) * nK * c->Npad);
    DALLOC(c->d_dx, sizeof(double) * nK * c->Npad);
    DALLOC(c->d_nrm, sizeof(double) * 2 * nK);
    DALLOC(c->d_status, sizeof(int32_t) * nK);
    DALLOC(c->d_iters, sizeof(int32_t) * nK);
    DALLOC(c->d_conv, sizeof(int32_t) * nK);
    DALLOC(c->d_cnt, sizeof(int32_t));
    if (vis) {
        const size_t qb = sizeof(double) * nK * 15 * (size_t)t.Nn;
        DALLOC(c->d_RQ, qb); DALLOC(c->d_z, qb); DALLOC(c->d_dq, qb); DALLOC(c->d_qt1, qb); DALLOC(c->d_qt2, qb);
        DALLOC(c->d_Minv, sizeof(double) * t.n * t.n);
        DALLOC(c->d_C1, sizeof(double) * t.n * t.n);
    }
    DALLOC(c->d_pj, sizeof(double) * 100 * (size_t)nK * t.m * t.m * t.m * t.npt);
    DALLOC(c->d_pjf, sizeof(double) * 25 * (size_t)nK * 6 * t.m * t.m * t.ng * t.ng);
    if (vis) DALLOC(c->d_pqf, sizeof(double) * 75 * (size_t)nK * 6 * t.m * t.m * t.ng * t.ng);
    if (vis) DALLOC(c->d_pq, sizeof(double) * 225 * (size_t)nK * t.m * t.m * t.m * t.npt);
    DALLOC(c->d_S, Sbytes);
    DALLOC(c->d_piv, sizeof(int32_t) * nK * c->Npad);
    c->work_bytes = lu_work_bytes(nK, c->Npad, fp64, c->prm.prec);
    DALLOC(c->d_work, c->work_bytes);
#undef DALLOC
    if (cudaMallocHost((void**)&c->h_cnt, sizeof(int32_t)) != cudaSuccess) { free_mesh(c); return MEHDG_ENOMEM; }
    if (cudaMemcpy(c->d_box, box, sizeof(double) * 6 * nK, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_gid, face_gid, sizeof(int64_t) * 6 * nK, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_g2l, g2l.data(), sizeof(int64_t) * 2 * G, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int32_t) * nK) != cudaSuccess ||
        cudaMemset(c->d_iters, 0, sizeof(int32_t) * nK) != cudaSuccess) {
        set_err(c, "set_mesh: copy failed"); free_mesh(c); return MEHDG_ECUDA;
    }
    if (vis) {
        std::vector<double> Minv(t.n * t.n), C1(t.n * t.n);
        host_build_qtables(t, Minv.data(), C1.data());
        if (cudaMemcpy(c->d_Minv, Minv.data(), sizeof(double) * t.n * t.n, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_C1, C1.data(), sizeof(double) * t.n * t.n, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_err(c, "set_mesh: copy failed"); free_mesh(c); return MEHDG_ECUDA;
        }
    }
    return MEHDG_OK;
}

int mehdg_set_state(mehdg_ctx* c, const double* v, const double* vhat, const double* q, const double* vstar,
                    void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0) { set_err(c, "set_state before set_mesh"); return MEHDG_ESTATE; }
    if (!v || !vhat || (c->prm.viscous && !q) || (c->prm.time_term && !vstar)) {
        set_err(c, "set_state: missing array"); return MEHDG_EINVAL;
    }
    if (c->batch) return batch_set_state(c, v, vhat, q, vstar, (cudaStream_t)stream);
    c->v = v; c->vh = vhat; c->q = q; c->vs = vstar;
    c->condensed = false;
    c->pj_ready = false;
    return MEHDG_OK;
}

int mehdg_residual(mehdg_ctx* c, double* R_V, double* R_Q, double* R_Vhat, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->v) { set_err(c, "residual before set_state"); return MEHDG_ESTATE; }
    if (!R_V || !R_Vhat || (c->batch && c->prm.viscous && !R_Q)) { set_err(c, "residual: null output"); return MEHDG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (c->batch) return batch_residual(c, R_V, R_Q, R_Vhat, st);
    TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * c->nK, st));
    ResidualArgs a = base_args(c);
    a.RV = R_V; a.RQ = viscous(c) ? R_Q : nullptr; a.RH = c->d_RHloc;
    int ev = prof_begin(&c->prof, PH_RESIDUAL, st);
    TRY(launch_residual(a, c->nK, viscous(c), false, st));
    if (c->src) TRY(launch_add(c->src, R_V, c->nK * (int64_t)c->Nv, st));
    prof_end(&c->prof, ev, st, 0.0);
    TRY(launch_trace_gather(c->d_RHloc, c->d_g2l, c->G, c->tab.n2, R_Vhat, 1.0, nullptr, 0.0, st));
    return MEHDG_OK;
}

int mehdg_condense(mehdg_ctx* c, double* bhat, double* Ahat_local, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->v) { set_err(c, "condense before set_state"); return MEHDG_ESTATE; }
    if (!bhat) { set_err(c, "condense: null bhat"); return MEHDG_EINVAL; }
    if (Ahat_local) { set_err(c, "condense: the explicit A-hat^K is not formed; use mehdg_apply_condensed"); return MEHDG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (c->batch) return batch_condense(c, bhat, st);
    const bool fp64 = c->prm.prec == MEHDG_FP64;
    const bool vis = viscous(c);
    const int64_t nK = c->nK, ld = c->Npad;
    TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * nK, st));
    TRY(cudaMemsetAsync(c->d_iters, 0, sizeof(int32_t) * nK, st));
    // S^K := 0 on the context's side stream while the (FP64-bound) residual
    // runs; the Jacobian waits for it
    const size_t sbytes = (size_t)nK * ld * ld * (fp64 ? 8 : 4);
    if (!c->lu_stream) TRY(cudaStreamCreateWithFlags(&c->lu_stream, cudaStreamNonBlocking));
    if (!c->zs_ev_in) TRY(cudaEventCreateWithFlags(&c->zs_ev_in, cudaEventDisableTiming));
    if (!c->zs_ev_out) TRY(cudaEventCreateWithFlags(&c->zs_ev_out, cudaEventDisableTiming));
    TRY(cudaEventRecord(c->zs_ev_in, st));
    TRY(cudaStreamWaitEvent(c->lu_stream, c->zs_ev_in, 0));
    TRY(cudaMemsetAsync(c->d_S, 0, sbytes, c->lu_stream));
    TRY(cudaEventRecord(c->zs_ev_out, c->lu_stream));
    // residual at the state
    ResidualArgs a = base_args(c);
    a.RV = c->d_RV; a.RH = c->d_RHloc; a.RQ = vis ? c->d_RQ : nullptr;
    int ev = prof_begin(&c->prof, PH_RESIDUAL, st);
    TRY(launch_residual(a, nK, vis, false, st));
    if (c->src) TRY(launch_add(c->src, c->d_RV, nK * (int64_t)c->Nv, st));
    prof_end(&c->prof, ev, st, 0.0);
    // z = A_qq^-1 R_Q
    int rc;
    if (vis && (rc = qproj(c, 1.0, nullptr, 0.0, nullptr, 0.0, c->d_z, nullptr, st))) return rc;
    // S^K = A_vv - A_vq C (dense), padded identity: the point passes (FP64-bound, S untouched) also
    // run beside the zeroing of S; the passes that add into S wait for it
    JacobianArgs ja;
    ja.tab = c->tab; ja.ph = c->ph; ja.box = c->d_box; ja.v = c->v; ja.vs = c->vs; ja.vh = c->vh; ja.q = c->q;
    ja.gid = c->d_gid; ja.S = c->d_S; ja.ld = ld; ja.status = c->d_status; ja.C1 = c->d_C1;
    ja.pj = c->d_pj; ja.pjf = c->d_pjf; ja.pq = c->d_pq; ja.pqf = c->d_pqf;
    ev = prof_begin(&c->prof, PH_JACOBIAN, st);
    TRY(launch_jacobian(ja, nK, fp64, st, 1));
    TRY(cudaStreamWaitEvent(st, c->zs_ev_out, 0));
    TRY(launch_pad_identity(c->d_S, nK, ld, c->Nv, fp64, st));
    TRY(launch_jacobian(ja, nK, fp64, st, 2));
    c->pj_ready = c->d_pj != nullptr;
    prof_end(&c->prof, ev, st, 0.0);
    // LU
    LUPlan P = plan(c);
    TRY(factor_all(c, P, st));
    // y = S^-1 (-R_V + A_vq z)
    if (vis) {
        if ((rc = tangent(c, nullptr, nullptr, c->d_z, c->d_tRV, nullptr, nullptr, st))) return rc;
        TRY(launch_set_rhs(nK, c->Nv, ld, c->tab.Nn, c->d_RV, -1.0, c->d_tRV, 1.0, c->d_r, st));
    } else {
        TRY(launch_set_rhs(nK, c->Nv, ld, c->tab.Nn, c->d_RV, -1.0, nullptr, 0.0, c->d_r, st));
    }
    if ((rc = refine_solve(c, c->d_r, c->d_x, st))) return rc;
    // bhat^K = -R_Vhat^K - dR_Vhat[dv = y, dq = -C y - z], summed over sides
    TRY(launch_copy_unpad(nK, c->Nv, ld, c->d_x, c->d_xu, 1.0, st));
    if (vis && (rc = qproj(c, -1.0, c->d_xu, -1.0, nullptr, 0.0, c->d_dq, nullptr, st))) return rc;
    if ((rc = tangent(c, c->d_xu, nullptr, c->d_dq, c->d_tRV, c->d_tRHloc, nullptr, st))) return rc;
    TRY(launch_trace_gather(c->d_RHloc, c->d_g2l, c->G, c->tab.n2, bhat, -1.0, nullptr, 0.0, st));
    TRY(launch_trace_gather(c->d_tRHloc, c->d_g2l, c->G, c->tab.n2, bhat, -1.0, bhat, 1.0, st));
    c->condensed = true;
    return MEHDG_OK;
}

int mehdg_apply_condensed(mehdg_ctx* c, const double* x, double* y, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->condensed) { set_err(c, c->batch ? "apply_condensed: no condensation kept (before condense, or the batch "
                                       "streamed in waves)" : "apply_condensed before condense"); return MEHDG_ESTATE; }
    if (!x || !y) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (c->batch) return batch_apply(c, x, y, st);
    const bool vis = viscous(c);
    const int64_t nK = c->nK, ld = c->Npad;
    int rc;
    // stage 1: y1 = -dR_V[dvhat = x, dq = -C_t x]
    if (vis && (rc = qproj(c, 0.0, nullptr, 0.0, x, -1.0, c->d_dq, nullptr, st))) return rc;
    if ((rc = tangent(c, nullptr, x, c->d_dq, c->d_tRV, nullptr, nullptr, st))) return rc;
    // stage 2: y2 = S^-1 y1
    TRY(launch_set_rhs(nK, c->Nv, ld, c->tab.Nn, c->d_tRV, -1.0, nullptr, 0.0, c->d_r, st));
    if ((rc = refine_solve(c, c->d_r, c->d_x, st))) return rc;
    // stages 3-4: y = dR_Vhat[dv = y2, dvhat = x, dq = -C y2 - C_t x], summed over sides
    TRY(launch_copy_unpad(nK, c->Nv, ld, c->d_x, c->d_xu, 1.0, st));
    if (vis && (rc = qproj(c, 0.0, c->d_xu, -1.0, x, -1.0, c->d_dq, nullptr, st))) return rc;
    if ((rc = tangent(c, c->d_xu, x, c->d_dq, c->d_tRV, c->d_tRHloc, nullptr, st))) return rc;
    TRY(launch_trace_gather(c->d_tRHloc, c->d_g2l, c->G, c->tab.n2, y, 1.0, nullptr, 0.0, st));
    return MEHDG_OK;
}

int mehdg_recover(mehdg_ctx* c, const double* dVhat, double* dV, double* dQ, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->condensed) { set_err(c, c->batch ? "recover: no condensation kept (before condense, or the batch "
                                       "streamed in waves)" : "recover before condense"); return MEHDG_ESTATE; }
    if (!dVhat || !dV || (viscous(c) && !dQ)) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (c->batch) return batch_recover(c, dVhat, dV, dQ, st);
    const bool vis = viscous(c);
    const int64_t nK = c->nK, ld = c->Npad;
    int rc;
    // eq. R2: S dV = -R_V - dR_V[dvhat = dVhat, dq = -z - C_t dVhat]
    if (vis && (rc = qproj(c, -1.0, nullptr, 0.0, dVhat, -1.0, c->d_dq, nullptr, st))) return rc;
    if ((rc = tangent(c, nullptr, dVhat, c->d_dq, c->d_tRV, nullptr, nullptr, st))) return rc;
    TRY(launch_set_rhs(nK, c->Nv, ld, c->tab.Nn, c->d_RV, -1.0, c->d_tRV, -1.0, c->d_r, st));
    if ((rc = refine_solve(c, c->d_r, c->d_x, st))) return rc;
    TRY(launch_copy_unpad(nK, c->Nv, ld, c->d_x, dV, 1.0, st));
    // eq. R6: dQ = -z - C dV - C_t dVhat
    if (vis && (rc = qproj(c, -1.0, dV, -1.0, dVhat, -1.0, dQ, nullptr, st))) return rc;
    return MEHDG_OK;
}

int mehdg_status(mehdg_ctx* c, int32_t* per_K_status, int32_t* iters) {
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0) return MEHDG_ESTATE;
    TRY(cudaDeviceSynchronize());
    if (per_K_status) TRY(cudaMemcpy(per_K_status, c->d_status, sizeof(int32_t) * c->nK, cudaMemcpyDeviceToHost));
    if (iters) TRY(cudaMemcpy(iters, c->d_iters, sizeof(int32_t) * c->nK, cudaMemcpyDeviceToHost));
    return MEHDG_OK;
}

int mehdg_status_device(mehdg_ctx* c, int32_t* per_K_status, int32_t* iters, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0) return MEHDG_ESTATE;
    if (!per_K_status && !iters) return MEHDG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (per_K_status)
        TRY(cudaMemcpyAsync(per_K_status, c->d_status, sizeof(int32_t) * c->nK, cudaMemcpyDeviceToDevice, st));
    if (iters) TRY(cudaMemcpyAsync(iters, c->d_iters, sizeof(int32_t) * c->nK, cudaMemcpyDeviceToDevice, st));
    return MEHDG_OK;
}

const char* mehdg_last_error(const mehdg_ctx* c) { return c ? c->err : "null context"; }

int mehdg_batch_layout(mehdg_ctx* c, int64_t* voff, int64_t* toff) {
    if (!c) return MEHDG_EINVAL;
    if (!c->batch) { set_err(c, "batch_layout: not a batch context"); return MEHDG_EINVAL; }
    batch_layout(c, voff, toff);
    return MEHDG_OK;
}

int mehdg_batch_autotune(mehdg_ctx* c, int64_t trial_max, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->batch) { set_err(c, "batch_autotune: not a batch context"); return MEHDG_EINVAL; }
    return batch_autotune(c, trial_max, (cudaStream_t)stream);
}

int mehdg_batch_report(mehdg_ctx* c, char* buf, size_t len) {
    if (!c || !c->batch) return MEHDG_EINVAL;
    return batch_report(c, buf, len);
}

void mehdg_destroy(mehdg_ctx* c) {
    if (!c) return;
    free_mesh(c);
    prof_free(&c->prof);
    delete c;
}

int mehdg_profile_enable(mehdg_ctx* c, int enable) {
    if (!c) return MEHDG_EINVAL;
    return prof_enable(&c->prof, enable) ? MEHDG_OK : MEHDG_ECUDA;
}

int mehdg_profile_read(mehdg_ctx* c, double* ms, int64_t* launches, double* flops, int nphase) {
    if (!c || !ms || !launches || !flops) return MEHDG_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return MEHDG_ECUDA;
    prof_read(&c->prof, ms, launches, flops, nphase);
    return MEHDG_OK;
}

int64_t mehdg_launch_count(void) { return (int64_t)g_mehdg_launches.load(); }

}  // extern "C"
