// newton.cu -- the nonlinear loop around the local steps: inexact Newton with
// pseudo-transient continuation (Sec. 6.1, eqs. C31221-C31223).
//
// Every pseudo-time step k solves the linearised system of eq. C312 for the
// state V_k = (Q, V, V-hat) with the stage term (u(v) - u(v_k)) / tau_k of
// eq. C242 (one stage, v* = v_k), through Algorithm 1: condensation (local),
// the global trace solve (restarted GMRES on sum_K A-hat^K), and recovery
// (local); then V_{k+1} = V_k + dV (eq. C31223).  The step tau grows with the
// residual (switched evolution relaxation: tau_{k+1} = tau_k ||R_k|| /
// ||R_{k+1}||, at most tau_max), starting from tau_init; ||R|| is the steady
// residual (Q, V and V-hat rows) at the iterate, which is the residual with
// the stage term at v* = v.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int NRM_THREADS = 256;
constexpr int NRM_BLOCKS = 256;

// partial[b] = sum of x[i]^2 over block b's share (fixed order per block)
__global__ void __launch_bounds__(NRM_THREADS)
sumsq_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
    __shared__ double red[NRM_THREADS / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NRM_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * NRM_THREADS)
        s += x[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < NRM_THREADS / 32; ++i) t += red[i];
        partial[blockIdx.x] = t;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += partial[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

// y += x
__global__ void add_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

__global__ void sub_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] -= x[i];
}
__global__ void axpy_s_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

unsigned grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

struct NewtonWork {
    double *vstar, *RV, *RQ, *RH, *bhat, *dvh, *dV, *dQ, *part, *sums;
};

// layout of the workspace (kept in the context after the first call)
size_t newton_layout(const mehdg_ctx* c, NewtonWork* w, unsigned char* base) {
    const int64_t nv = ctx_state_len(c), nq = c->prm.viscous ? 3 * nv : 0;
    const int64_t nt = ctx_trace_len(c);
    size_t off = 0;
    auto take = [&](double*& p, int64_t count) {
        p = base ? reinterpret_cast<double*>(base + off) : nullptr;
        off += ((size_t)count * sizeof(double) + 255) & ~(size_t)255;
    };
    take(w->vstar, nv); take(w->RV, nv); take(w->RQ, nq > 0 ? nq : 1); take(w->RH, nt); take(w->bhat, nt);
    take(w->dvh, nt); take(w->dV, nv); take(w->dQ, nq > 0 ? nq : 1); take(w->part, 3 * NRM_BLOCKS);
    take(w->sums, 4);
    return off;
}

#define NTRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return MEHDG_ECUDA; } } while (0)

// ||R||^2 over the steady residual rows at the state set in the context
int residual_norm(mehdg_ctx* c, const NewtonWork& w, double* out, cudaStream_t st) {
    int rc = mehdg_residual(c, w.RV, c->prm.viscous ? w.RQ : nullptr, w.RH, st);
    if (rc) return rc;
    const int64_t nv = ctx_state_len(c), nt = ctx_trace_len(c);
    const double* arr[3] = {w.RV, w.RH, c->prm.viscous ? w.RQ : nullptr};
    const int64_t len[3] = {nv, nt, 3 * nv};
    for (int a = 0; a < 3; ++a) {
        if (!arr[a]) {
            NTRY(cudaMemsetAsync(w.sums + a, 0, sizeof(double), st));
            continue;
        }
        sumsq_kernel<<<NRM_BLOCKS, NRM_THREADS, 0, st>>>(arr[a], len[a], w.part + a * NRM_BLOCKS);
        sum_partials_kernel<<<1, 32, 0, st>>>(w.part + a * NRM_BLOCKS, NRM_BLOCKS, w.sums + a);
        MEHDG_COUNT(2);
    }
    double h[3];
    NTRY(cudaMemcpyAsync(h, w.sums, sizeof(h), cudaMemcpyDeviceToHost, st));
    NTRY(cudaStreamSynchronize(st));
    *out = std::sqrt(h[0] + h[1] + h[2]);
    return MEHDG_OK;
}

}  // namespace

cudaError_t launch_add(const double* x, double* y, int64_t n, cudaStream_t st) {
    add_kernel<<<grid_n(n), 256, 0, st>>>(x, y, n);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

extern "C" int mehdg_set_source(mehdg_ctx* c, const double* src) {
    if (!c) return MEHDG_EINVAL;
    if (c->batch) { set_err(c, "set_source: not available for elements of uneven p, m"); return MEHDG_EINVAL; }
    c->src = src;
    c->condensed = false;
    return MEHDG_OK;
}

namespace {

// out = (u(va_h) - u(vb_h), w): the stage term at dt = 1, as the difference of
// two residual evaluations whose other terms are identical
int stage_difference(mehdg_ctx* c, const double* va, const double* vb, double* out, double* tmp, cudaStream_t st) {
    ResidualArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tab = c->tab; a.ph = c->ph; a.box = c->d_box; a.gid = c->d_gid;
    a.ph.inv_dt = 1.0; a.ph.time_term = 1;
    a.vh = c->vh; a.q = c->q; a.status = c->d_status;
    a.RH = c->d_tRHloc2;
    a.v = va; a.vs = vb; a.RV = out;
    NTRY(launch_residual(a, c->nK, c->prm.viscous != 0, false, st));
    a.vs = va; a.RV = tmp;
    NTRY(launch_residual(a, c->nK, c->prm.viscous != 0, false, st));
    const int64_t nv = c->nK * (int64_t)c->Nv;
    sub_kernel<<<grid_n(nv), 256, 0, st>>>(tmp, out, nv);
    MEHDG_COUNT(1);
    NTRY(cudaGetLastError());
    return MEHDG_OK;
}

// Butcher table of the three-stage, third-order, L-stable, stiffly accurate
// DIRK method of Alexander: alpha is the root of x^3 - 3x^2 + 3/2 x - 1/6 in
// (1/6, 1/2) (found by bisection); D = A^-1 (lower triangular)
void dirk33_D(double D[3][3]) {
    double lo = 1.0 / 6.0, hi = 0.5;
    auto f = [](double x) { return x * x * x - 3.0 * x * x + 1.5 * x - 1.0 / 6.0; };
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (f(lo) * f(mid) <= 0.0) hi = mid; else lo = mid;
    }
    const double al = 0.5 * (lo + hi), t2 = 0.5 * (1.0 + al);
    const double b1 = -(6.0 * al * al - 16.0 * al + 1.0) / 4.0, b2 = (6.0 * al * al - 20.0 * al + 5.0) / 4.0;
    const double A[3][3] = {{al, 0, 0}, {t2 - al, al, 0}, {b1, b2, al}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i][j] = 0.0;
    for (int j = 0; j < 3; ++j) {         // column j of A^-1 by forward substitution
        for (int i = 0; i < 3; ++i) {
            double s = i == j ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= A[i][k] * D[k][j];
            D[i][j] = s / A[i][i];
        }
    }
}

}  // namespace

extern "C" int mehdg_dirk_step(mehdg_ctx* c, double* v, double* vhat, double* q, double dt, double newton_tol,
                               int newton_max, double lin_rtol, int restart, int max_iter, int* newton_iters,
                               double* res_norms, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0) { set_err(c, "dirk_step before set_mesh"); return MEHDG_ESTATE; }
    if (c->batch || !c->prm.time_term) { set_err(c, "dirk_step: one element type, with the stage term"); return MEHDG_EINVAL; }
    if (!v || !vhat || (c->prm.viscous && !q) || !(dt > 0.0) || !(newton_tol > 0.0) || newton_max < 1 ||
        !(lin_rtol > 0.0) || restart < 1 || max_iter < 1) {
        set_err(c, "dirk_step: bad arguments");
        return MEHDG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    NewtonWork w;
    const size_t need = newton_layout(c, &w, nullptr);
    if (c->newton_bytes < need) {
        if (c->d_newton) cudaFree(c->d_newton);
        c->d_newton = nullptr; c->newton_bytes = 0;
        if (cudaMalloc(&c->d_newton, need) != cudaSuccess) { set_err(c, "dirk_step: out of memory"); return MEHDG_ENOMEM; }
        c->newton_bytes = need;
    }
    newton_layout(c, &w, reinterpret_cast<unsigned char*>(c->d_newton));
    const int64_t nv = c->nK * (int64_t)c->Nv, nt = c->G * 5 * (int64_t)c->tab.n2, nq = 3 * nv;
    // v^n, the stages, the source and a difference buffer
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, sizeof(double) * 7 * (size_t)nv) != cudaSuccess) {
        set_err(c, "dirk_step: out of memory"); return MEHDG_ENOMEM;
    }
    double *vn = buf, *stg = buf + nv, *src = buf + 4 * nv, *dif = buf + 5 * nv, *tmp = buf + 6 * nv;
    const double dt0 = c->prm.dt;
    double D[3][3];
    dirk33_D(D);
    auto done = [&](int rc) {
        c->src = nullptr;
        mehdg_set_dt(c, dt0);
        cudaFree(buf);
        // the context's v* and source pointed into the freed buffer
        c->v = nullptr; c->vh = nullptr; c->vs = nullptr; c->q = nullptr; c->condensed = false;
        return rc;
    };
#define DTRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return done(MEHDG_ECUDA); } } while (0)
#define DRC(x) do { int r_ = (x); if (r_) return done(r_); } while (0)
    DTRY(cudaMemcpyAsync(vn, v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    DRC(mehdg_set_state(c, v, vhat, q, vn, stream));
    for (int i = 0; i < 3; ++i) {
        // known stages: src = sum_{j<i} (d_ij / dt) (u(v^{n,j}) - u(v^n), w)
        DTRY(cudaMemsetAsync(src, 0, sizeof(double) * nv, st));
        for (int j = 0; j < i; ++j) {
            DRC(stage_difference(c, stg + (size_t)j * nv, vn, dif, tmp, st));
            axpy_s_kernel<<<grid_n(nv), 256, 0, st>>>(D[i][j] / dt, dif, src, nv);
            MEHDG_COUNT(1);
        }
        DRC(mehdg_set_dt(c, dt / D[i][i]));
        DRC(mehdg_set_source(c, i > 0 ? src : nullptr));
        int it = 0;
        double rn = 0.0;
        for (;; ++it) {
            DRC(mehdg_set_state(c, v, vhat, q, vn, stream));
            DRC(residual_norm(c, w, &rn, st));
            if (!std::isfinite(rn)) { set_err(c, "dirk_step: non-finite residual in stage %d", i); return done(MEHDG_ENONPHYS); }
            if (rn <= newton_tol || it == newton_max) break;
            DRC(mehdg_condense(c, w.bhat, nullptr, stream));
            DTRY(cudaMemsetAsync(w.dvh, 0, sizeof(double) * nt, st));
            DRC(mehdg_solve_condensed(c, w.bhat, w.dvh, lin_rtol, restart, max_iter, nullptr, nullptr, stream));
            DRC(mehdg_recover(c, w.dvh, w.dV, c->prm.viscous ? w.dQ : nullptr, stream));
            add_kernel<<<grid_n(nv), 256, 0, st>>>(w.dV, v, nv);
            add_kernel<<<grid_n(nt), 256, 0, st>>>(w.dvh, vhat, nt);
            MEHDG_COUNT(2);
            if (c->prm.viscous) { add_kernel<<<grid_n(nq), 256, 0, st>>>(w.dQ, q, nq); MEHDG_COUNT(1); }
            DTRY(cudaGetLastError());
        }
        if (newton_iters) newton_iters[i] = it;
        if (res_norms) res_norms[i] = rn;
        if (rn > newton_tol) { set_err(c, "dirk_step: stage %d residual %.3e after %d Newton steps", i, rn, it); return done(MEHDG_ENOCONV); }
        DTRY(cudaMemcpyAsync(stg + (size_t)i * nv, v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    }
    DTRY(cudaStreamSynchronize(st));
    // stiffly accurate: u^{n+1} = u^{n,3}, already in (v, vhat, q)
    return done(MEHDG_OK);
#undef DTRY
#undef DRC
}

extern "C" int mehdg_set_dt(mehdg_ctx* c, double dt) {
    if (!c) return MEHDG_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) { set_err(c, "set_dt: dt must be positive and finite"); return MEHDG_EINVAL; }
    c->prm.dt = dt;
    c->ph.inv_dt = c->prm.time_term ? 1.0 / dt : 0.0;
    c->condensed = false;       // the Jacobian changes with the stage term
    c->pj_ready = false;
    return c->batch ? batch_set_dt(c) : MEHDG_OK;
}

extern "C" int mehdg_pseudo_time_newton(mehdg_ctx* c, double* v, double* vhat, double* q, int nsteps,
                                        double tau_init, double tau_max, double lin_rtol, int restart,
                                        int max_iter, double* res_norms, double* taus, int* lin_iters,
                                        void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (c->nK == 0) { set_err(c, "pseudo_time_newton before set_mesh"); return MEHDG_ESTATE; }
    if (!c->prm.time_term) { set_err(c, "pseudo_time_newton needs a context with the stage term"); return MEHDG_EINVAL; }
    if (!v || !vhat || (c->prm.viscous && !q) || nsteps < 0 || !(tau_init > 0.0) || !(tau_max >= tau_init) ||
        !(lin_rtol > 0.0) || restart < 1 || max_iter < 1) {
        set_err(c, "pseudo_time_newton: bad arguments");
        return MEHDG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    NewtonWork w;
    const size_t need = newton_layout(c, &w, nullptr);
    if (c->newton_bytes < need) {
        if (c->d_newton) cudaFree(c->d_newton);
        c->d_newton = nullptr; c->newton_bytes = 0;
        if (cudaMalloc(&c->d_newton, need) != cudaSuccess) { set_err(c, "pseudo_time_newton: out of memory"); return MEHDG_ENOMEM; }
        c->newton_bytes = need;
    }
    newton_layout(c, &w, reinterpret_cast<unsigned char*>(c->d_newton));
    const int64_t nv = ctx_state_len(c), nt = ctx_trace_len(c);
    const double dt0 = c->prm.dt;
    // the residual at the start of a step is the steady one: v* = v
    auto at_state = [&]() -> int {
        NTRY(cudaMemcpyAsync(w.vstar, v, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        return mehdg_set_state(c, v, vhat, q, w.vstar, stream);
    };
    int rc;
    double rn = 0.0, tau = tau_init;
    if ((rc = at_state())) return rc;
    if ((rc = residual_norm(c, w, &rn, st))) return rc;
    if (res_norms) res_norms[0] = rn;
    for (int k = 0; k < nsteps; ++k) {
        if (taus) taus[k] = tau;
        if ((rc = mehdg_set_dt(c, tau))) return rc;
        if ((rc = at_state())) return rc;
        if ((rc = mehdg_condense(c, w.bhat, nullptr, stream))) return rc;
        NTRY(cudaMemsetAsync(w.dvh, 0, sizeof(double) * nt, st));
        int its = 0;
        double rr = 0.0;
        rc = mehdg_solve_condensed(c, w.bhat, w.dvh, lin_rtol, restart, max_iter, &its, &rr, stream);
        if (lin_iters) lin_iters[k] = its;
        if (rc) return rc;
        if ((rc = mehdg_recover(c, w.dvh, w.dV, c->prm.viscous ? w.dQ : nullptr, stream))) return rc;
        add_kernel<<<grid_n(nv), 256, 0, st>>>(w.dV, v, nv);
        add_kernel<<<grid_n(nt), 256, 0, st>>>(w.dvh, vhat, nt);
        MEHDG_COUNT(2);
        if (c->prm.viscous) {
            add_kernel<<<grid_n(3 * nv), 256, 0, st>>>(w.dQ, q, 3 * nv);
            MEHDG_COUNT(1);
        }
        NTRY(cudaGetLastError());
        const double rprev = rn;
        if ((rc = at_state())) return rc;
        if ((rc = residual_norm(c, w, &rn, st))) return rc;
        if (res_norms) res_norms[k + 1] = rn;
        if (!std::isfinite(rn)) { set_err(c, "pseudo_time_newton: non-finite residual after step %d", k); return MEHDG_ENONPHYS; }
        tau = rn > 0.0 ? std::fmin(tau_max, tau * rprev / rn) : tau_max;
    }
    // leave the context at the final state, with the caller's step size
    if ((rc = mehdg_set_dt(c, dt0))) return rc;
    return at_state();
}
