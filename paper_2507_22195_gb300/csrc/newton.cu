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
