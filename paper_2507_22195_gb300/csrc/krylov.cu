// krylov.cu -- the global trace solve of Algorithm 1: sum_K A-hat^K dVhat =
// bhat (eqs. R5a/R5b summed over the elements) by restarted GMRES, matrix-free
// through mehdg_apply_condensed (the products y1..y4 of Sec. 6.3).  The paper
// leaves the preconditioner out of its statement of the method; none is used.
//
// The trace vectors ([G][5][n^2] doubles) and the Arnoldi basis live on the
// device (the basis in the context, allocated on first use); orthogonalisation
// is classical Gram-Schmidt applied twice, so each Arnoldi step needs two
// batched multi-dot reductions (deterministic two-pass sums) instead of j+1
// dependent ones.  The small Hessenberg matrix, its Givens rotations and the
// triangular solve of each cycle are host arithmetic on a few hundred numbers.
#include <cmath>
#include <cstdio>
#include <vector>
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 512;

// partial[j][b] = sum over block b's share of V_j . w  (j < k)
__global__ void __launch_bounds__(RED_THREADS)
multi_dot_kernel(const double* __restrict__ V, int64_t ldv, int k, const double* __restrict__ w, int64_t n,
                 double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < k; ++j) {
        const double* v = V + (size_t)j * ldv;
        double s = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_THREADS)
            s += v[i] * w[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < RED_THREADS / 32; ++i) t += red[i];
            partial[(size_t)j * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[j] = sum_b partial[j][b], in a fixed order (one warp per j)
__global__ void finish_dot_kernel(const double* __restrict__ partial, int nb, int k, double* __restrict__ out) {
    const int j = blockIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += partial[(size_t)j * nb + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[j] = s;
}

// w += alpha * sum_j V_j c[j]  (c on the device, j < k)
__global__ void gemv_add_kernel(const double* __restrict__ V, int64_t ldv, int k, const double* __restrict__ c,
                                double alpha, double* __restrict__ w, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += V[(size_t)j * ldv + i] * c[j];
        w[i] += alpha * s;
    }
}

// y = a x + b y (y is not read when b = 0: the basis slots start uninitialised)
__global__ void axpby_kernel(double a, const double* x, double b, double* y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

extern "C" int mehdg_solve_condensed(mehdg_ctx* c, const double* bhat, double* x, double rtol, int restart,
                                     int max_iter, int* iters_out, double* relres_out, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->condensed) { set_err(c, "solve_condensed before condense"); return MEHDG_ESTATE; }
    if (!bhat || !x || restart < 1 || max_iter < 1 || !(rtol > 0.0)) return MEHDG_EINVAL;
    return gmres_trace(c, mehdg_apply_condensed, bhat, x, rtol, restart, max_iter, iters_out, relres_out, stream);
}

int gmres_trace(mehdg_ctx* c, trace_op_fn op, const double* bhat, double* x, double rtol, int restart, int max_iter,
                int* iters_out, double* relres_out, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int m = restart;
    const int64_t n = ctx_trace_len(c);
    // workspace: basis V [m+1][n], w [n], partial sums, small device arrays
    const size_t need = sizeof(double) * ((size_t)(m + 2) * n + (size_t)(m + 1) * RED_BLOCKS + 2 * (m + 1));
    if (c->krylov_bytes < need) {
        if (c->d_krylov) cudaFree(c->d_krylov);
        c->d_krylov = nullptr; c->krylov_bytes = 0;
        if (cudaMalloc(&c->d_krylov, need) != cudaSuccess) { set_err(c, "solve_condensed: out of memory"); return MEHDG_ENOMEM; }
        c->krylov_bytes = need;
    }
    double* V = reinterpret_cast<double*>(c->d_krylov);
    double* w = V + (size_t)(m + 1) * n;
    double* part = w + n;
    double* dsm = part + (size_t)(m + 1) * RED_BLOCKS;      // device: dots / coefficients
    const unsigned gv = grid_for(n);
    auto dots = [&](int k, const double* vec, std::vector<double>& out) -> int {
        multi_dot_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(V, n, k, vec, n, part);
        finish_dot_kernel<<<k, 32, 0, st>>>(part, RED_BLOCKS, k, dsm);
        MEHDG_COUNT(2);
        out.assign(k, 0.0);
        if (cudaMemcpyAsync(out.data(), dsm, sizeof(double) * k, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return MEHDG_ECUDA;
        return MEHDG_OK;
    };
    // squared norm of a vector through the first basis slot's machinery
    auto norm = [&](const double* vec, double& nr) -> int {
        multi_dot_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(vec, n, 1, vec, n, part);
        finish_dot_kernel<<<1, 32, 0, st>>>(part, RED_BLOCKS, 1, dsm);
        MEHDG_COUNT(2);
        double s = 0.0;
        if (cudaMemcpyAsync(&s, dsm, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return MEHDG_ECUDA;
        nr = std::sqrt(s);
        return MEHDG_OK;
    };
    int rc;
    double bn;
    if ((rc = norm(bhat, bn))) return rc;
    if (bn == 0.0) bn = 1.0;
    // r = b - A x into V_0
    if ((rc = op(c, x, V, stream))) return rc;
    axpby_kernel<<<gv, 256, 0, st>>>(1.0, bhat, -1.0, V, n);
    MEHDG_COUNT(1);
    double beta;
    if ((rc = norm(V, beta))) return rc;
    int it = 0;
    double res = beta / bn;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h1, h2;
    while (res > rtol && it < max_iter) {
        axpby_kernel<<<gv, 256, 0, st>>>(0.0, V, 1.0 / beta, V, n);    // V_0 = r / beta
        MEHDG_COUNT(1);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m && it < max_iter; ++j) {
            double* vj1 = V + (size_t)(j + 1) * n;
            if ((rc = op(c, V + (size_t)j * n, w, stream))) return rc;
            ++it;
            // classical Gram-Schmidt, twice
            if ((rc = dots(j + 1, w, h1))) return rc;
            if (cudaMemcpyAsync(dsm, h1.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return MEHDG_ECUDA;
            gemv_add_kernel<<<gv, 256, 0, st>>>(V, n, j + 1, dsm, -1.0, w, n);
            if ((rc = dots(j + 1, w, h2))) return rc;
            if (cudaMemcpyAsync(dsm, h2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return MEHDG_ECUDA;
            gemv_add_kernel<<<gv, 256, 0, st>>>(V, n, j + 1, dsm, -1.0, w, n);
            MEHDG_COUNT(2);
            double hn;
            if ((rc = norm(w, hn))) return rc;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h1[i] + h2[i];
            H[(size_t)(j + 1) * m + j] = hn;
            axpby_kernel<<<gv, 256, 0, st>>>(hn > 0.0 ? 1.0 / hn : 0.0, w, 0.0, vj1, n);
            MEHDG_COUNT(1);
            // previous rotations on the new column, then a new rotation
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            const double r = std::hypot(a, b);
            cs[j] = r > 0.0 ? a / r : 1.0;
            sn[j] = r > 0.0 ? b / r : 0.0;
            H[(size_t)j * m + j] = r;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res = std::fabs(g[j + 1]) / bn;
            if (res <= rtol || hn == 0.0) { ++j; break; }
        }
        // y = H^-1 g (upper triangular, size j), x += V y
        std::vector<double> y(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
        }
        if (j > 0) {
            if (cudaMemcpyAsync(dsm, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return MEHDG_ECUDA;
            gemv_add_kernel<<<gv, 256, 0, st>>>(V, n, j, dsm, 1.0, x, n);
            MEHDG_COUNT(1);
        }
        // true residual for the restart (and the reported value)
        if ((rc = op(c, x, V, stream))) return rc;
        axpby_kernel<<<gv, 256, 0, st>>>(1.0, bhat, -1.0, V, n);
        MEHDG_COUNT(1);
        if ((rc = norm(V, beta))) return rc;
        res = beta / bn;
        if (beta == 0.0) break;
    }
    if (cudaGetLastError() != cudaSuccess) return MEHDG_ECUDA;
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = res;
    if (res > rtol) {
        set_err(c, "solve_condensed: relative residual %.3e after %d products (tolerance %.1e)", res, it, rtol);
        return MEHDG_ENOCONV;
    }
    return MEHDG_OK;
}
