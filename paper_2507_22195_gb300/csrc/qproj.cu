// qproj.cu -- the gradient-equation operators of the viscous condensation
// (eqs. R2, R3, R5, R6), matrix-free along grid lines:
//   out = alpha A_qq^-1 Rq + beta A_qq^-1 A_qv x + gamma A_qq^-1 A_qvhat xh
// (all q-shaped [nK][5][3][Nn]).  With A_qq = I_15 (x) M, M = M1_x (x) M1_y (x) M1_z
// (exact Gauss quadrature on the tensor grid) and A_qv of the weak gradient,
// these become 1-D operators along the lines of the macro-element:
//   A_qq^-1 Rq          : M1_d^-1 = (2/h_d) Minv_ref applied along x, y and z;
//   A_qq^-1 A_qv x      : component (l,d) = (2/h_d) C1_ref applied to x_l along d;
//   A_qq^-1 A_qvhat xh  : component (l,d) = -(2/h_d) sum_sides s Minv_ref[a_d][i_side] xh_l,
//                         the trace of the two faces normal to d spread along their normal lines.
#include "kernels.cuh"

namespace {

__device__ __forceinline__ double inv_half_h(const double* box, int K, int d, int m) {
    return 2.0 * m / (box[6 * K + 3 + d] - box[6 * K + d]);
}

// out[K][c][a] = alpha (2/h_d) sum_j Minv[a_d][j] in[K][c][a with a_d = j], 15 components
__global__ void line_minv_kernel(const double* __restrict__ in, double* __restrict__ out, int d,
                                 const double* __restrict__ Minv, const double* __restrict__ box, int m, int n,
                                 int64_t nK, double alpha, const int32_t* skip) {
    const int64_t Nn = (int64_t)n * n * n;
    const int64_t per = 15 * Nn;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nK * per) return;
    const int64_t K = idx / per, r = idx % per;
    if (skip && skip[K]) return;
    const int64_t c = r / Nn, a = r % Nn;
    int co[3] = {(int)(a % n), (int)((a / n) % n), (int)(a / (n * n))};
    const int ad = co[d];
    const int64_t stride = d == 0 ? 1 : (d == 1 ? n : (int64_t)n * n);
    const int64_t base = a - (int64_t)ad * stride;
    const double* src = in + (size_t)K * per + (size_t)c * Nn;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += Minv[ad * n + j] * src[base + j * stride];
    out[idx] = alpha * inv_half_h(box, (int)K, d, m) * s;
}

// out[K][l*3+d][a] (+)= beta (2/h_d) sum_j C1[a_d][j] x[K][l][a(a_d=j)]
//                     + gamma (2/h_d) sum_{sides} (-s) Minv[a_d][i_side] xh_side[l][a_perp]
__global__ void qgrad_kernel(const double* __restrict__ x, double beta, const double* __restrict__ xh, double gamma,
                             const int64_t* __restrict__ gid, const double* __restrict__ C1,
                             const double* __restrict__ Minv, const double* __restrict__ box, int m, int n,
                             int64_t nK, double* __restrict__ out, int accumulate, const int32_t* skip) {
    const int64_t Nn = (int64_t)n * n * n, n2 = (int64_t)n * n;
    const int64_t per = 15 * Nn;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nK * per) return;
    const int64_t K = idx / per, r = idx % per;
    if (skip && skip[K]) return;
    const int ld_ = (int)(r / Nn);
    const int l = ld_ / 3, d = ld_ % 3;
    const int64_t a = r % Nn;
    int co[3] = {(int)(a % n), (int)((a / n) % n), (int)(a / n2)};
    const int ad = co[d];
    const double sc = inv_half_h(box, (int)K, d, m);
    double val = 0.0;
    if (x) {
        const int64_t stride = d == 0 ? 1 : (d == 1 ? n : n2);
        const double* src = x + (size_t)K * 5 * Nn + (size_t)l * Nn + (a - (int64_t)ad * stride);
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += C1[ad * n + j] * src[j * stride];
        val += beta * sc * s;
    }
    if (xh) {
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const int64_t c = co[t1] + (int64_t)n * co[t2];
        double s = 0.0;
        for (int side = 0; side < 2; ++side) {
            const int64_t g = gid[6 * K + 2 * d + side];
            const int iside = side ? n - 1 : 0;
            const double sgn = side ? 1.0 : -1.0;
            s -= sgn * Minv[ad * n + iside] * xh[(size_t)g * 5 * n2 + (size_t)l * n2 + c];
        }
        val += gamma * sc * s;
    }
    out[idx] = accumulate ? out[idx] + val : val;
}

}  // namespace

cudaError_t launch_qproj(const QProjArgs& q, int64_t nK, const double* Rq, double alpha, const double* x, double beta,
                         const double* xh, double gamma, double* out, const int32_t* skip, cudaStream_t st) {
    const int n = q.tab.n, m = q.tab.m;
    const int64_t total = nK * 15 * (int64_t)q.tab.Nn;
    const int bs = 256;
    const unsigned g = (unsigned)((total + bs - 1) / bs);
    int accumulate = 0;
    if (Rq) {
        line_minv_kernel<<<g, bs, 0, st>>>(Rq, q.tmp1, 0, q.Minv, q.box, m, n, nK, 1.0, skip);
        line_minv_kernel<<<g, bs, 0, st>>>(q.tmp1, q.tmp2, 1, q.Minv, q.box, m, n, nK, 1.0, skip);
        line_minv_kernel<<<g, bs, 0, st>>>(q.tmp2, out, 2, q.Minv, q.box, m, n, nK, alpha, skip);
        MEHDG_COUNT(3);
        accumulate = 1;
    }
    if (x || xh || !accumulate) {
        qgrad_kernel<<<g, bs, 0, st>>>(x, beta, xh, gamma, q.gid, q.C1, q.Minv, q.box, m, n, nK, out, accumulate, skip);
        MEHDG_COUNT(1);
    }
    return cudaGetLastError();
}
