// refine.cu -- vector kernels of the FP64 iterative refinement
//   x_{i+1} = x_i + LU^-1 (r - S x_i),  S x evaluated matrix-free in FP64
// (forward-mode tangent of the residual), stopped per element when
// ||r - S x|| <= tol ||r|| (2-norms over the element's unknowns).
// The LU works on node-major vectors (entry 5 A + k, padded to ld); the
// residual kernels use the component-major layout [5][Nn] of the C-ABI.
#include "kernels.cuh"

namespace {

// out[K][5A+k] = sa a[K][k Nn + A] + sb b[K][k Nn + A]; 0 in the padding
__global__ void set_rhs_kernel(int Nn, int64_t ld, const double* a, double sa, const double* b, double sb,
                               double* out) {
    int K = blockIdx.y;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ld) return;
    double v = 0.0;
    const int Nv = 5 * Nn;
    if (i < Nv) {
        const int64_t j = (i % 5) * Nn + i / 5;
        if (a) v += sa * a[(size_t)K * Nv + j];
        if (b) v += sb * b[(size_t)K * Nv + j];
    }
    out[(size_t)K * ld + i] = v;
}

// out[K][k Nn + A] = s x[K][5A+k]
__global__ void copy_unpad_kernel(int Nn, int64_t ld, const double* x, double* out, double s) {
    int K = blockIdx.y;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int Nv = 5 * Nn;
    if (j >= Nv) return;
    const int64_t i = (j % Nn) * 5 + j / Nn;
    out[(size_t)K * Nv + j] = s * x[(size_t)K * ld + i];
}

// per element: res = r - Sx; convergence test; count unconverged elements
__global__ void __launch_bounds__(256)
refine_update_kernel(int Nn, int64_t ld, const double* r, const double* Sx, double* res, double* nrm,
                     int32_t* conv, int32_t* iters, int32_t* status, double tol, int it, int last,
                     int32_t* cnt) {
    int K = blockIdx.x;
    if (conv[K]) return;
    const int Nv = 5 * Nn;
    __shared__ double red[2][8];
    double s_r = 0.0, s_e = 0.0;
    for (int i = threadIdx.x; i < Nv; i += blockDim.x) {
        double rv = r[(size_t)K * ld + i];
        double e = rv - Sx[(size_t)K * Nv + (i % 5) * Nn + i / 5];
        res[(size_t)K * ld + i] = e;
        s_r += rv * rv; s_e += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_r += __shfl_xor_sync(0xffffffffu, s_r, o);
        s_e += __shfl_xor_sync(0xffffffffu, s_e, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s_r; red[1][threadIdx.x >> 5] = s_e; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { a += red[0][w]; b += red[1][w]; }
        a = sqrt(a); b = sqrt(b);
        nrm[2 * K] = a; nrm[2 * K + 1] = b;
        iters[K] = it + 1;
        if (b <= tol * a || a == 0.0) conv[K] = 1;
        else if (!isfinite(b)) { conv[K] = 1; if (status[K] == 0) status[K] = MEHDG_ENOCONV; }
        else if (last) { if (status[K] == 0) status[K] = MEHDG_ENOCONV; }
        else atomicAdd(cnt, 1);
    }
}

__global__ void axpy_kernel(int64_t ld, const double* dx, double* x, const int32_t* conv) {
    int K = blockIdx.y;
    if (conv && conv[K]) return;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ld) x[(size_t)K * ld + i] += dx[(size_t)K * ld + i];
}

}  // namespace

cudaError_t launch_set_rhs(int64_t nK, int Nv, int64_t ld, int Nn, const double* a, double sa, const double* b,
                           double sb, double* out, cudaStream_t st) {
    (void)Nv;
    dim3 g((unsigned)((ld + 255) / 256), (unsigned)nK);
    set_rhs_kernel<<<g, 256, 0, st>>>(Nn, ld, a, sa, b, sb, out);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_unpad(int64_t nK, int Nv, int64_t ld, const double* x, double* out, double s,
                              cudaStream_t st) {
    dim3 g((unsigned)((Nv + 255) / 256), (unsigned)nK);
    copy_unpad_kernel<<<g, 256, 0, st>>>(Nv / 5, ld, x, out, s);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t nK, int64_t ld, const double* dx, double* x, const int32_t* conv, cudaStream_t st) {
    dim3 g((unsigned)((ld + 255) / 256), (unsigned)nK);
    axpy_kernel<<<g, 256, 0, st>>>(ld, dx, x, conv);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

cudaError_t launch_refine_update(int64_t nK, int Nv, int64_t ld, const double* r, const double* Sx,
                                 double* res, double* nrm, int32_t* conv, int32_t* iters, int32_t* status,
                                 double tol, int it, int last, const double*, double*, int32_t* cnt,
                                 cudaStream_t st) {
    refine_update_kernel<<<(unsigned)nK, 256, 0, st>>>(Nv / 5, ld, r, Sx, res, nrm, conv, iters, status, tol, it,
                                                         last, cnt);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}
