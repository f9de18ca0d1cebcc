// gemm_tc.cu -- trailing update of the mixed-precision LU (placeholder: SIMT FP32)
#include "lu_internal.cuh"

cudaError_t gemm_tc_update(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st) {
    return gemm_simt_update_f32(P, r0, c0, k0, M, N, Kd, st);
}
size_t gemm_tc_work_bytes(int64_t, int64_t, int) { return 0; }
