// lu_internal.cuh -- pieces shared by lu.cu and gemm_tc.cu
#pragma once
#include "kernels.cuh"

constexpr int LU_NB = 256;   // outer panel width (depth of the big trailing update)
constexpr int LU_PW = 1 + 4 * LU_NB;   // ints of one net permutation: nr, rows[2 NB], cont[2 NB]

// workspace layout: [inner permutation scratch][outer-panel permutations][operand panels]
// The outer-panel permutations ([ld/NB][nK][LU_PW]) are kept for the solves.
inline size_t lu_perm_scratch_bytes(int64_t nK) { return ((size_t)nK * LU_PW * 4 + 255) & ~(size_t)255; }
inline size_t lu_perm_panels_bytes(int64_t nK, int64_t ld) {
    return ((size_t)(ld / LU_NB) * nK * LU_PW * 4 + 255) & ~(size_t)255;
}
inline size_t lu_perm_bytes(int64_t nK, int64_t ld) { return lu_perm_scratch_bytes(nK) + lu_perm_panels_bytes(nK, ld); }

// C[r0.., c0..] -= L[r0.., k0..k0+Kd) * U[k0..k0+Kd, c0..] on the tensor cores
// (TF32 or BF16 operands, FP32 accumulation), S^K column-major FP32.
// With ph_gemm >= 0 the update kernel alone is timed under that phase (flops
// recorded with it) and the operand packing under ph_pack.
// b_packed: the B panel already packed (split BF16) by the TRSM product, or null
cudaError_t gemm_tc_update(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st,
                           int ph_pack = -1, int ph_gemm = -1, double flops = 0.0, const void* b_packed = nullptr);
size_t gemm_tc_work_bytes(int64_t nK, int64_t ld, int prec);
// row exchanges of the columns right of outer panel c0 by its net permutation
// (perm: [nK][LU_PW]) and the TRSM of their rows [c0, c0+256), fused
// (update_b, if not null, receives the next update's packed B panel, or null
// when the precision mode does not fuse it)
cudaError_t gemm_tc_swap_trsm256(const LUPlan& P, const int32_t* perm, int c0, cudaStream_t st,
                                 const void** update_b);
cudaError_t gemm_simt_update_f32(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st);
