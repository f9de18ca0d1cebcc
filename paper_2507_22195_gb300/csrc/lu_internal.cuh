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

// A B panel already packed in split BF16 by a TRSM product: per element nc
// rows (one per column of the trailing matrix), each [hi (kp) | lo (kp)];
// this update's first column is row c0 of it.
struct PackedB {
    const void* p = nullptr;
    int nc = 0, c0 = 0, kp = 0;
};
// Rows of the A operand taken from other rows of S for their first kn K
// entries: slot i in [i0, i1) of a net permutation (rows[i] takes the old
// content of rows[cont[i]]) with cont[i] != i gives operand row rows[i] the
// values of row rows[cont[i]] (the deferred update's first-half multipliers,
// which the second half's exchanges did not move).
struct AGather {
    const int32_t* perm = nullptr;   // [nK][LU_PW]
    int kn = 0, i0 = 0, i1 = 0;
};
// An A operand already packed in split BF16 (the fourth operand panel): per
// element erows rows of [hi (kp) | lo (kp)]; this update's first row is row
// row0 of it.
struct PackedA {
    const void* p = nullptr;
    int erows = 0, row0 = 0, kp = 0;
};
// The TRSM product's copy of U12 as the next update's B operand (split BF16):
// per element nc rows of [hi (kp) | lo (kp)]; product column n goes to row
// c0 + n, its K index k (the row inside the 256 block) to entry k0 + k.  Given
// to an update (split BF16), C - D goes instead to FP32 rows of kp entries
// (row c0 + n, entry k0 + k: the next TRSM product's B operand) and S is not
// written.
struct BqOut {
    void* p = nullptr;
    int nc = 0, c0 = 0, k0 = 0, kp = 0;
};

// C[r0.., c0..] -= L[r0.., k0..k0+Kd) * U[k0..k0+Kd, c0..] on the tensor cores
// (TF32 or BF16 operands, FP32 accumulation), S^K column-major FP32.
// With ph_gemm >= 0 the update kernel alone is timed under that phase (flops
// recorded with it) and the operand packing under ph_pack.
// b: the B panel already packed (split BF16) by a TRSM product, or null;
// g: A rows gathered through a net permutation, or null
// out: the result as the next TRSM's FP32 B operand instead of into S, or null;
// a: the A operand already packed (then g must be null), or null
cudaError_t gemm_tc_update(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st,
                           int ph_pack = -1, int ph_gemm = -1, double flops = 0.0, const PackedB* b = nullptr,
                           const AGather* g = nullptr, const BqOut* out = nullptr, const PackedA* a = nullptr);
// The fourth operand panel (split BF16 only): the multipliers of a pair of
// outer panels, packed once for the three updates of the pair
void* gemm_tc_a2_panel(const LUPlan& P);
// Rows [r0, r0+M) of S's columns [k0, k0+Kd) (Kd a multiple of 32) into it: per
// element erows rows of [hi (kp) | lo (kp)], S row r0 + m at row row0 + m, K
// entries kout.. kout+Kd
cudaError_t gemm_tc_pack_a2(const LUPlan& P, int erows, int row0, int kp, int kout, int r0, int k0, int M, int Kd,
                            cudaStream_t st);
// Its rows re-packed through a net permutation (row 0 = S row r0; K entries
// 0..g.kn from S's columns k0..)
cudaError_t gemm_tc_gather_a2(const LUPlan& P, int erows, int kp, int r0, int k0, const AGather& g, cudaStream_t st);
size_t gemm_tc_work_bytes(int64_t nK, int64_t ld, int prec);
// The next update's B panel of the split-BF16 mode (written by the TRSM products)
void* gemm_tc_bq_panel(const LUPlan& P);
// The TRSM's FP32 B panel ([nK][columns][256] floats; the product splits it)
void* gemm_tc_bp_panel(const LUPlan& P);
// Row exchanges of the columns right of outer panel c0 by its net permutation
// (perm: [nK][LU_PW]) and the TRSM of their rows [c0, c0+256), fused.  bq:
// where the product also writes U12 as split-BF16 B operand (null: not
// written; only the split-BF16 mode has it).
cudaError_t gemm_tc_swap_trsm256(const LUPlan& P, const int32_t* perm, int c0, cudaStream_t st, const BqOut* bq);
// The TRSM of rows [c0, c0+256) of the columns right of them, with its B
// operand already in the FP32 B panel (written by an update with out set)
cudaError_t gemm_tc_trsm256(const LUPlan& P, int c0, cudaStream_t st, const BqOut* bq);
cudaError_t gemm_simt_update_f32(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st);
