// kernels.cuh -- launch interfaces between the C-ABI layer and the kernels.
#pragma once
#include "common.cuh"

struct ResidualArgs {
    Tab tab;
    Phys ph;
    const double* box;        // [nK][6]
    const int64_t* gid;       // [nK][6]
    const double *v, *vs, *vh, *q;        // state (vs may be null if no time term)
    const double *dv, *dvh, *dq;          // tangent directions (null = 0)
    double *RV, *RQ, *RH;                 // values (null = skip); RH = per-element sides
    double *tRV, *tRQ, *tRH;              // tangents (tangent launches only)
    int32_t* status;
    const int32_t* skip;                  // [nK] nonzero = skip element (may be null)
    const double* pj;                     // stored point Jacobians: tangent volume pass is linear (may be null)
    const double* pjf;                    // stored face point Jacobians dFhat/dv: face pass linear when dvh = 0
    const double* pq;                     // stored viscous blocks W dG/dq [nK][m^3][225][npt] (with pj: the
                                          // viscous volume tangent is linear in dv and dq)
    const double* pqf;                    // stored viscous face blocks W dGhat/dq [nK][6 m^2][75][fpt] (with
                                          // pjf: the viscous face tangent is linear when dvh = 0)
};

cudaError_t launch_residual(const ResidualArgs& a, int64_t nK, bool visc, bool tangent, cudaStream_t st);
cudaError_t launch_trace_gather(const double* loc, const int64_t* g2l, int64_t G, int n2, double* out,
                                double alpha, const double* add, double beta, cudaStream_t st);

// gradient-equation line operators (qproj.cu), q-shaped outputs [nK][15][Nn]:
// out = alpha A_qq^-1 Rq + beta A_qq^-1 A_qv x + gamma A_qq^-1 A_qvhat xh
struct QProjArgs {
    Tab tab;
    const double* box;
    const int64_t* gid;
    const double* Minv;       // [n][n] M1_ref^-1
    const double* C1;         // [n][n] M1_ref^-1 G1_ref
    double *tmp1, *tmp2;      // [nK][15][Nn] scratch
};
cudaError_t launch_qproj(const QProjArgs& q, int64_t nK, const double* Rq, double alpha, const double* x, double beta,
                         const double* xh, double gamma, double* out, const int32_t* skip, cudaStream_t st);
void host_build_qtables(const Tab& t, double* Minv_ref, double* C1_ref);

// dense S^K assembly (col-major, leading dimension ld = Npad), element by element
struct JacobianArgs {
    Tab tab;
    Phys ph;
    const double* box;
    const double *v, *vs, *vh, *q;
    const int64_t* gid;
    void* S;                  // float or double [nK][ld][ld]
    int64_t ld;
    int32_t* status;
    const double* C1;         // [n][n] M1_ref^-1 G1_ref (viscous only)
    double* pj;               // if set: the weighted FP64 point Jacobians [nK][m^3][100][npt] (inviscid)
    double* pjf;              // if set: the weighted FP64 face blocks dFhat/dv [nK][6 m^2][25][fpt] (inviscid)
    double* pq;               // if set: scratch for the viscous point blocks dG/dq [nK][m^3][225][npt]
    double* pqf;              // if set: the weighted FP64 viscous face blocks dGhat/dq [nK][6 m^2][75][fpt]
};
// phase: 1 = the point passes (stored point Jacobians only, S untouched), 2 = the passes that add
// into S (they read what phase 1 wrote), 3 = both
cudaError_t launch_jacobian(const JacobianArgs& a, int64_t nK, bool fp64, cudaStream_t st, int phase = 3);
cudaError_t launch_pad_identity(void* S, int64_t nK, int64_t ld, int Nv, bool fp64, cudaStream_t st);

// batched dense LU with partial pivoting and solves (lu.cu)
struct LUPlan {
    int64_t nK, ld, N;        // ld = padded size (multiple of 256), N = true size
    bool fp64;
    int prec;                 // mehdg_prec
    void* S;                  // factors in place
    int32_t* piv;             // [nK][ld] absolute row swapped with row i at step i
    int32_t* status;
    void* work;               // scratch (operand panels, permutation lists)
    size_t work_bytes;
    Prof* prof;
    int leaf_ctas = 0;        // leaf panel CTAs per SM: 1, 2, or 0 = chosen from the element count
    int solve_ctas = 0;       // CTAs per element in the solves: 1, 2, 4, 8, or 0 = chosen from the count
};
size_t lu_work_bytes(int64_t nK, int64_t ld, bool fp64, int prec);
cudaError_t lu_factor(const LUPlan& P, cudaStream_t st);
// solve S x = r for every element whose conv flag is 0: x (FP64) = LU^-1 r,
// computed in the factor precision; r, x: [nK][ld] FP64 (padded tail 0).
cudaError_t lu_solve(const LUPlan& P, const double* r, double* x, const int32_t* skip, cudaStream_t st);
// the transposed system S^T x = r with the same factors (FP64 accumulation)
cudaError_t lu_solve_T(const LUPlan& P, const double* r, double* x, const int32_t* skip, cudaStream_t st);

// small vector kernels for the refinement (refine.cu)
cudaError_t launch_refine_update(int64_t nK, int Nv, int64_t ld, const double* r, const double* Sx,
                                 double* res, double* nrm, int32_t* conv, int32_t* iters, int32_t* status,
                                 double tol, int it, int last, const double* dx, double* x, int32_t* cnt,
                                 cudaStream_t st);
cudaError_t launch_set_rhs(int64_t nK, int Nv, int64_t ld, int Nn, const double* a, double sa,
                           const double* b, double sb, double* out, cudaStream_t st);
cudaError_t launch_copy_unpad(int64_t nK, int Nv, int64_t ld, const double* x, double* out, double s,
                              cudaStream_t st);

// residual VJP passes at the context's state (vjp.cu); Euler only
cudaError_t launch_vjp(mehdg_ctx* c, const double* lam_V, const double* lam_Vhat, double* g_v, double* g_vhat,
                       cudaStream_t st);
// restarted GMRES on a matrix-free trace operator (krylov.cu)
typedef int (*trace_op_fn)(mehdg_ctx* c, const double* x, double* y, void* stream);
int gmres_trace(mehdg_ctx* c, trace_op_fn op, const double* b, double* x, double rtol, int restart, int max_iter,
                int* iters_out, double* relres_out, void* stream);
// y += x (n doubles; newton.cu)
cudaError_t launch_add(const double* x, double* y, int64_t n, cudaStream_t st);
