/*
 * mehdg.h -- C-ABI of the GB300 (sm_103a) hot path of the entropy-variable
 * macro-element HDG method (Badrkhani, ten Eikelder, Hasse, Schillinger,
 * arXiv 2507.22195): the per-macro-element Newton step.
 *
 *   residual  : eq. s32 (a-c) with the one-stage implicit term of eq. C242,
 *               inviscid fluxes of eqs. Flux_En_Inv (ES), EC and ES (KEPES),
 *               viscous flux of eq. Flux_En_Vis;
 *   condense  : local Jacobian (eq. R1), Q-elimination and Schur complement
 *               (eqs. R2, R3), LU of S, right-hand side b-hat (eq. R5b);
 *   apply     : the four-stage reduced mat-vec of Sec. 6.3 (Algorithm 1,
 *               global matrix-vector product);
 *   recover   : local back-substitution, eqs. R2 and R6 (Algorithm 1,
 *               local recovery).
 *
 * Discretisation: each macro-element K is an axis-aligned box split into m^3
 * hexahedral micro-elements carrying Q_p on Gauss-Lobatto-Legendre nodes,
 * continuous inside K; tensor Gauss quadrature with p+2 points per direction
 * per micro-element (volume and faces).  n = m p + 1 nodes per direction,
 * Nn = n^3, node index A = i + n (j + n k).
 *
 * Layouts (all FP64, C-contiguous):
 *   v, v*      [nK][5][Nn]            entropy variables (eq. s222)
 *   q, R_Q, dQ [nK][5][3][Nn]         q ~ grad v (eq. s32a); viscous only
 *   R_V, dV    [nK][5][Nn]
 *   trace      [n_global_faces][5][n^2]   v-hat, R_V-hat, b-hat, dV-hat, x, y
 *              face node c = i_t1 + n i_t2, (t1,t2) = the two tangential
 *              axes in increasing order; local faces x-,x+,y-,y+,z-,z+.
 * Global trace quantities (R_V-hat, b-hat, y) are sums over the elements
 * adjacent to each global face (eq. s32c; Algorithm 1, assembly).
 *
 * Ownership: every array argument is a caller-owned pointer; the library
 * never frees it.  Pointers to state (set_state) must stay valid and
 * unchanged until the next set_state or destroy.  Arrays passed to
 * residual/condense/apply/recover are DEVICE pointers unless stated
 * otherwise; mesh arrays (set_mesh) are HOST pointers.  The context owns
 * its device workspaces (the LU factors of every S^K, pivots, residuals).
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Work is enqueued on it; condense/apply/recover
 * synchronise that stream once per refinement sweep to test convergence.
 *
 * Errors: functions return MEHDG_OK (0) or a negative code below, and keep
 * a message readable with mehdg_last_error.  Per-element failures (a
 * non-physical state, a zero pivot, refinement not converged, a device wait
 * that ran out) are also recorded per element, readable with mehdg_status.
 */
#ifndef MEHDG_H
#define MEHDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mehdg_ctx mehdg_ctx;

/* inviscid numerical flux */
typedef enum {
    MEHDG_FLUX_EC = 0,     /* entropy-conservative, kinetic-energy-preserving, eq. EC   */
    MEHDG_FLUX_ES = 1,     /* entropy-stable Lax-Friedrichs type, eq. Flux_En_Inv       */
    MEHDG_FLUX_KEPES = 2   /* KEP and entropy-stable, hybrid LF/Roe dissipation, eq. ES */
} mehdg_flux;

/* precision of the local LU and Schur products (residuals, Jacobian point
 * physics and the refinement residual are always FP64) */
typedef enum {
    MEHDG_FP64 = 0,        /* FP64 LU on the FP64 pipe                              */
    MEHDG_MIXED_TF32 = 1,  /* FP32 storage, TF32 tensor-core updates, FP32 accumulate */
    MEHDG_MIXED_BF16 = 2,  /* FP32 storage, BF16 tensor-core updates, FP32 accumulate */
    /* split precision: each product a b taken as a_hi b_hi + a_hi b_lo + a_lo b_hi
     * (hi = round(a), lo = round(a - hi)) on the tensor cores, FP32 accumulate */
    MEHDG_MIXED_TF32X3 = 3,
    MEHDG_MIXED_BF16X3 = 4
} mehdg_prec;

enum {
    MEHDG_OK = 0,
    MEHDG_EINVAL = -1,     /* bad argument, shape or pointer                        */
    MEHDG_ENONPHYS = -2,   /* beta <= 0, rho <= 0 or non-finite state at a point    */
    MEHDG_ESINGULAR = -3,  /* zero pivot in LU(S)                                    */
    MEHDG_ENOCONV = -4,    /* iterative refinement did not reach refine_tol         */
    MEHDG_ECUDA = -5,      /* CUDA runtime error                                     */
    MEHDG_ENOMEM = -6,     /* device allocation failed                               */
    MEHDG_ESTATE = -7,     /* call out of order (e.g. recover before condense)       */
    MEHDG_ETIMEOUT = -8    /* a bounded device wait ran out                          */
};

typedef struct {
    double gamma;          /* ratio of specific heats                                */
    double Re, Pr, Mach;   /* viscous data: mu/Re_c = Mach/Re, kappa from Pr         */
    double dt;             /* time step of the stage term (u(v)-u(v*))/dt, eq. C242  */
    int viscous;           /* 0 Euler, 1 Navier-Stokes                               */
    int flux;              /* mehdg_flux                                              */
    int prec;              /* mehdg_prec                                              */
    double refine_tol;     /* ||r - S x|| <= refine_tol ||r|| ends refinement         */
    int refine_max_iter;   /* refinement sweeps before MEHDG_ENOCONV                  */
    int time_term;         /* 1: include the stage term (default), 0: steady        */
} mehdg_params;

/* Fill *prm with defaults: gamma 1.4, Re 1600, Pr 0.71, Mach 0.1, dt 1,
 * Euler, KEPES, MIXED_TF32, refine_tol 1e-12, refine_max_iter 10, time_term 1. */
void mehdg_default_params(mehdg_params* prm);

/* Create a context.  prm: host pointer, copied.  *out receives the handle. */
int mehdg_create(mehdg_ctx** out, const mehdg_params* prm);

/* Mesh (Sec. 3.1): nK macro-elements of degree p[K] (1..4) and micro-element
 * count m[K] per direction (p[], m[]: host arrays of length nK).  When they
 * differ between elements the context becomes a BATCH context: elements are
 * grouped by (p, m) and each group runs through its own uniform workspaces
 * (groups in order of decreasing cost per element, 2/3 N_v^3 dominating);
 * state and trace arrays are then flattened (element K's [5][Nn(K)] block at
 * voff[K], face g's [5][n_g^2] block at toff[g]; see mehdg_batch_layout), a
 * face shared by two elements must join equal n = m p + 1, and the
 * workspaces of all groups must fit 60 % of the free device memory for the
 * factors to be kept (otherwise condense streams each group in balanced
 * waves of elements that fit, keeps no factors, and apply/recover/solve
 * return MEHDG_ESTATE; MEHDG_BATCH_BUDGET_MB in the environment sets another
 * budget, MEHDG_FORCE_BATCH=1 takes this path for a uniform mesh too).  The
 * residual VJP is not available for batch contexts.
 * box: host [nK][6] = x0 y0 z0 x1 y1 z1.
 * face_gid: host [nK][6], global face of each local face, in
 * [0, n_global_faces); a global face used by two elements couples them
 * (interior face), one used once is an unshared face.  Allocates the device
 * workspaces: one dense S^K per element in the precision of prm->prec (ld^2
 * values, ld = N_v rounded up to 256), three LU operand panels of 2 KB per
 * row of S^K (mixed precisions), and the FP64 point and
 * face Jacobians that make the tangents linear (100 doubles per volume Gauss
 * point and 25 per face point; viscous 225 and 75 more).  Returns
 * MEHDG_ENOMEM when they do not fit. */
int mehdg_set_mesh(mehdg_ctx* ctx, int64_t nK, const int32_t* p, const int32_t* m,
                   const double* box, const int64_t* face_gid, int64_t n_global_faces);

/* State of the Newton iterate (device pointers, not copied): v [nK][5][Nn],
 * vhat [G][5][n^2], q [nK][5][3][Nn] (NULL for Euler), vstar [nK][5][Nn]
 * (state at the start of the step; may be NULL when time_term = 0). */
int mehdg_set_state(mehdg_ctx* ctx, const double* v, const double* vhat, const double* q,
                    const double* vstar, void* stream);

/* Residual of eq. s32 at the state: R_V [nK][5][Nn], R_Q [nK][5][3][Nn]
 * (may be NULL; ignored for Euler), R_Vhat [G][5][n^2] summed over both
 * sides of every face.  Device pointers, overwritten. */
int mehdg_residual(mehdg_ctx* ctx, double* R_V, double* R_Q, double* R_Vhat, void* stream);

/* Condensation (eqs. R1-R3, R5b): residual, Jacobian, Q-elimination, LU of
 * S^K (kept in the context), refined S^-1 products, and
 * bhat [G][5][n^2] = sum_K bhat^K (device, overwritten).
 * Ahat_local must be NULL (the explicit A-hat^K is not formed; use apply). */
int mehdg_condense(mehdg_ctx* ctx, double* bhat, double* Ahat_local, void* stream);

/* The same condensation as mehdg_condense (Ahat_local NULL), replayed from
 * one CUDA graph: the first call (and any call after set_state, set_source or
 * a batch's state changed pointers, or with another bhat) condenses once
 * directly, then records the whole condensation -- residual, Jacobian,
 * Q-elimination, LU, refinement, b-hat; for a batch context every (p, m)
 * group in order -- and later calls launch that graph.  For the recording
 * the refinement runs all refine_max_iter sweeps without synchronising the
 * stream; elements that have converged skip the remaining sweeps on the
 * device, so the result equals mehdg_condense's.  The graph reads the state
 * through the pointers given to set_state: new values in the same arrays
 * need no new recording (a batch context gathers them in set_state).
 * MEHDG_EINVAL for a batch streamed in waves or with phase profiling on. */
int mehdg_condense_graph(mehdg_ctx* ctx, double* bhat, void* stream);

/* y = A-hat x for a global trace vector x (the four stages y1..y4 of
 * Sec. 6.3 summed over elements).  Needs a prior condense.  Device. */
int mehdg_apply_condensed(mehdg_ctx* ctx, const double* x, double* y, void* stream);

/* Recovery after the global trace solve: dV (eq. R2) and dQ (eq. R6, NULL
 * or ignored for Euler) from dVhat [G][5][n^2].  Needs a prior condense. */
int mehdg_recover(mehdg_ctx* ctx, const double* dVhat, double* dV, double* dQ, void* stream);

/* Vector-Jacobian product of the residual of eq. s32 at the state (Euler
 * only): g_v = (dR_V/dv)^T lam_V + (dR_Vhat/dv)^T lam_Vhat and g_vhat =
 * (dR_V/dvhat)^T lam_V + (dR_Vhat/dvhat)^T lam_Vhat, for cotangents lam_V
 * [nK][5][Nn] and lam_Vhat [G][5][n^2] (of the trace residual summed over
 * both sides; may be NULL = 0).  Device arrays; g_v [nK][5][Nn] and g_vhat
 * [G][5][n^2] are overwritten.  Point states and point Jacobians are
 * recomputed from the nodal state (nothing is kept from the forward
 * residual).  MEHDG_EINVAL for a viscous context, MEHDG_ESTATE before
 * set_state; a non-physical point sets the element's status. */
int mehdg_residual_vjp(mehdg_ctx* ctx, const double* lam_V, const double* lam_Vhat, double* g_v,
                       double* g_vhat, void* stream);

/* Adjoint (transposed) condensation of the Newton system of eq. R1, for the
 * VJP through a Newton step (Euler contexts of one element type; needs a
 * prior condense, whose LU factors of S = A_vv it reuses).  The transposed
 * system J^T (lam_V, lam_Vhat) = (g_V, g_Vhat) condenses like eqs. R2-R5
 * with every block transposed:
 *   condense_adjoint : bhat_a = g_Vhat - A_v,vhat^T S^-T g_V   (g_Vhat may be NULL = 0)
 *   apply_..._adjoint: y = A-hat^T x = A_vhat,vhat^T x - A_v,vhat^T S^-T A_vhat,v^T x
 *   solve_..._adjoint: GMRES on A-hat^T x = bhat_a (arguments and returns as
 *                      mehdg_solve_condensed)
 *   recover_adjoint  : lam_V = S^-T (g_V - A_vhat,v^T lam_Vhat)
 * DEVICE arrays: g_V, lam_V [nK][5][Nn]; g_Vhat, bhat_a, x, y, lam_Vhat
 * [G][5][n^2].  S^-T is applied with the stored factors (transposed solve)
 * and refined in FP64 against the exact product S^T x (the residual's VJP),
 * to refine_tol, like the forward solves; every other transposed block
 * product is a VJP of the residual at the state.  MEHDG_EINVAL for viscous or
 * batch contexts, MEHDG_ESTATE before condense. */
int mehdg_condense_adjoint(mehdg_ctx* ctx, const double* g_V, const double* g_Vhat, double* bhat_a, void* stream);
int mehdg_apply_condensed_adjoint(mehdg_ctx* ctx, const double* x, double* y, void* stream);
int mehdg_solve_condensed_adjoint(mehdg_ctx* ctx, const double* bhat_a, double* x, double rtol, int restart,
                                  int max_iter, int* iters, double* relres, void* stream);
int mehdg_recover_adjoint(mehdg_ctx* ctx, const double* g_V, const double* lam_Vhat, double* lam_V, void* stream);

/* A constant added to R_V by residual and condense: src DEVICE [nK][5][Nn]
 * (caller-owned, kept until the next set_source; NULL removes it).  The
 * known stages of a DIRK step enter the stage equation this way (eq. C242).
 * Invalidates a previous condensation.  MEHDG_EINVAL for batch contexts. */
int mehdg_set_source(mehdg_ctx* ctx, const double* src);

/* One time step of size dt of the three-stage DIRK method of Sec. 5.3 (the
 * third-order, L-stable, stiffly accurate DIRK(3,3) of Alexander; D = A^-1)
 * on the state (v, vhat, q: DEVICE, updated in place; q NULL for Euler).
 * Stage i solves eq. C242,
 *   (d_ii/dt)(u(v) - u(v^n)) + sum_{j<i} (d_ij/dt)(u(v^{n,j}) - u(v^n)) + spatial terms = 0
 * (tested against w), by Newton steps (condense, GMRES as
 * mehdg_solve_condensed, recover) until the 2-norm of its residual is below
 * newton_tol, at most newton_max steps; its stage term is the context's with
 * step dt/d_ii and v* = v^n, the known stages a source (mehdg_set_source).
 * The step's result is the last stage (eq. C241 with e = b^T D = e_3).
 * HOST outputs (may be NULL): newton_iters [3], res_norms [3] (final stage
 * residual norms).  Needs a context with the stage term; its dt is
 * restored; on return it holds no state (call set_state next).  Returns
 * MEHDG_ENOCONV when a stage does not reach newton_tol. */
int mehdg_dirk_step(mehdg_ctx* ctx, double* v, double* vhat, double* q, double dt, double newton_tol, int newton_max,
                    double lin_rtol, int restart, int max_iter, int* newton_iters, double* res_norms, void* stream);

/* Vector-Jacobian product through nsteps pseudo-time Newton steps (Sec. 6.1,
 * eqs. C312, C31223) with a fixed step tau (Euler contexts of one element
 * type, created with the stage term).  Forward: from the state (v, vhat)
 * (DEVICE, updated in place to the final iterate), step k solves J(s_k) d_k
 * = -R(s_k) with v* = v_k by condense, GMRES (lin_rtol, restart, max_iter as
 * mehdg_solve_condensed) and recover, and s_{k+1} = s_k + d_k.  Reverse:
 * given the cotangent (gbar_v [nK][5][Nn], gbar_vhat [G][5][n^2] or NULL = 0)
 * of the final state, for k = nsteps-1 .. 0
 *   lam = J(s_k)^-T gbar            (mehdg_condense_adjoint, _solve_, _recover_)
 *   gbar -= J_steady(s_k)^T lam + (d/de J(s_k + e d_k)^T lam)|e=0
 * where J_steady is the Jacobian without the stage term (the stage term's
 * derivatives in v and v* = v cancel) and the last term, the transposed
 * second derivative along the step, is the central difference of the
 * residual VJP at s_k +- h d_k with v* = v_k fixed, h = fd_step max|s_k| /
 * max|d_k| (fd_step 1e-7 is a good choice: the ES and KEPES dissipations
 * carry |.| kinks, e.g. |V-hat . n|, that a larger step can straddle).  The result is the cotangent (g_v0, g_vhat0) of the initial state
 * (DEVICE, same layouts).  Allocates the trajectory (2 nsteps + 8 state
 * vectors) for the call.  On return the context holds no state (call
 * set_state before the next residual or condense). */
int mehdg_pseudo_time_newton_vjp(mehdg_ctx* ctx, double* v, double* vhat, int nsteps, double tau, double lin_rtol,
                                 int restart, int max_iter, const double* gbar_v, const double* gbar_vhat,
                                 double* g_v0, double* g_vhat0, double fd_step, void* stream);

/* Global trace solve of Algorithm 1: dVhat with sum_K A-hat^K dVhat = bhat
 * (eq. R5 summed over the elements), by restarted GMRES(restart) without a
 * preconditioner, matrix-free through mehdg_apply_condensed (needs a prior
 * condense).  bhat and dVhat are device arrays [G][5][n^2]; dVhat holds the
 * initial guess on entry (zeros are fine) and the iterate on return.  Stops
 * when ||bhat - A dVhat||_2 <= rtol ||bhat||_2 (checked on the true residual
 * at every restart) or after max_iter products with A.  iters and relres
 * (HOST, may be NULL) receive the products used and the final relative
 * residual.  Returns MEHDG_ENOCONV (with the iterate in dVhat) when the
 * tolerance was not met, MEHDG_EINVAL for bad arguments, MEHDG_ESTATE
 * before condense, MEHDG_ENOMEM if the (restart + 2) trace vectors of its
 * workspace cannot be allocated (kept in the context for later calls).
 * Synchronises the stream at every Arnoldi step. */
int mehdg_solve_condensed(mehdg_ctx* ctx, const double* bhat, double* dVhat, double rtol, int restart,
                          int max_iter, int* iters, double* relres, void* stream);

/* Step size of the stage term (u(v) - u(v*)) / dt of eq. C242 (and of the
 * pseudo-time term of Sec. 6.1): dt > 0.  The next condense uses it; a
 * previous condensation is invalidated (apply/recover return MEHDG_ESTATE
 * until the next condense). */
int mehdg_set_dt(mehdg_ctx* ctx, double dt);

/* Inexact Newton with pseudo-transient continuation (Sec. 6.1, eqs.
 * C31221-C31223), nsteps steps on the state (v [nK][5][Nn], vhat
 * [G][5][n^2], q [nK][5][3][Nn] or NULL for Euler: DEVICE arrays, updated in
 * place).  Step k: v* = v_k, stage term (u(v) - u(v*)) / tau_k; condense,
 * global trace solve (restarted GMRES(restart), relative tolerance lin_rtol,
 * at most max_iter products, as mehdg_solve_condensed), recover; v += dV,
 * vhat += dVhat, q += dQ.  tau_0 = tau_init, tau_{k+1} = min(tau_max, tau_k
 * ||R_k|| / ||R_{k+1}||) with ||R|| the 2-norm of the steady residual (R_V,
 * R_Vhat and R_Q) at the iterate.  HOST outputs (may be NULL): res_norms
 * [nsteps+1] (||R|| before the first and after every step), taus [nsteps],
 * lin_iters [nsteps] (GMRES products).  Needs a context created with
 * time_term = 1; its dt is restored on return and its state is left at the
 * final iterate (with v* = v, in a buffer of the context).  Allocates its
 * workspace on the first call (kept in the context).  Returns the first
 * failing step's code (MEHDG_ENOCONV from the trace solve, MEHDG_ENONPHYS
 * for a non-finite residual). */
int mehdg_pseudo_time_newton(mehdg_ctx* ctx, double* v, double* vhat, double* q, int nsteps, double tau_init,
                             double tau_max, double lin_rtol, int restart, int max_iter, double* res_norms,
                             double* taus, int* lin_iters, void* stream);

/* Batch contexts (elements of uneven p, m; see mehdg_set_mesh): the offsets
 * of the flattened arrays, HOST int64 voff [nK+1] (element K's [5][Nn(K)]
 * block of v, v*, R_V, dV starts at voff[K]; its [5][3][Nn(K)] block of q,
 * R_Q, dQ at 3 voff[K]) and toff [n_global_faces+1] (face g's [5][n_g^2]
 * block of every trace vector starts at toff[g]).  Either may be NULL.
 * MEHDG_EINVAL for a uniform context.  (No counterpart in the paper, whose
 * elements share one p and m; it describes the layout of the batch.) */
int mehdg_batch_layout(mehdg_ctx* ctx, int64_t* voff, int64_t* toff);

/* Autotuner of a batch context (after set_state): for every (p, m) group,
 * times one condensation of its first min(trial_max, wave) elements for each
 * candidate LU launch shape (leaf-panel CTAs per SM 1, 2 or 4, then CTAs per
 * element in the solves 1, 2, 4, 8 with the better leaf; one untimed
 * warm-up each), keeps the fastest, and records every trial (read with
 * mehdg_batch_report).  Later condensations use the choices.  Invalidates a
 * previous condensation. */
int mehdg_batch_autotune(mehdg_ctx* ctx, int64_t trial_max, void* stream);

/* JSON record of a batch context: resident or streamed, memory budget, and
 * per group p, m, elements, wave size, cost estimate, bytes per element, the
 * launch choices and the autotuner's trials.  Writes at most len bytes
 * (NUL-terminated) into buf (may be NULL) and returns the record's length,
 * or MEHDG_EINVAL for a uniform context. */
int mehdg_batch_report(mehdg_ctx* ctx, char* buf, size_t len);

/* Copy the per-element status words (0 or a negative code above) of the
 * last call into the HOST array per_K_status [nK]; synchronises the device.
 * Also copies, if iters != NULL, the refinement sweeps used per element. */
int mehdg_status(mehdg_ctx* ctx, int32_t* per_K_status, int32_t* iters);

/* The per-element status words (and, if iters != NULL, the refinement
 * sweeps) of the last call, copied on `stream` into the DEVICE arrays
 * per_K_status [nK] and iters [nK]: asynchronous, valid after a
 * synchronisation of that stream (the form Algorithm 1's local steps need
 * when the status stays on the GPU).  The work of the last call must have
 * been enqueued on the same stream or be ordered before it. */
int mehdg_status_device(mehdg_ctx* ctx, int32_t* per_K_status, int32_t* iters, void* stream);

/* Message of the last error of this context (static storage of ctx). */
const char* mehdg_last_error(const mehdg_ctx* ctx);

/* Optional timing of the phases with CUDA events recorded on the caller's
 * stream (off by default).  enable != 0 starts a new record. */
int mehdg_profile_enable(mehdg_ctx* ctx, int enable);

/* Per-phase sums since profile_enable (synchronises the device): event-timed
 * milliseconds, launches timed and algorithmic flops (host arrays of length
 * nphase).  Phases: 0 residual, 1 Jacobian assembly, 2 LU panels (leaf
 * panels, swaps, TRSM, inner updates), 3 LU outer trailing update kernel
 * (depth 256), 4 triangular solves, 5 matrix-free tangent residuals,
 * 6 operand packing of the outer trailing updates. */
int mehdg_profile_read(mehdg_ctx* ctx, double* ms, int64_t* launches, double* flops, int nphase);

/* Number of kernels this library has launched since it was loaded. */
int64_t mehdg_launch_count(void);

/* Residual without any device allocation (the paper has no counterpart; it
 * exists for callers that must not allocate device memory after start-up,
 * e.g. a host application whose own pool allocator owns the whole GPU, where
 * a stray cudaMalloc fails or breaks its accounting, or a real-time loop
 * that forbids allocation).  Same result as mehdg_residual, but no context:
 * prm (host), p, m, and DEVICE arrays box [nK][6], face_gid [nK][6],
 * v, vhat, q (NULL for Euler), vstar, R_V, R_Q (NULL for Euler), R_Vhat in
 * the layouts above.  Its scratch is one static device array of 24 MiB per
 * GPU, held until the process exits; the call needs
 * nK * 30 n^2 doubles + 2 n_global_faces int64 + nK int32 (+ alignment) of
 * it and returns MEHDG_EINVAL (message on stderr) when that does not fit.
 * The first call made on a device looks up the array's device address (once
 * per device).  Calls share the array: calls that overlap on the GPU race.
 * The call synchronises `stream` twice: after checking the face ids on the
 * device (before the residual kernels read with them), and at the end to
 * read the elements' status words; a non-physical state at any point
 * returns MEHDG_ENONPHYS (count and first element on stderr), with the
 * outputs written but not meaningful for those elements. */
int mehdg_residual_static(const mehdg_params* prm, int64_t nK, int p, int m, const double* box,
                          const int64_t* face_gid, int64_t n_global_faces, const double* v,
                          const double* vhat, const double* q, const double* vstar, double* R_V,
                          double* R_Q, double* R_Vhat, void* stream);

/* Diagnostics: one tensor-core trailing update of the mixed-precision LU,
 *   S[r0+i, c0+j] -= sum_k S[r0+i, k0+k] S[k0+k, c0+j]  (i<M, j<N, k<Kd),
 * on nK column-major FP32 matrices S [nK][ld][ld] (device), with operands
 * rounded to TF32 (prec 1) or BF16 (prec 2) and FP32 accumulation; the
 * Schur-complement update step of the LU of S^K (eq. R3 factorisation).
 * M, N, Kd and the offsets are multiples of 32; work: device scratch of
 * mehdg_test_trailing_work_bytes(nK, ld) bytes.  Returns MEHDG_OK or
 * MEHDG_ECUDA. */
int mehdg_test_trailing_update(int64_t nK, int64_t ld, float* S, int r0, int c0, int k0, int M, int N,
                               int Kd, int prec, void* work, void* stream);
size_t mehdg_test_trailing_work_bytes(int64_t nK, int64_t ld);

/* Free every device workspace and the context. */
void mehdg_destroy(mehdg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MEHDG_H */
