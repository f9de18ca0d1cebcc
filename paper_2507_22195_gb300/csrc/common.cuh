// common.cuh -- shared definitions of the GB300 hot path (device + host).
//
// Discretisation (Sec. 3.1 with hexahedral micro-elements): a macro-element
// is an axis-aligned box of m^3 micro-elements, Q_p on Gauss-Lobatto-Legendre
// nodes, C0 inside the box; tensor Gauss quadrature with p+2 points per
// direction per micro-element.  n = m p + 1, node A = i + n (j + n k).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <atomic>
#include "../../include/mehdg.h"
#include "prof.cuh"

#define MEHDG_MAXP 4
#define MEHDG_MAXG (MEHDG_MAXP + 2)

// 1-D reference tables, passed to kernels by value.
struct Tab {
    int p, m, n, ng, nq, Nn, n2;
    int nl;                         // (p+1)^3 local nodes of a micro-element
    int npt;                        // (p+2)^3 Gauss points of a micro-element
    double L[MEHDG_MAXG][MEHDG_MAXP + 1];   // Lagrange value at Gauss point g
    double dL[MEHDG_MAXG][MEHDG_MAXP + 1];  // reference derivative d/dxi
    double w[MEHDG_MAXG];                    // Gauss weight on [-1,1]
};

// physical and numerical parameters, by value
struct Phys {
    double gamma;
    double mu, kappa;     // mu/Re_c = Mach/Re, kappa = mu c_p / Pr
    double sv_mom, sv_en; // viscous penalty sigma^vis (momentum, energy)
    double inv_dt;
    int viscous, flux, time_term;
};

void host_build_tables(int p, int m, Tab* t);   // tables.cpp

// ------------------------------------------------------------------ duals
// Forward-mode dual number with N tangent directions.
template <int N>
struct Dual {
    double v;
    double d[N];
};

template <class T> struct ScalarTraits;
template <> struct ScalarTraits<double> { static constexpr int N = 0; };
template <int N> struct ScalarTraits<Dual<N>> { static constexpr int N_ = N; };

__host__ __device__ __forceinline__ double val(double x) { return x; }
template <int N> __host__ __device__ __forceinline__ double val(const Dual<N>& x) { return x.v; }

template <int N>
__host__ __device__ __forceinline__ Dual<N> mkdual(double v) {
    Dual<N> r; r.v = v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = 0.0;
    return r;
}

#define DUAL_BIN(OP, VEXPR, DEXPR)                                                     \
    template <int N> __host__ __device__ __forceinline__ Dual<N> operator OP(const Dual<N>& a, const Dual<N>& b) { \
        Dual<N> r; r.v = VEXPR;                                                        \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.d[i] = DEXPR;                  \
        return r; }
DUAL_BIN(+, a.v + b.v, a.d[i] + b.d[i])
DUAL_BIN(-, a.v - b.v, a.d[i] - b.d[i])
DUAL_BIN(*, a.v * b.v, a.d[i] * b.v + a.v * b.d[i])
#undef DUAL_BIN

template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; double ib = 1.0 / b.v; r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r; r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
// mixed with double
template <int N> __host__ __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator+(double b, const Dual<N>& a) { Dual<N> r = a; r.v += b; return r; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator-(double b, const Dual<N>& a) { Dual<N> r = -a; r.v += b; return r; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r; r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> __host__ __device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) {
    Dual<N> r; double ib = 1.0 / b.v; r.v = a * ib;
    double s = -r.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = s * b.d[i];
    return r;
}
template <int N> __host__ __device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> __host__ __device__ __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }

// elementary functions (CUDA's log/exp/sqrt for the values; derivatives
// from the calculus: d log x = dx/x, d exp x = exp x dx, d sqrt x = dx/(2 sqrt x))
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
template <int N> __device__ __forceinline__ Dual<N> dlog(const Dual<N>& a) {
    Dual<N> r; r.v = log(a.v); double s = 1.0 / a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> dexp(const Dual<N>& a) {
    Dual<N> r; r.v = exp(a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v;
    return r;
}
template <int N> __device__ __forceinline__ Dual<N> dsqrt(const Dual<N>& a) {
    Dual<N> r; r.v = sqrt(a.v); double s = r.v > 0 ? 0.5 / r.v : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
    return r;
}
// |x| with the derivative convention d|x| = sgn(x) dx, sgn(0) = +1
__device__ __forceinline__ double dabs(double x) { return x >= 0.0 ? x : -x; }
template <int N> __device__ __forceinline__ Dual<N> dabs(const Dual<N>& a) { return a.v >= 0.0 ? a : -a; }

template <class T> __device__ __forceinline__ T cst(double x);
template <> __device__ __forceinline__ double cst<double>(double x) { return x; }
template <> __device__ __forceinline__ Dual<1> cst<Dual<1>>(double x) { return mkdual<1>(x); }
template <> __device__ __forceinline__ Dual<5> cst<Dual<5>>(double x) { return mkdual<5>(x); }
template <> __device__ __forceinline__ Dual<15> cst<Dual<15>>(double x) { return mkdual<15>(x); }
template <> __device__ __forceinline__ Dual<10> cst<Dual<10>>(double x) { return mkdual<10>(x); }

// ------------------------------------------------------------------ context
struct DeviceLU;   // defined in lu.cuh
struct Batch;      // macro-elements of uneven p and m (batch.cu)

struct mehdg_ctx {
    mehdg_params prm;
    Phys ph;
    char err[512];
    // mesh
    int64_t nK = 0, G = 0;
    int p = 0, m = 0;
    Tab tab;
    int Nv = 0, Nt_loc = 0, Npad = 0;
    double* d_box = nullptr;            // [nK][6]
    int64_t* d_gid = nullptr;           // [nK][6]
    int64_t* d_g2l = nullptr;           // [G][2] (K*6+f) or -1
    // state (caller-owned)
    const double *v = nullptr, *vh = nullptr, *q = nullptr, *vs = nullptr;
    const double* src = nullptr;        // optional constant added to R_V ([nK][5][Nn], caller-owned)
    // workspaces
    double* d_RV = nullptr;             // [nK][5][Nn]      residual at the condensed state
    double* d_RHloc = nullptr;          // [nK][6][5][n2]   per-element trace residual
    double* d_tRHloc = nullptr;         // tangent of the trace residual
    double* d_tRHloc2 = nullptr;        // second tangent trace buffer
    double* d_tRV = nullptr;            // tangent of R_V
    double* d_xu = nullptr;             // [nK][5][Nn] unpadded solution (tangent direction)
    // viscous: gradient-equation data, q-shaped [nK][15][Nn]
    double* d_RQ = nullptr;             // R_Q at the condensed state
    double* d_z = nullptr;              // A_qq^-1 R_Q
    double* d_dq = nullptr;             // q-direction of a tangent
    double *d_qt1 = nullptr, *d_qt2 = nullptr;   // line-operator scratch
    double *d_Minv = nullptr, *d_C1 = nullptr;   // [n][n] 1-D tables
    double* d_pj = nullptr;             // [nK][m^3][100][npt] weighted FP64 point Jacobians (inviscid)
    double* d_pjf = nullptr;            // [nK][6 m^2][25][fpt] weighted FP64 face blocks dFhat/dv (inviscid)
    double* d_pq = nullptr;             // [nK][m^3][225][npt] viscous point blocks W dG/dq
    double* d_pqf = nullptr;            // [nK][6 m^2][75][fpt] viscous face blocks W dGhat/dq
    bool pj_ready = false;              // d_pj holds the Jacobians at the current state
    double* d_r = nullptr;              // [nK][Npad] FP64 right-hand side
    double* d_x = nullptr;              // [nK][Npad] FP64 solution
    double* d_res = nullptr;            // [nK][Npad] FP64 refinement residual
    double* d_dx = nullptr;             // [nK][Npad] FP64 correction
    double* d_nrm = nullptr;            // [nK][2] norms
    int32_t* d_status = nullptr;        // [nK]
    int32_t* d_iters = nullptr;         // [nK]
    int32_t* d_conv = nullptr;          // [nK] converged flag
    int32_t* h_cnt = nullptr;           // pinned counter
    int32_t* d_cnt = nullptr;
    void* d_S = nullptr;                // [nK][Npad][Npad] col-major, FP32 or FP64
    int32_t* d_piv = nullptr;           // [nK][Npad]
    void* d_work = nullptr;             // LU work buffers
    size_t work_bytes = 0;
    float* d_rf = nullptr;              // [nK][Npad] FP32 solve vector
    bool condensed = false;
    cudaGraphExec_t lu_graph = nullptr; // the factorisation's launches, captured on first use
    cudaStream_t lu_stream = nullptr;   // stream the graph is replayed on
    cudaEvent_t lu_ev_in = nullptr, lu_ev_out = nullptr;
    cudaEvent_t zs_ev_in = nullptr, zs_ev_out = nullptr;   // zeroing of S beside the residual
    long long lu_graph_launches = 0;    // kernels in the graph
    bool lu_graph_failed = false;       // capture failed once: the LU is launched directly
    bool graph_refine = false;          // refinement without host synchronisation (graph capture)
    cudaGraphExec_t cond_graph = nullptr; // the whole condensation, captured (mehdg_condense_graph)
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_in = nullptr, cap_out = nullptr;
    const void* cap_key[7] = {};        // pointers the captured graph was recorded with
    long long cond_graph_launches = 0;
    int tune_leaf_ctas = 0;             // LU launch choices (0 = automatic), set by the batch autotuner
    int tune_solve_ctas = 0;
    void* d_krylov = nullptr;           // GMRES basis and scratch of the trace solve (first use)
    size_t krylov_bytes = 0;
    void* d_newton = nullptr;           // pseudo-time Newton loop: v*, residuals, increments (first use)
    size_t newton_bytes = 0;
    void* d_adj = nullptr;              // adjoint condensation scratch (first use)
    size_t adj_bytes = 0;
    Batch* batch = nullptr;             // set when the elements have uneven p, m (the fields above then
                                        // describe no single element type)
    Prof prof;
};

// kernels launched by this library since load (reported by mehdg_launch_count)
extern std::atomic<long long> g_mehdg_launches;
#define MEHDG_COUNT(n) (g_mehdg_launches += (n))

// error helpers
#define MEHDG_CUDA_TRY(ctx, call)                                                    \
    do { cudaError_t e_ = (call);                                                    \
         if (e_ != cudaSuccess) { set_err(ctx, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
                                  return MEHDG_ECUDA; } } while (0)

void set_err(mehdg_ctx* ctx, const char* fmt, ...);

// batch contexts (batch.cu)
int batch_set_mesh(mehdg_ctx* c, int64_t nK, const int32_t* p, const int32_t* m, const double* box,
                   const int64_t* face_gid, int64_t G);
int batch_free(mehdg_ctx* c);
int batch_set_state(mehdg_ctx* c, const double* v, const double* vhat, const double* q, const double* vstar,
                    cudaStream_t st);
int batch_residual(mehdg_ctx* c, double* R_V, double* R_Q, double* R_Vhat, cudaStream_t st);
int batch_condense(mehdg_ctx* c, double* bhat, cudaStream_t st);
int batch_apply(mehdg_ctx* c, const double* x, double* y, cudaStream_t st);
int batch_recover(mehdg_ctx* c, const double* dVhat, double* dV, double* dQ, cudaStream_t st);
int batch_autotune(mehdg_ctx* c, int64_t trial_max, cudaStream_t st);
int batch_report(const mehdg_ctx* c, char* buf, size_t len);
void batch_layout(const mehdg_ctx* c, int64_t* voff, int64_t* toff);
int64_t batch_state_len(const mehdg_ctx* c);
int64_t batch_trace_len(const mehdg_ctx* c);
int batch_set_dt(mehdg_ctx* c);
bool batch_resident(const mehdg_ctx* c);
void batch_set_graph_refine(mehdg_ctx* c, bool on);
void batch_mark_condensed(mehdg_ctx* c);
void batch_end_captures(mehdg_ctx* c);
void end_captures(mehdg_ctx* c);        // graph.cu

// lengths of the state ([nK][5][Nn] in all) and global trace vectors
inline int64_t ctx_state_len(const mehdg_ctx* c) { return c->batch ? batch_state_len(c) : c->nK * (int64_t)c->Nv; }
inline int64_t ctx_trace_len(const mehdg_ctx* c) { return c->batch ? batch_trace_len(c) : c->G * 5 * (int64_t)c->tab.n2; }
