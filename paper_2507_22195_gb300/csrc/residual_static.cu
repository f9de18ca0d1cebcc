// residual_static.cu -- the residual entry point that allocates nothing.
//
// For callers that must not allocate device memory after start-up, such as a
// host application whose own pool allocator owns the whole GPU (a stray
// cudaMalloc there fails or breaks its accounting) or a real-time loop that
// forbids allocation: mehdg_residual_static computes the same residual as
// mehdg_residual from caller-owned device arrays only.  Its scratch (each
// element's side of the trace residual and the map from global faces to
// element sides) lives in the file-scope array below, which every GPU that
// loads this library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current, on the first call made on it) and passed to the kernels.
// All calls share the array and it keeps the last call's contents: every
// call re-initialises what it uses, and calls that overlap on the GPU (other
// streams, other host threads) race on it.
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include "common.cuh"
#include "kernels.cuh"

namespace {

// 24 MiB: per-element trace sides (nK * 30 n^2 doubles) + face map (2 G int64) + status
constexpr size_t kStaticScratchBytes = 24u << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

// face map: slot 0 = smallest element side (K*6+f) on the face, slot 1 = the other one.
// err[0]: face-id check; err[1], err[2]: number and first index of the
// elements whose status word is set (filled by status_summary_kernel)
__global__ void g2l_init_kernel(int64_t* g2l, int64_t G, int32_t* err) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g == 0) { err[0] = 0; err[1] = 0; err[2] = INT_MAX; }
    if (g < G) { g2l[2 * g] = LLONG_MAX; g2l[2 * g + 1] = -1; }
}
__global__ void status_zero_kernel(int32_t* status, int64_t nK) {
    int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K < nK) status[K] = 0;
}
__global__ void status_summary_kernel(const int32_t* status, int64_t nK, int32_t* err) {
    int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K < nK && status[K] != 0) {
        atomicAdd(&err[1], 1);
        atomicMin(&err[2], (int)K);
    }
}
__global__ void g2l_min_kernel(const int64_t* gid, int64_t nK, int64_t G, int64_t* g2l, int32_t* err) {
    int64_t kf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (kf >= 6 * nK) return;
    int64_t g = gid[kf];
    if (g < 0 || g >= G) { atomicExch(err, 1); return; }
    atomicMin(reinterpret_cast<long long*>(&g2l[2 * g]), (long long)kf);
}
__global__ void g2l_other_kernel(const int64_t* gid, int64_t nK, int64_t G, int64_t* g2l, int32_t* err) {
    int64_t kf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (kf >= 6 * nK) return;
    int64_t g = gid[kf];
    if (g < 0 || g >= G) return;
    if (g2l[2 * g] != kf) {
        long long old = atomicExch(reinterpret_cast<unsigned long long*>(&g2l[2 * g + 1]), (unsigned long long)kf);
        if (old != -1) atomicExch(err, 2);     // a face with more than two sides
    }
}
__global__ void g2l_finish_kernel(int64_t* g2l, int64_t G) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < G && g2l[2 * g] == LLONG_MAX) g2l[2 * g] = -1;
}

// device address of the scratch array for the current device (looked up once)
unsigned char* scratch_address(char* err, size_t errlen) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(err, errlen, "residual_static: no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(err, errlen, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return nullptr;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    return g_addr[dev];
}

// errors are returned as codes and described on stderr
void report(const char* msg) { fprintf(stderr, "mehdg_residual_static: %s\n", msg); }

}  // namespace

extern "C" int mehdg_residual_static(const mehdg_params* prm, int64_t nK, int p, int m, const double* box,
                                     const int64_t* face_gid, int64_t G, const double* v, const double* vhat,
                                     const double* q, const double* vstar, double* R_V, double* R_Q,
                                     double* R_Vhat, void* stream) {
    char t_err[256];
    if (!prm || nK <= 0 || G <= 0 || p < 1 || p > MEHDG_MAXP || m < 1 || m > 16 || !box || !face_gid || !v ||
        !vhat || !R_V || !R_Vhat || (prm->viscous && (!q || !R_Q)) || (prm->time_term && (!vstar || !(prm->dt > 0)))) {
        report("bad arguments");
        return MEHDG_EINVAL;
    }
    if (prm->flux < 0 || prm->flux > 2 || !(prm->gamma > 1.0)) {
        report("bad parameters");
        return MEHDG_EINVAL;
    }
    Tab tab;
    host_build_tables(p, m, &tab);
    const size_t side_bytes = (size_t)nK * 30 * tab.n2 * sizeof(double);
    const size_t map_off = (side_bytes + 255) & ~(size_t)255;
    const size_t map_bytes = (size_t)G * 2 * sizeof(int64_t);
    const size_t stat_off = (map_off + map_bytes + 255) & ~(size_t)255;
    const size_t err_off = (stat_off + (size_t)nK * sizeof(int32_t) + 255) & ~(size_t)255;
    if (err_off + 256 > kStaticScratchBytes) {
        snprintf(t_err, sizeof(t_err),
                 "needs %zu bytes of scratch, the static array holds %zu (nK x 30 n^2 doubles + 2 G int64 + nK int32)",
                 err_off + 256, kStaticScratchBytes);
        report(t_err);
        return MEHDG_EINVAL;
    }
    unsigned char* base = scratch_address(t_err, sizeof(t_err));
    if (!base) { report(t_err); return MEHDG_ECUDA; }
    double* RHloc = reinterpret_cast<double*>(base);
    int64_t* g2l = reinterpret_cast<int64_t*>(base + map_off);
    int32_t* dstat = reinterpret_cast<int32_t*>(base + stat_off);
    int32_t* derr = reinterpret_cast<int32_t*>(base + err_off);
    cudaStream_t st = (cudaStream_t)stream;

    Phys ph;
    std::memset(&ph, 0, sizeof(ph));
    ph.gamma = prm->gamma;
    ph.mu = prm->viscous ? prm->Mach / prm->Re : 0.0;
    ph.kappa = prm->viscous ? ph.mu / ((prm->gamma - 1.0) * prm->Pr) : 0.0;
    ph.sv_mom = prm->viscous ? 1.0 / prm->Re : 0.0;
    ph.sv_en = prm->viscous ? 1.0 / (prm->Re * (prm->gamma - 1.0) * prm->Mach * prm->Mach * prm->Pr) : 0.0;
    ph.inv_dt = prm->time_term ? 1.0 / prm->dt : 0.0;
    ph.viscous = prm->viscous; ph.flux = prm->flux; ph.time_term = prm->time_term;

    const int bs = 256;
    g2l_init_kernel<<<(unsigned)((G + bs - 1) / bs), bs, 0, st>>>(g2l, G, derr);
    g2l_min_kernel<<<(unsigned)((6 * nK + bs - 1) / bs), bs, 0, st>>>(face_gid, nK, G, g2l, derr);
    g2l_other_kernel<<<(unsigned)((6 * nK + bs - 1) / bs), bs, 0, st>>>(face_gid, nK, G, g2l, derr);
    g2l_finish_kernel<<<(unsigned)((G + bs - 1) / bs), bs, 0, st>>>(g2l, G);
    status_zero_kernel<<<(unsigned)((nK + bs - 1) / bs), bs, 0, st>>>(dstat, nK);
    MEHDG_COUNT(5);
    // the face ids index the trace arrays: check them before any kernel reads with them
    int32_t herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        report(cudaGetErrorString(e));
        return MEHDG_ECUDA;
    }
    if (herr) {
        report(herr == 1 ? "face id out of range" : "a global face has more than two sides");
        return MEHDG_EINVAL;
    }

    ResidualArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tab = tab; a.ph = ph; a.box = box; a.gid = face_gid;
    a.v = v; a.vs = vstar; a.vh = vhat; a.q = q;
    a.RV = R_V; a.RQ = prm->viscous ? R_Q : nullptr; a.RH = RHloc;
    a.status = dstat;
    e = launch_residual(a, nK, prm->viscous != 0, false, st);
    if (e == cudaSuccess) e = launch_trace_gather(RHloc, g2l, G, tab.n2, R_Vhat, 1.0, nullptr, 0.0, st);
    if (e == cudaSuccess) {
        status_summary_kernel<<<(unsigned)((nK + bs - 1) / bs), bs, 0, st>>>(dstat, nK, derr);
        MEHDG_COUNT(1);
        e = cudaGetLastError();
    }
    // second synchronisation: the elements' status words (a non-physical
    // state at a point: beta <= 0, rho <= 0 or a non-finite value)
    int32_t hsum[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hsum, derr + 1, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(t_err, sizeof(t_err), "launch failed: %s", cudaGetErrorString(e));
        report(t_err);
        return MEHDG_ECUDA;
    }
    if (hsum[0] > 0) {
        snprintf(t_err, sizeof(t_err), "non-physical state in %d element(s), first element %d", hsum[0], hsum[1]);
        report(t_err);
        return MEHDG_ENONPHYS;
    }
    return MEHDG_OK;
}
