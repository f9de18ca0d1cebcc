// batch.cu -- macro-elements of uneven polynomial degree p and micro-element
// count m in one context.
//
// The Newton step of Algorithm 1 is local to each macro-element up to the
// sums over the two sides of every face (eq. s32c; assembly of b-hat).  A
// batch context therefore groups its elements by (p, m), runs each group
// through a uniform sub-context whose faces are all unshared (so that every
// local face is one element side), and assembles the face sums from the
// per-side results in a fixed order (deterministic, no atomics).
//
// Groups are processed in order of decreasing cost per element (the dense
// LU, 2/3 N_v^3, dominates).  When every group fits the memory budget at
// once, each group keeps one sub-context over all of its elements: the LU
// factors stay resident and apply/recover/solve work as for a uniform mesh.
// Otherwise condense streams each group in waves of elements sized to the
// budget (balanced waves; a sub-context over one wave, re-pointed from wave
// to wave), and the factors are discarded: apply and recover then return
// MEHDG_ESTATE.  An autotuner times the LU launch choices of each group (leaf
// CTAs per SM, CTAs per element in the solves) on a trial wave and records
// its decisions with the measured times.
//
// Layouts of the caller's arrays (host offsets from mehdg_batch_layout):
//   v, v*, R_V, dV   element K at voff[K], [5][Nn(K)]; q, R_Q, dQ at 3 voff[K]
//   traces           face g at toff[g], [5][n_g^2] (n_g = n of its elements)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include "common.cuh"
#include "kernels.cuh"

int batch_free(mehdg_ctx* c);

namespace {

struct Group {
    int p = 0, m = 0, n = 0, Nn = 0, n2 = 0;
    std::vector<int64_t> elems;         // global element ids, ascending
    int64_t* d_elems = nullptr;         // the same on the device
    int64_t wave = 0;                   // elements per wave (sub-context size)
    double cost = 0.0;                  // flop estimate per element
    size_t bytes_per_elem = 0;          // device bytes per element of a sub-context
    mehdg_ctx* sub = nullptr;           // resident: over all elements; streaming: current wave
    int64_t sub_cap = 0;                // elements the sub-context was created for
    // sub-context state and outputs (wave-sized)
    double *sv = nullptr, *svs = nullptr, *svh = nullptr, *sq = nullptr;
    double *sRV = nullptr, *sRQ = nullptr, *sRH = nullptr, *sbh = nullptr, *sdV = nullptr, *sdQ = nullptr;
    double *sx = nullptr, *sy = nullptr;
    // autotuner
    int leaf_ctas = 0, solve_ctas = 0;
    bool tuned = false;
    std::string tune_log;
};

}  // namespace

struct Batch {
    std::vector<Group> groups;          // decreasing cost per element
    std::vector<int64_t> voff, toff, soff;
    std::vector<int32_t> ep, em;        // per element p, m
    int64_t *d_voff = nullptr, *d_toff = nullptr, *d_soff = nullptr, *d_gid = nullptr, *d_fside = nullptr;
    double* d_sides = nullptr;          // per element side traces, element K at soff[K] = [6][5][n^2]
    std::vector<double> box;            // [nK][6] host copy (the waves re-point the sub-context's boxes)
    size_t budget = 0;
    bool resident = false;
    const double *v = nullptr, *vh = nullptr, *q = nullptr, *vs = nullptr;
};

namespace {

unsigned blocks_for(int64_t n, int bs = 256) {
    int64_t g = (n + bs - 1) / bs;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(g, 1), 65535 * 16);
}

// dst[k][i] = src[scale voff[elems[k0 + k]] + i], i < len, k < n
__global__ void gather_elems_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                    const int64_t* __restrict__ voff, int64_t scale, const int64_t* __restrict__ elems,
                                    int64_t k0, int64_t n, int64_t len) {
    const int64_t tot = n * len;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / len, i = t - k * len;
        dst[t] = src[scale * voff[elems[k0 + k]] + i];
    }
}
__global__ void scatter_elems_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                     const int64_t* __restrict__ voff, int64_t scale, const int64_t* __restrict__ elems,
                                     int64_t k0, int64_t n, int64_t len) {
    const int64_t tot = n * len;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / len, i = t - k * len;
        dst[scale * voff[elems[k0 + k]] + i] = src[t];
    }
}
// sub trace of unshared faces, face 6k+f = side f of wave element k, from the
// global trace vector
__global__ void gather_sides_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                    const int64_t* __restrict__ toff, const int64_t* __restrict__ gid,
                                    const int64_t* __restrict__ elems, int64_t k0, int64_t n, int64_t len) {
    const int64_t tot = n * 6 * len;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / len, i = t - s * len;
        const int64_t K = elems[k0 + s / 6];
        dst[t] = src[toff[gid[6 * K + s % 6]] + i];
    }
}
// sub trace (one side per local face) into the per-side buffer
__global__ void scatter_sides_kernel(double* __restrict__ sides, const double* __restrict__ src,
                                     const int64_t* __restrict__ soff, const int64_t* __restrict__ elems, int64_t k0,
                                     int64_t n, int64_t len) {
    const int64_t tot = n * 6 * len;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / len, i = t - s * len;
        const int64_t K = elems[k0 + s / 6];
        sides[soff[K] + (s % 6) * len + i] = src[t];
    }
}
// out[toff[g] + i] = side a + side b (b absent: -1), in a fixed order
__global__ void face_sum_kernel(double* __restrict__ out, const double* __restrict__ sides,
                                const int64_t* __restrict__ toff, const int64_t* __restrict__ fside, int64_t G) {
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t len = toff[g + 1] - toff[g];
        const int64_t a = fside[2 * g], b = fside[2 * g + 1];
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
            double s = a >= 0 ? sides[a + i] : 0.0;
            if (b >= 0) s += sides[b + i];
            out[toff[g] + i] = s;
        }
    }
}
__global__ void scatter_status_kernel(int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                                      const int64_t* __restrict__ elems, int64_t k0, int64_t n) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) dst[elems[k0 + k]] = src[k];
}

#define BTRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e_)); return MEHDG_ECUDA; } } while (0)
#define BRC(x) do { int r_ = (x); if (r_) return r_; } while (0)

template <class T> void bfree(T*& p) { if (p) { cudaFree((void*)p); p = nullptr; } }

void free_group_buffers(Group& g) {
    bfree(g.sv); bfree(g.svs); bfree(g.svh); bfree(g.sq); bfree(g.sRV); bfree(g.sRQ); bfree(g.sRH);
    bfree(g.sbh); bfree(g.sdV); bfree(g.sdQ); bfree(g.sx); bfree(g.sy);
    if (g.sub) { mehdg_destroy(g.sub); g.sub = nullptr; }
    g.sub_cap = 0;
}

// device bytes per element of a uniform sub-context of degree p, m (with the
// batch's own wave buffers), from the allocations mehdg_set_mesh makes
size_t bytes_per_element(const mehdg_params& prm, int p, int m) {
    Tab t;
    host_build_tables(p, m, &t);
    const size_t Nv = 5 * (size_t)t.Nn, ld = (Nv + 255) / 256 * 256, nt = 30 * (size_t)t.n2;
    const bool fp64 = prm.prec == MEHDG_FP64, vis = prm.viscous != 0;
    size_t b = ld * ld * (fp64 ? 8 : 4);
    b += lu_work_bytes(1, (int64_t)ld, fp64, prm.prec) + 4 * ld;                           // LU workspace, pivots
    b += 8 * (100 * (size_t)t.m * t.m * t.m * t.npt + 25 * 6 * (size_t)t.m * t.m * t.ng * t.ng);  // point Jacobians
    if (vis) b += 8 * (225 * (size_t)t.m * t.m * t.m * t.npt + 75 * 6 * (size_t)t.m * t.m * t.ng * t.ng + 5 * 15 * (size_t)t.Nn);
    b += 8 * (4 * Nv + 4 * ld + 4 * nt);                                                   // context vectors
    b += 8 * (5 * Nv + 4 * nt + (vis ? 6 * 15 * (size_t)t.Nn / 5 * 5 : 0));               // wave buffers
    return b + b / 16;
}

int alloc_group_buffers(mehdg_ctx* c, Group& g, int64_t cap) {
    const size_t nv = (size_t)cap * 5 * g.Nn, nq = c->prm.viscous ? 3 * nv : 0, nt = (size_t)cap * 30 * g.n2;
#define BALLOC(ptr, count) do { if ((count) > 0 && cudaMalloc((void**)&(ptr), sizeof(double) * (count)) != cudaSuccess) { \
        set_err(c, "batch: cudaMalloc of %zu doubles failed", (size_t)(count)); free_group_buffers(g); return MEHDG_ENOMEM; } } while (0)
    BALLOC(g.sv, nv); BALLOC(g.svs, nv); BALLOC(g.svh, nt); BALLOC(g.sRV, nv); BALLOC(g.sRH, nt); BALLOC(g.sbh, nt);
    BALLOC(g.sdV, nv); BALLOC(g.sx, nt); BALLOC(g.sy, nt);
    if (nq) { BALLOC(g.sq, nq); BALLOC(g.sRQ, nq); BALLOC(g.sdQ, nq); }
#undef BALLOC
    return MEHDG_OK;
}

// a uniform sub-context over `cap` elements with unshared faces (boxes of
// the first cap elements of the group; waves re-point them)
int make_sub(mehdg_ctx* c, Group& g, int64_t cap) {
    Batch& B = *c->batch;
    free_group_buffers(g);
    mehdg_ctx* s = nullptr;
    BRC(mehdg_create(&s, &c->prm));
    std::vector<int32_t> pp(cap, g.p), mm(cap, g.m);
    std::vector<double> box(6 * cap);
    std::vector<int64_t> gid(6 * cap);
    for (int64_t k = 0; k < cap; ++k) {
        for (int i = 0; i < 6; ++i) box[6 * k + i] = B.box[6 * g.elems[k] + i];
        for (int f = 0; f < 6; ++f) gid[6 * k + f] = 6 * k + f;
    }
    int rc = mehdg_set_mesh(s, cap, pp.data(), mm.data(), box.data(), gid.data(), 6 * cap);
    if (rc) { set_err(c, "batch group p=%d m=%d: %s", g.p, g.m, mehdg_last_error(s)); mehdg_destroy(s); return rc; }
    s->tune_leaf_ctas = g.leaf_ctas;
    s->tune_solve_ctas = g.solve_ctas;
    g.sub = s;
    g.sub_cap = cap;
    return alloc_group_buffers(c, g, cap);
}

// point the sub-context at wave [k0, k0+n) of the group: its boxes, its
// element count, and the gathered state
int load_wave(mehdg_ctx* c, Group& g, int64_t k0, int64_t n, cudaStream_t st) {
    Batch& B = *c->batch;
    mehdg_ctx* s = g.sub;
    if (n != s->nK || k0 != 0 || !B.resident) {
        std::vector<double> box(6 * n);
        for (int64_t k = 0; k < n; ++k)
            for (int i = 0; i < 6; ++i) box[6 * k + i] = B.box[6 * g.elems[k0 + k] + i];
        BTRY(cudaMemcpyAsync(s->d_box, box.data(), sizeof(double) * 6 * n, cudaMemcpyHostToDevice, st));
        BTRY(cudaStreamSynchronize(st));          // box is a host temporary
        if (n != s->nK) {
            // a shorter last wave runs on a prefix of the sub-context's arrays
            s->nK = n;
            s->G = 6 * n;
            if (s->lu_graph) { cudaGraphExecDestroy(s->lu_graph); s->lu_graph = nullptr; }
        }
    }
    if (!B.v) return MEHDG_OK;
    const int64_t len = 5 * (int64_t)g.Nn, tl = 5 * (int64_t)g.n2;
    gather_elems_kernel<<<blocks_for(n * len), 256, 0, st>>>(g.sv, B.v, B.d_voff, 1, g.d_elems, k0, n, len);
    if (B.vs) gather_elems_kernel<<<blocks_for(n * len), 256, 0, st>>>(g.svs, B.vs, B.d_voff, 1, g.d_elems, k0, n, len);
    gather_sides_kernel<<<blocks_for(n * 6 * tl), 256, 0, st>>>(g.svh, B.vh, B.d_toff, B.d_gid, g.d_elems, k0, n, tl);
    MEHDG_COUNT(B.vs ? 3 : 2);
    if (c->prm.viscous) {
        gather_elems_kernel<<<blocks_for(n * 3 * len), 256, 0, st>>>(g.sq, B.q, B.d_voff, 3, g.d_elems, k0, n, 3 * len);
        MEHDG_COUNT(1);
    }
    BTRY(cudaGetLastError());
    return mehdg_set_state(s, g.sv, g.svh, c->prm.viscous ? g.sq : nullptr, B.vs ? g.svs : nullptr, st);
}

// restore a resident sub-context to its full element count after a wave
void restore_full(Group& g) {
    if (g.sub && g.sub->nK != g.sub_cap) {
        g.sub->nK = g.sub_cap;
        g.sub->G = 6 * g.sub_cap;
        if (g.sub->lu_graph) { cudaGraphExecDestroy(g.sub->lu_graph); g.sub->lu_graph = nullptr; }
    }
}

int scatter_elem_out(mehdg_ctx* c, Group& g, double* dst, const double* src, int64_t scale, int64_t k0, int64_t n,
                     cudaStream_t st) {
    if (!dst) return MEHDG_OK;
    const int64_t len = scale * 5 * (int64_t)g.Nn;
    scatter_elems_kernel<<<blocks_for(n * len), 256, 0, st>>>(dst, src, c->batch->d_voff, scale, g.d_elems, k0, n, len);
    MEHDG_COUNT(1);
    BTRY(cudaGetLastError());
    return MEHDG_OK;
}

int scatter_side_out(mehdg_ctx* c, Group& g, const double* src, int64_t k0, int64_t n, cudaStream_t st) {
    const int64_t tl = 5 * (int64_t)g.n2;
    scatter_sides_kernel<<<blocks_for(n * 6 * tl), 256, 0, st>>>(c->batch->d_sides, src, c->batch->d_soff, g.d_elems,
                                                                 k0, n, tl);
    MEHDG_COUNT(1);
    BTRY(cudaGetLastError());
    return MEHDG_OK;
}

int scatter_status(mehdg_ctx* c, Group& g, int64_t k0, int64_t n, cudaStream_t st) {
    scatter_status_kernel<<<blocks_for(n), 256, 0, st>>>(c->d_status, g.sub->d_status, g.d_elems, k0, n);
    scatter_status_kernel<<<blocks_for(n), 256, 0, st>>>(c->d_iters, g.sub->d_iters, g.d_elems, k0, n);
    MEHDG_COUNT(2);
    BTRY(cudaGetLastError());
    return MEHDG_OK;
}

int face_sum(mehdg_ctx* c, double* out, cudaStream_t st) {
    face_sum_kernel<<<(unsigned)std::min<int64_t>(c->G, 65535), 128, 0, st>>>(out, c->batch->d_sides, c->batch->d_toff,
                                                                           c->batch->d_fside, c->G);
    MEHDG_COUNT(1);
    BTRY(cudaGetLastError());
    return MEHDG_OK;
}

// waves of a group: balanced, each at most g.wave elements
std::vector<std::pair<int64_t, int64_t>> waves(const Group& g) {
    const int64_t ng = (int64_t)g.elems.size();
    const int64_t nw = (ng + g.wave - 1) / g.wave;
    std::vector<std::pair<int64_t, int64_t>> w;
    int64_t k0 = 0;
    for (int64_t i = 0; i < nw; ++i) {
        const int64_t n = ng / nw + (i < ng % nw ? 1 : 0);
        w.push_back({k0, n});
        k0 += n;
    }
    return w;
}

int ensure_sub(mehdg_ctx* c, Group& g) {
    if (g.sub && g.sub_cap >= g.wave) return MEHDG_OK;
    return make_sub(c, g, g.wave);
}

void release_streaming(mehdg_ctx* c, Group& g) {
    if (!c->batch->resident) free_group_buffers(g);
    else restore_full(g);
}

}  // namespace

// ---------------------------------------------------------------- entry points used by api.cu
int batch_set_mesh(mehdg_ctx* c, int64_t nK, const int32_t* p, const int32_t* m, const double* box,
                   const int64_t* face_gid, int64_t G) {
    Batch* B = new Batch();
    c->batch = B;
    c->nK = nK; c->G = G;
    B->ep.assign(p, p + nK);
    B->em.assign(m, m + nK);
    B->box.assign(box, box + 6 * nK);
    // face sizes: both sides of a face need the same n; each face must be used
    std::vector<int> fn(G, 0);
    std::vector<int64_t> fside(2 * G, -1);
    B->voff.assign(nK + 1, 0);
    B->soff.assign(nK + 1, 0);
    for (int64_t K = 0; K < nK; ++K) {
        if (p[K] < 1 || p[K] > MEHDG_MAXP || m[K] < 1 || m[K] > 16) { set_err(c, "set_mesh: p in 1..4, m in 1..16"); return MEHDG_EINVAL; }
        if (c->prm.viscous && c->prm.prec == MEHDG_FP64 && p[K] > 3) { set_err(c, "set_mesh: the FP64 viscous Jacobian supports p <= 3"); return MEHDG_EINVAL; }
        const int n = m[K] * p[K] + 1;
        B->voff[K + 1] = B->voff[K] + 5 * (int64_t)n * n * n;
        B->soff[K + 1] = B->soff[K] + 30 * (int64_t)n * n;
        for (int d = 0; d < 3; ++d)
            if (!(box[6 * K + 3 + d] > box[6 * K + d])) { set_err(c, "set_mesh: degenerate box %lld", (long long)K); return MEHDG_EINVAL; }
        for (int f = 0; f < 6; ++f) {
            const int64_t g = face_gid[6 * K + f];
            if (g < 0 || g >= G) { set_err(c, "set_mesh: face id out of range"); return MEHDG_EINVAL; }
            if (fn[g] && fn[g] != n) { set_err(c, "set_mesh: face %lld joins elements of different n = m p + 1", (long long)g); return MEHDG_EINVAL; }
            fn[g] = n;
            const int64_t side = B->soff[K] + f * 5 * (int64_t)n * n;
            if (fside[2 * g] < 0) fside[2 * g] = side;
            else if (fside[2 * g + 1] < 0) fside[2 * g + 1] = side;
            else { set_err(c, "set_mesh: global face %lld used more than twice", (long long)g); return MEHDG_EINVAL; }
        }
    }
    B->toff.assign(G + 1, 0);
    for (int64_t g = 0; g < G; ++g) {
        if (!fn[g]) { set_err(c, "set_mesh: global face %lld is used by no element", (long long)g); return MEHDG_EINVAL; }
        B->toff[g + 1] = B->toff[g] + 5 * (int64_t)fn[g] * fn[g];
    }
    // groups by (p, m), decreasing cost per element
    std::vector<std::pair<int, int>> keys;
    for (int64_t K = 0; K < nK; ++K) keys.push_back({p[K], m[K]});
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (auto& k : keys) {
        Group g;
        g.p = k.first; g.m = k.second; g.n = g.m * g.p + 1; g.Nn = g.n * g.n * g.n; g.n2 = g.n * g.n;
        for (int64_t K = 0; K < nK; ++K) if (p[K] == g.p && m[K] == g.m) g.elems.push_back(K);
        const double Nv = 5.0 * g.Nn;
        g.cost = 2.0 / 3.0 * Nv * Nv * Nv + 2.0 * 4 * Nv * Nv + 2.0e3 * g.Nn;
        g.bytes_per_elem = bytes_per_element(c->prm, g.p, g.m);
        B->groups.push_back(std::move(g));
    }
    std::stable_sort(B->groups.begin(), B->groups.end(), [](const Group& a, const Group& b) { return a.cost > b.cost; });
    // memory budget: 60 % of the free device memory (MEHDG_BATCH_BUDGET_MB overrides)
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    B->budget = (size_t)(0.6 * (double)freeb);
    if (const char* e = std::getenv("MEHDG_BATCH_BUDGET_MB")) {
        const double mb = std::atof(e);
        if (mb > 0) B->budget = (size_t)(mb * 1048576.0);
    }
    size_t all = 0;
    for (auto& g : B->groups) all += g.bytes_per_elem * g.elems.size();
    B->resident = all <= B->budget;
    for (auto& g : B->groups) {
        const int64_t fit = (int64_t)(B->budget / std::max<size_t>(g.bytes_per_elem, 1));
        if (fit < 1) {
            set_err(c, "set_mesh: one element of p=%d m=%d needs %zu bytes, over the %zu-byte budget", g.p, g.m,
                    g.bytes_per_elem, B->budget);
            return MEHDG_ENOMEM;
        }
        g.wave = B->resident ? (int64_t)g.elems.size() : std::min<int64_t>((int64_t)g.elems.size(), fit);
    }
    // device tables
#define DAL(ptr, bytes) do { if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) { set_err(c, "set_mesh: cudaMalloc failed"); return MEHDG_ENOMEM; } } while (0)
    DAL(B->d_voff, sizeof(int64_t) * (nK + 1));
    DAL(B->d_soff, sizeof(int64_t) * (nK + 1));
    DAL(B->d_toff, sizeof(int64_t) * (G + 1));
    DAL(B->d_gid, sizeof(int64_t) * 6 * nK);
    DAL(B->d_fside, sizeof(int64_t) * 2 * G);
    DAL(B->d_sides, sizeof(double) * B->soff[nK]);
    DAL(c->d_status, sizeof(int32_t) * nK);
    DAL(c->d_iters, sizeof(int32_t) * nK);
    for (auto& g : B->groups) DAL(g.d_elems, sizeof(int64_t) * g.elems.size());
#undef DAL
    if (cudaMemcpy(B->d_voff, B->voff.data(), sizeof(int64_t) * (nK + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_soff, B->soff.data(), sizeof(int64_t) * (nK + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_toff, B->toff.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_gid, face_gid, sizeof(int64_t) * 6 * nK, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_fside, fside.data(), sizeof(int64_t) * 2 * G, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int32_t) * nK) != cudaSuccess ||
        cudaMemset(c->d_iters, 0, sizeof(int32_t) * nK) != cudaSuccess) {
        set_err(c, "set_mesh: copy failed");
        return MEHDG_ECUDA;
    }
    for (auto& g : B->groups)
        if (cudaMemcpy(g.d_elems, g.elems.data(), sizeof(int64_t) * g.elems.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            set_err(c, "set_mesh: copy failed");
            return MEHDG_ECUDA;
        }
    if (B->resident)
        for (auto& g : B->groups) BRC(make_sub(c, g, g.wave));
    return MEHDG_OK;
}

int batch_free(mehdg_ctx* c) {
    Batch* B = c->batch;
    if (!B) return MEHDG_OK;
    for (auto& g : B->groups) { free_group_buffers(g); bfree(g.d_elems); }
    bfree(B->d_voff); bfree(B->d_soff); bfree(B->d_toff); bfree(B->d_gid); bfree(B->d_fside); bfree(B->d_sides);
    delete B;
    c->batch = nullptr;
    return MEHDG_OK;
}

int batch_set_state(mehdg_ctx* c, const double* v, const double* vhat, const double* q, const double* vstar, cudaStream_t st) {
    Batch& B = *c->batch;
    B.v = v; B.vh = vhat; B.q = q; B.vs = vstar;
    c->v = v; c->vh = vhat; c->q = q; c->vs = vstar;
    c->condensed = false;
    if (B.resident)
        for (auto& g : B.groups) { restore_full(g); BRC(load_wave(c, g, 0, (int64_t)g.elems.size(), st)); }
    return MEHDG_OK;
}

int batch_residual(mehdg_ctx* c, double* R_V, double* R_Q, double* R_Vhat, cudaStream_t st) {
    Batch& B = *c->batch;
    BTRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * c->nK, st));
    for (auto& g : B.groups) {
        BRC(ensure_sub(c, g));
        for (auto [k0, n] : waves(g)) {
            if (!B.resident || n != (int64_t)g.elems.size()) BRC(load_wave(c, g, k0, n, st));
            BRC(mehdg_residual(g.sub, g.sRV, c->prm.viscous ? g.sRQ : nullptr, g.sRH, st));
            BRC(scatter_elem_out(c, g, R_V, g.sRV, 1, k0, n, st));
            if (c->prm.viscous) BRC(scatter_elem_out(c, g, R_Q, g.sRQ, 3, k0, n, st));
            BRC(scatter_side_out(c, g, g.sRH, k0, n, st));
            BRC(scatter_status(c, g, k0, n, st));
        }
        release_streaming(c, g);
    }
    return face_sum(c, R_Vhat, st);
}

int batch_condense(mehdg_ctx* c, double* bhat, cudaStream_t st) {
    Batch& B = *c->batch;
    BTRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * c->nK, st));
    BTRY(cudaMemsetAsync(c->d_iters, 0, sizeof(int32_t) * c->nK, st));
    for (auto& g : B.groups) {
        BRC(ensure_sub(c, g));
        for (auto [k0, n] : waves(g)) {
            if (!B.resident || n != (int64_t)g.elems.size()) BRC(load_wave(c, g, k0, n, st));
            const int rc = mehdg_condense(g.sub, g.sbh, nullptr, st);
            if (rc) { set_err(c, "batch group p=%d m=%d: %s", g.p, g.m, mehdg_last_error(g.sub)); return rc; }
            BRC(scatter_side_out(c, g, g.sbh, k0, n, st));
            BRC(scatter_status(c, g, k0, n, st));
        }
        release_streaming(c, g);
    }
    c->condensed = B.resident;
    return face_sum(c, bhat, st);
}

// resident batches only: y = sum_K A-hat^K x_K (apply), or dV, dQ (recover)
int batch_apply(mehdg_ctx* c, const double* x, double* y, cudaStream_t st) {
    Batch& B = *c->batch;
    for (auto& g : B.groups) {
        const int64_t n = (int64_t)g.elems.size(), tl = 5 * (int64_t)g.n2;
        gather_sides_kernel<<<blocks_for(n * 6 * tl), 256, 0, st>>>(g.sx, x, B.d_toff, B.d_gid, g.d_elems, 0, n, tl);
        MEHDG_COUNT(1);
        BRC(mehdg_apply_condensed(g.sub, g.sx, g.sy, st));
        BRC(scatter_side_out(c, g, g.sy, 0, n, st));
    }
    return face_sum(c, y, st);
}

int batch_recover(mehdg_ctx* c, const double* dVhat, double* dV, double* dQ, cudaStream_t st) {
    Batch& B = *c->batch;
    for (auto& g : B.groups) {
        const int64_t n = (int64_t)g.elems.size(), tl = 5 * (int64_t)g.n2;
        gather_sides_kernel<<<blocks_for(n * 6 * tl), 256, 0, st>>>(g.sx, dVhat, B.d_toff, B.d_gid, g.d_elems, 0, n, tl);
        MEHDG_COUNT(1);
        BRC(mehdg_recover(g.sub, g.sx, g.sdV, c->prm.viscous ? g.sdQ : nullptr, st));
        BRC(scatter_elem_out(c, g, dV, g.sdV, 1, 0, n, st));
        if (c->prm.viscous) BRC(scatter_elem_out(c, g, dQ, g.sdQ, 3, 0, n, st));
        BRC(scatter_status(c, g, 0, n, st));
    }
    return MEHDG_OK;
}

int64_t batch_state_len(const mehdg_ctx* c) { return c->batch->voff.back(); }

// the stage term's step of every sub-context (new ones copy the parameters)
int batch_set_dt(mehdg_ctx* c) {
    for (auto& g : c->batch->groups)
        if (g.sub) BRC(mehdg_set_dt(g.sub, c->prm.dt));
    return MEHDG_OK;
}
int64_t batch_trace_len(const mehdg_ctx* c) { return c->batch->toff.back(); }

// ---------------------------------------------------------------- autotuner
namespace {

// device time of one condensation of the group's first `n` elements
int time_trial(mehdg_ctx* c, Group& g, int64_t n, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    BTRY(cudaEventCreate(&e0));
    BTRY(cudaEventCreate(&e1));
    int rc = load_wave(c, g, 0, n, st);
    if (!rc) rc = mehdg_condense(g.sub, g.sbh, nullptr, st);            // warm-up (graph capture)
    if (!rc) {
        cudaEventRecord(e0, st);
        rc = mehdg_condense(g.sub, g.sbh, nullptr, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rc = MEHDG_ECUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc && g.sub) set_err(c, "autotune p=%d m=%d: %s", g.p, g.m, mehdg_last_error(g.sub));
    return rc;
}

void set_choice(Group& g, int leaf, int solve) {
    g.leaf_ctas = leaf; g.solve_ctas = solve;
    if (g.sub) {
        g.sub->tune_leaf_ctas = leaf;
        g.sub->tune_solve_ctas = solve;
        if (g.sub->lu_graph) { cudaGraphExecDestroy(g.sub->lu_graph); g.sub->lu_graph = nullptr; }
    }
}

}  // namespace

int batch_autotune(mehdg_ctx* c, int64_t trial_max, cudaStream_t st) {
    Batch& B = *c->batch;
    if (!B.v) { set_err(c, "autotune before set_state"); return MEHDG_ESTATE; }
    for (auto& g : B.groups) {
        BRC(ensure_sub(c, g));
        const int64_t n = std::min<int64_t>({(int64_t)g.elems.size(), g.wave, std::max<int64_t>(trial_max, 1)});
        char buf[160];
        g.tune_log.clear();
        // greedy: leaf CTAs per SM first (solves automatic), then the solve's CTAs per element
        float best = 1e30f;
        int bl = 0, bs = 0;
        for (int leaf : {1, 2, 4}) {
            set_choice(g, leaf, 0);
            float ms = 0.f;
            BRC(time_trial(c, g, n, st, &ms));
            snprintf(buf, sizeof(buf), "%s{\"leaf_ctas\":%d,\"solve_ctas\":0,\"ms\":%.4f}", g.tune_log.empty() ? "" : ",", leaf, ms);
            g.tune_log += buf;
            if (ms < best) { best = ms; bl = leaf; }
        }
        for (int sc : {1, 2, 4, 8}) {
            set_choice(g, bl, sc);
            float ms = 0.f;
            BRC(time_trial(c, g, n, st, &ms));
            snprintf(buf, sizeof(buf), ",{\"leaf_ctas\":%d,\"solve_ctas\":%d,\"ms\":%.4f}", bl, sc, ms);
            g.tune_log += buf;
            if (ms < best) { best = ms; bs = sc; }
        }
        set_choice(g, bl, bs);
        g.tuned = true;
        snprintf(buf, sizeof(buf), "],\"trial_elements\":%lld,\"best_ms\":%.4f", (long long)n, best);
        g.tune_log = "[" + g.tune_log + buf;
        release_streaming(c, g);
        if (B.resident) BRC(load_wave(c, g, 0, (int64_t)g.elems.size(), st));
    }
    c->condensed = false;
    return MEHDG_OK;
}

int batch_report(const mehdg_ctx* c, char* buf, size_t len) {
    const Batch& B = *c->batch;
    std::string s = "{\"resident\":";
    s += B.resident ? "true" : "false";
    char t[256];
    snprintf(t, sizeof(t), ",\"budget_bytes\":%zu,\"groups\":[", B.budget);
    s += t;
    for (size_t i = 0; i < B.groups.size(); ++i) {
        const Group& g = B.groups[i];
        snprintf(t, sizeof(t),
                 "%s{\"p\":%d,\"m\":%d,\"elements\":%zu,\"wave\":%lld,\"cost_flop\":%.4g,\"bytes_per_element\":%zu,"
                 "\"leaf_ctas\":%d,\"solve_ctas\":%d,\"tuned\":%s",
                 i ? "," : "", g.p, g.m, g.elems.size(), (long long)g.wave, g.cost, g.bytes_per_elem, g.leaf_ctas,
                 g.solve_ctas, g.tuned ? "true" : "false");
        s += t;
        if (g.tuned) s += ",\"trials\":" + g.tune_log;
        s += "}";
    }
    s += "]}";
    if (buf && len) {
        std::strncpy(buf, s.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    return (int)s.size();
}

void batch_layout(const mehdg_ctx* c, int64_t* voff, int64_t* toff) {
    const Batch& B = *c->batch;
    if (voff) std::memcpy(voff, B.voff.data(), sizeof(int64_t) * B.voff.size());
    if (toff) std::memcpy(toff, B.toff.data(), sizeof(int64_t) * B.toff.size());
}

bool batch_resident(const mehdg_ctx* c) { return c->batch && c->batch->resident; }

void batch_set_graph_refine(mehdg_ctx* c, bool on) {
    for (auto& g : c->batch->groups)
        if (g.sub) g.sub->graph_refine = on;
}

void batch_mark_condensed(mehdg_ctx* c) {
    for (auto& g : c->batch->groups)
        if (g.sub) g.sub->condensed = true;
}

void batch_end_captures(mehdg_ctx* c) {
    for (auto& g : c->batch->groups)
        if (g.sub) end_captures(g.sub);
}
