// prof.cuh -- optional CUDA-event timing of the phases of a Newton step, on
// the caller's stream (off by default; no cost when off).
#pragma once
#include <vector>
#include <cuda_runtime.h>

enum { PH_RESIDUAL = 0, PH_JACOBIAN, PH_LU_PANELS, PH_GEMM_OUTER, PH_SOLVE, PH_TANGENT, PH_PACK_OUTER, PH_N };

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec { int ph; int e0, e1; double flops; };
    std::vector<Rec> recs;
};

inline int prof_begin(Prof* p, int ph, cudaStream_t st) {
    if (!p || !p->on) return -1;
    while (p->pool.size() < p->used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        p->pool.push_back(e);
    }
    Prof::Rec r{ph, (int)p->used, (int)p->used + 1, 0.0};
    p->used += 2;
    cudaEventRecord(p->pool[r.e0], st);
    p->recs.push_back(r);
    return (int)p->recs.size() - 1;
}

inline void prof_end(Prof* p, int idx, cudaStream_t st, double flops) {
    if (!p || !p->on || idx < 0) return;
    cudaEventRecord(p->pool[p->recs[idx].e1], st);
    p->recs[idx].flops = flops;
}

inline bool prof_enable(Prof* p, int on) {
    p->on = on != 0;
    p->recs.clear();
    p->used = 0;
    return true;
}

inline void prof_read(Prof* p, double* ms, int64_t* n, double* flops, int nph) {
    for (int i = 0; i < nph; ++i) { ms[i] = 0; n[i] = 0; flops[i] = 0; }
    for (auto& r : p->recs) {
        if (r.ph >= nph) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->pool[r.e0], p->pool[r.e1]) == cudaSuccess) ms[r.ph] += t;
        n[r.ph] += 1;
        flops[r.ph] += r.flops;
    }
}

inline void prof_free(Prof* p) {
    for (auto e : p->pool) cudaEventDestroy(e);
    p->pool.clear(); p->recs.clear(); p->used = 0; p->on = false;
}
