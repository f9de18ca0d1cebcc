// graph.cu -- the condensation of a context as one CUDA graph.
//
// mehdg_condense issues, per call, the residual and Jacobian kernels, the LU
// (already replayed from a graph of its own), and the FP64 refinement, whose
// sweeps synchronise the stream to test convergence.  For capture the
// refinement instead records every sweep up to refine_max_iter: elements
// that have converged skip their work on the device (their flags are set by
// the update kernel), so the result is the same as with the synchronising
// loop.  The captured condensation -- of one element type, or of every
// (p, m) group of a resident batch in order -- is replayed with one graph
// launch per call.
#include "common.cuh"
#include "kernels.cuh"

namespace {
// after a failed recording: no stream of the context (or of a batch's groups)
// may stay in capture mode
void end_capture_of(cudaStream_t s) {
    if (!s) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
    }
}
}  // namespace

void end_captures(mehdg_ctx* c) {
    end_capture_of(c->cap_stream);
    end_capture_of(c->lu_stream);
    if (c->batch) batch_end_captures(c);
    (void)cudaGetLastError();
}

extern "C" int mehdg_condense_graph(mehdg_ctx* c, double* bhat, void* stream) {
    if (!c) return MEHDG_EINVAL;
    if (!c->v && !c->batch) { set_err(c, "condense_graph before set_state"); return MEHDG_ESTATE; }
    if (!bhat) return MEHDG_EINVAL;
    if (c->batch && !batch_resident(c)) {
        set_err(c, "condense_graph: the batch is streamed in waves (it exceeds the memory budget)");
        return MEHDG_EINVAL;
    }
    if (c->prof.on) { set_err(c, "condense_graph: phase profiling is on"); return MEHDG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const void* key[7] = {c->v, c->vh, c->q, c->vs, c->src, bhat, c->batch};
    bool same = c->cond_graph != nullptr;
    for (int i = 0; i < 7 && same; ++i) same = key[i] == c->cap_key[i];
    cudaError_t e;
#define GTRY(x) do { if ((e = (x)) != cudaSuccess) { set_err(c, "%s: %s", #x, cudaGetErrorString(e)); return MEHDG_ECUDA; } } while (0)
    if (!same) {
        if (c->cond_graph) { cudaGraphExecDestroy(c->cond_graph); c->cond_graph = nullptr; }
        // one direct condensation first: workspaces, side streams and the LU graphs exist afterwards
        int rc = mehdg_condense(c, bhat, nullptr, stream);
        if (rc) return rc;
        GTRY(cudaStreamSynchronize(st));
        if (!c->cap_stream) GTRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (!c->cap_in) GTRY(cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming));
        if (!c->cap_out) GTRY(cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming));
        const long long before = g_mehdg_launches.load();
        GTRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
        c->graph_refine = true;
        if (c->batch) batch_set_graph_refine(c, true);
        rc = mehdg_condense(c, bhat, nullptr, c->cap_stream);
        c->graph_refine = false;
        if (c->batch) batch_set_graph_refine(c, false);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        if (rc == MEHDG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->cond_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (rc != MEHDG_OK || e != cudaSuccess) end_captures(c);
        c->cond_graph_launches = g_mehdg_launches.load() - before;
        g_mehdg_launches = before;                      // counted when the graph runs
        if (rc) { c->cond_graph = nullptr; return rc; }
        if (e != cudaSuccess) {
            c->cond_graph = nullptr;
            (void)cudaGetLastError();
            set_err(c, "condense_graph: capture failed: %s", cudaGetErrorString(e));
            return MEHDG_ECUDA;
        }
        for (int i = 0; i < 7; ++i) c->cap_key[i] = key[i];
    }
    GTRY(cudaEventRecord(c->cap_in, st));
    GTRY(cudaStreamWaitEvent(c->cap_stream, c->cap_in, 0));
    GTRY(cudaGraphLaunch(c->cond_graph, c->cap_stream));
    GTRY(cudaEventRecord(c->cap_out, c->cap_stream));
    GTRY(cudaStreamWaitEvent(st, c->cap_out, 0));
    g_mehdg_launches += c->cond_graph_launches;
    c->condensed = c->batch ? batch_resident(c) : true;
    if (c->batch) batch_mark_condensed(c);
    return MEHDG_OK;
#undef GTRY
}
