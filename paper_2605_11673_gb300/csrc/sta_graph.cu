// CUDA-graph mode of a context (sta_graph_enable): the per-frame device work of the streaming
// update, of the refold and of the full rebuild is captured once and replayed with one
// cudaGraphLaunch per call.  The streaming graph reads the number of edited tetrahedra from
// device memory and uses grids sized for a fixed capacity, so the same graph serves frames of
// any size up to that capacity (larger frames take the regular launch path).
#include "sta_internal.cuh"

namespace sta {

void graph_release(Ctx *c) {
    for (int b = 0; b < 2; ++b) {  // a frame still reading its staging block finishes first
        if (c->g_pending[b] && c->g_done[b]) cudaEventSynchronize(c->g_done[b]);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->g_streams[b]) cudaGraphExecDestroy(c->g_streams[b]);
        if (c->h_gframe[b]) cudaFreeHost(c->h_gframe[b]);
        if (c->g_done[b]) cudaEventDestroy(c->g_done[b]);
        c->g_streams[b] = nullptr;
        c->h_gframe[b] = c->m_gframe[b] = nullptr;
        c->g_done[b] = nullptr;
        c->g_pending[b] = false;
    }
    if (c->g_refold) cudaGraphExecDestroy(c->g_refold);
    if (c->g_rebuild) cudaGraphExecDestroy(c->g_rebuild);
    if (c->d_gcnt) cudaFree(c->d_gcnt);
    c->g_refold = c->g_rebuild = nullptr;
    c->d_gcnt = nullptr;
    c->graph_on = false;
    c->g_next = 0;
    c->gcap = 0;
}

namespace {

// Keep the last frame's touched counts when the graph staging goes away (sta_last_touched).
int keep_last_counters(Ctx *c) {
    if (c->d_gcnt && (c->last_counters == c->d_gcnt || c->last_counters == c->d_gcnt + 4)) {
        STA_CUDA_TRY(cudaMemcpy(c->counters + 1, c->last_counters + 1,
                                3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice));
        c->last_counters = c->counters;
    }
    return STA_OK;
}

template <typename F> int capture(cudaStream_t cs, F &&body, cudaGraphExec_t *exec) {
    cudaGraph_t g = nullptr;
    STA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = body(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != STA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(STA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return fail(STA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return STA_OK;
}

}  // namespace
}  // namespace sta

using namespace sta;

extern "C" int sta_graph_enable(sta_ctx *x, int64_t max_edited, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (max_edited < 1 || max_edited > (INT32_MAX / 32))
        return fail(STA_EINVAL, "max_edited must be in [1, 2^26]");
    Ctx *c = &x->c;
    STA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    STA_TRY(keep_last_counters(c));
    graph_release(c);
    int rc = STA_OK;
    cudaStream_t cs = nullptr;
    auto bail = [&](int code) {
        if (cs) cudaStreamDestroy(cs);
        graph_release(c);
        return code;
    };
    if (cudaMalloc((void **)&c->d_gcnt, 8 * sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(STA_ENOMEM, "graph counters"));
    for (int b = 0; b < 2; ++b) {
        void *dp = nullptr;
        if (cudaHostAlloc((void **)&c->h_gframe[b], frame_bytes(max_edited), cudaHostAllocMapped) !=
                cudaSuccess ||
            cudaHostGetDevicePointer(&dp, c->h_gframe[b], 0) != cudaSuccess)
            return bail(fail(STA_ENOMEM, "graph staging buffers (host-mapped)"));
        c->m_gframe[b] = static_cast<FrameHeader *>(dp);
        if (cudaEventCreateWithFlags(&c->g_done[b], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(STA_ECUDA, "graph event"));
    }
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(STA_ECUDA, "graph stream"));
    // both counter sets start at zero; each frame's last kernel then zeroes the other set for
    // the frame after it (the two sequences alternate), so the sequences carry no memset node
    // (a memset node at the head of the graph delayed its first kernel by about 2 us)
    if (cudaMemsetAsync(c->d_gcnt, 0, 8 * sizeof(unsigned long long), cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
        return bail(fail(STA_ECUDA, "graph counters"));
    c->gcap = max_edited;
    for (int b = 0; b < 2; ++b) {
        unsigned long long *cnt = c->d_gcnt + 4 * b, *next = c->d_gcnt + 4 * (b ^ 1);
        FrameHeader *fb = c->m_gframe[b];
        if ((rc = capture(cs, [&](cudaStream_t s) {
                 return launch_stream_frame(c, frame_edited(fb), &fb->m, cnt, c->gcap, s, next);
             }, &c->g_streams[b])))
            return bail(rc);
    }
    if ((rc = capture(cs, [&](cudaStream_t s) { return launch_values(c, s); }, &c->g_refold)))
        return bail(rc);
    if ((rc = capture(cs, [&](cudaStream_t s) {
             int r = launch_mask_bits(c, s);
             return r != STA_OK ? r : launch_values(c, s);
         }, &c->g_rebuild)))
        return bail(rc);
    cudaStreamDestroy(cs);
    c->graph_on = true;
    return STA_OK;
}

extern "C" int sta_graph_disable(sta_ctx *x, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    STA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    STA_TRY(keep_last_counters(&x->c));
    graph_release(&x->c);
    return STA_OK;
}
