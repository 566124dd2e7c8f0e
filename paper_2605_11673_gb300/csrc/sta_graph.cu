// CUDA-graph mode of a context (sta_graph_enable): the per-frame device work of the streaming
// update, of the refold and of the full rebuild is captured once and replayed with one
// cudaGraphLaunch per call.  The streaming graph reads the number of edited tetrahedra from
// device memory and uses grids sized for a fixed capacity, so the same graph serves frames of
// any size up to that capacity (larger frames take the regular launch path).
#include "sta_internal.cuh"

namespace sta {

void graph_release(Ctx *c) {
    if (c->g_stream) cudaGraphExecDestroy(c->g_stream);
    if (c->g_refold) cudaGraphExecDestroy(c->g_refold);
    if (c->g_rebuild) cudaGraphExecDestroy(c->g_rebuild);
    if (c->d_gframe) cudaFree(c->d_gframe);
    if (c->h_gframe) cudaFreeHost(c->h_gframe);
    if (c->g_h2d) cudaEventDestroy(c->g_h2d);
    c->g_stream = c->g_refold = c->g_rebuild = nullptr;
    c->d_gframe = c->h_gframe = nullptr;
    c->g_h2d = nullptr;
    c->graph_on = false;
    c->g_pending = false;
    c->gcap = 0;
}

namespace {

// Keep the last frame's touched counts when the graph staging goes away (sta_last_touched).
int keep_last_counters(Ctx *c) {
    if (c->d_gframe && c->last_counters == frame_counters(c->d_gframe)) {
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
    if (cudaMalloc((void **)&c->d_gframe, frame_bytes(max_edited)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_gframe, frame_bytes(max_edited)) != cudaSuccess)
        return bail(fail(STA_ENOMEM, "graph staging buffers"));
    if (cudaEventCreateWithFlags(&c->g_h2d, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(STA_ECUDA, "graph stream/event"));
    c->gcap = max_edited;
    if ((rc = capture(cs, [&](cudaStream_t s) {
             return launch_stream_frame(c, c->d_gframe, c->gcap, s);
         }, &c->g_stream)))
        return bail(rc);
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
