// Allocation-free streaming update (sta_apply_edits_noalloc, declared in include/sta.h).
//
// sta_apply_edits may allocate: its first call, and any call with more edited tetrahedra
// than before, grows a pinned host buffer and a device buffer.  Some callers cannot allow
// that -- a frame loop that must never hit cudaMalloc's implicit device synchronisation, or a
// process whose device memory is owned by a framework's caching allocator.  This variant
// keeps its per-call scratch (edited-tet list, touched-unit list, counters) in one
// file-scope device array of fixed size, so it calls no allocator at all.
#include <mutex>

#include "sta_internal.cuh"

namespace {

constexpr int64_t kMaxEdited = STA_NOALLOC_MAX_EDITED;
// Every writer of the touched list (k_stream_claim, k_fx_claim, k_proxy_claim) appends at
// most one entry per unit slot of an edited tetrahedron, and a tetrahedron has 10 slots (4
// diagonal, 6 node pairs).
constexpr int64_t kMaxTouched = 10 * kMaxEdited;
// layout: counters (4 x u64) | edited tets (kMaxEdited x i32) | touched units (kMaxTouched x i32)
constexpr size_t kCountersBytes = 4 * sizeof(unsigned long long);
constexpr size_t kScratchBytes =
    kCountersBytes + sizeof(int32_t) * (size_t)kMaxEdited + sizeof(int32_t) * (size_t)kMaxTouched;

// Resident on every GPU that loads the library, until the process exits.  Host code must not
// pass its name to a kernel: on the host it is only a stand-in, the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;                      // guards the set-up table and the host staging array
unsigned char *g_dev_addr[kMaxDevices];  // device address of g_scratch, per device
int32_t g_host_stage[kMaxEdited];        // edited tets (id | new state << 31), host side

}  // namespace

using namespace sta;

extern "C" int sta_apply_edits_noalloc(sta_ctx *x, const sta_edit *edits, int64_t n_edits,
                                       void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (n_edits < 0 || (n_edits > 0 && !edits)) return fail(STA_EINVAL, "bad edit list");
    int dev = -1;
    STA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(STA_EINVAL, "the context's device must be current for this call");
    if (dev < 0 || dev >= kMaxDevices) return fail(STA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_addr[dev]) {  // one-time set-up on this device
        void *p = nullptr;
        STA_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
        g_dev_addr[dev] = static_cast<unsigned char *>(p);
    }
    // validate against the host mirror of the mask (nothing changes on a bad edit)
    int64_t m = 0, bad = -1;
    std::string why;
    for (int64_t e = 0; e < n_edits; ++e) {
        const sta_edit &E = edits[e];
        if (E.op < 0 || E.op > 2) { bad = e; why = "bad op"; break; }
        if (E.tet < 0 || E.tet >= c->T) { bad = e; why = "tet out of range"; break; }
        if (c->seen[E.tet]) { bad = e; why = "tet named twice"; break; }
        c->seen[E.tet] = 1;
        if (E.op == STA_DEACTIVATE && !ts_active(c, E.tet)) { bad = e; why = "deactivating an inactive tet"; break; }
        if (E.op == STA_ACTIVATE && ts_active(c, E.tet)) { bad = e; why = "activating an active tet"; break; }
        if (E.op == STA_SWAP) {
            if (E.tet2 < 0 || E.tet2 >= c->T) { bad = e; why = "tet2 out of range"; break; }
            if (c->seen[E.tet2]) { bad = e; why = "tet2 named twice"; break; }
            c->seen[E.tet2] = 1;
            if (!ts_active(c, E.tet) || ts_active(c, E.tet2)) { bad = e; why = "swap needs an active tet and an inactive tet2"; break; }
            ++m;
        }
        ++m;
    }
    for (int64_t e = 0; e < n_edits; ++e) {
        if (edits[e].tet >= 0 && edits[e].tet < c->T) c->seen[edits[e].tet] = 0;
        if (edits[e].op == STA_SWAP && edits[e].tet2 >= 0 && edits[e].tet2 < c->T)
            c->seen[edits[e].tet2] = 0;
    }
    if (bad >= 0) return fail(STA_EINVAL, "edit " + std::to_string(bad) + ": " + why);
    if (m > kMaxEdited)
        return fail(STA_ERANGE, "sta_apply_edits_noalloc: " + std::to_string(m) +
                                    " edited tetrahedra exceed the fixed maximum of " +
                                    std::to_string(kMaxEdited) + " per call");
    int64_t k = 0;
    for (int64_t e = 0; e < n_edits; ++e) {
        const sta_edit &E = edits[e];
        if (E.op == STA_DEACTIVATE) {
            g_host_stage[k++] = E.tet;
            ts_set_active(c, E.tet, false);
            --c->n_active;
        } else if (E.op == STA_ACTIVATE) {
            g_host_stage[k++] = (int32_t)((uint32_t)E.tet | 0x80000000u);
            ts_set_active(c, E.tet, true);
            ++c->n_active;
        } else {
            g_host_stage[k++] = E.tet;
            g_host_stage[k++] = (int32_t)((uint32_t)E.tet2 | 0x80000000u);
            ts_set_active(c, E.tet, false);
            ts_set_active(c, E.tet2, true);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = g_dev_addr[dev];
    auto *counters = reinterpret_cast<unsigned long long *>(base);
    auto *d_edited = reinterpret_cast<int32_t *>(base + kCountersBytes);
    int32_t *touched = d_edited + kMaxEdited;
    if (m > 0)  // pageable source: the copy is staged before this call returns
        STA_CUDA_TRY(cudaMemcpyAsync(d_edited, g_host_stage, sizeof(int32_t) * m,
                                     cudaMemcpyHostToDevice, s));
    return launch_stream_scratch(c, m, d_edited, touched, counters, s);
}
