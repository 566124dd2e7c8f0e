// C-ABI entry points of libsta (declared in include/sta.h): argument and edit validation on
// the host, device memory management, and the launch sequence of each call.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sta_internal.cuh"

namespace sta {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

}  // namespace sta

using namespace sta;


// The host mirror of a new mask (and its 0/1 staging copy); returns the active count.  Plain
// byte loops over restrict pointers, which the compiler vectorises.
static int64_t set_host_mask(Ctx *c, const uint8_t *__restrict__ mask, uint8_t *__restrict__ stage) {
    uint8_t *__restrict__ ts = c->tstate.data();
    const int64_t T = c->T;
    int64_t na = 0;
    for (int64_t t = 0; t < T; ++t) {
        const uint8_t on = mask[t] != 0;
        ts[t] = (uint8_t)((ts[t] & TS_STAMP) | (on << 7));
        na += on;
    }
    if (stage)
        for (int64_t t = 0; t < T; ++t) stage[t] = mask[t] != 0;
    return na;
}

static int wait_staging(sta_ctx *x) {
    if (x->h2d_pending) {
        STA_CUDA_TRY(cudaEventSynchronize(x->h2d_done));
        x->h2d_pending = false;
    }
    return STA_OK;
}

static void free_ctx(sta_ctx *x) {
    if (!x) return;
    for (void *p : x->c.allocations) cudaFree(p);
    x->c.allocations.clear();
    if (x->c.h_frame) cudaFreeHost(x->c.h_frame);
    if (x->c.d_frame) cudaFree(x->c.d_frame);
    if (x->h_mask) cudaFreeHost(x->h_mask);
    if (x->h_count) cudaFreeHost(x->h_count);
    if (x->c.h_count_mapped) cudaFreeHost(x->c.h_count_mapped);
    if (x->h2d_done) cudaEventDestroy(x->h2d_done);
    if (x->c.g_cg) cudaGraphExecDestroy(x->c.g_cg);
    graph_release(&x->c);
    delete x;
}

extern "C" {

void sta_default_options(sta_options *opt) {
    if (!opt) return;
    opt->eps = 0.0;
    opt->block_threads = 0;
    opt->blocks_per_sm = 0;
}

const char *sta_last_error(void) { return g_last_error.c_str(); }

const char *sta_status_string(int status) {
    switch (status) {
    case STA_OK: return "ok";
    case STA_EINVAL: return "invalid argument";
    case STA_ESTATE: return "invalid state";
    case STA_ERANGE: return "index range overflow";
    case STA_ENOMEM: return "out of memory";
    case STA_ECUDA: return "CUDA error";
    default: return "unknown status";
    }
}

int sta_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
               const double *young, const double *poisson, const sta_options *opt,
               void *stream, sta_ctx **out) {
    return sta::create_impl(nodes, n_nodes, tets, n_tets, young, poisson, opt, stream, out);
}

}  // extern "C"

int sta::create_impl(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                     const double *young, const double *poisson, const sta_options *opt,
                     void *stream, sta_ctx **out) {
    if (!out) return fail(STA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_nodes < 0 || n_tets < 0) return fail(STA_EINVAL, "negative size");
    if ((n_nodes > 0 && !nodes) || (n_tets > 0 && (!tets || !young || !poisson)))
        return fail(STA_EINVAL, "NULL input array");
    if (n_tets >= (1LL << 27)) return fail(STA_ERANGE, "n_tets must be < 2^27");
    if (n_tets * KE_STRIDE >= (1LL << 31))  // element cache offsets of the folds are 31-bit
        return fail(STA_ERANGE, "n_tets must be < 2^31 / " + std::to_string(KE_STRIDE));
    if (3 * n_nodes + 1 > INT32_MAX) return fail(STA_ERANGE, "3 * n_nodes + 1 exceeds int32");
    for (int64_t t = 0; t < n_tets; ++t) {
        const int32_t *q = tets + 4 * t;
        for (int a = 0; a < 4; ++a) {
            if (q[a] < 0 || q[a] >= n_nodes)
                return fail(STA_EINVAL, "tet " + std::to_string(t) + ": node id out of range");
            for (int b = 0; b < a; ++b)
                if (q[a] == q[b])
                    return fail(STA_EINVAL, "tet " + std::to_string(t) + ": repeated node");
        }
    }
    sta_options o;
    sta_default_options(&o);
    if (opt) o = *opt;
    if (o.block_threads != 0 && o.block_threads != 64 && o.block_threads != 128 && o.block_threads != 256)
        return fail(STA_EINVAL, "block_threads must be 64, 128 or 256");
    if (o.blocks_per_sm < 0) return fail(STA_EINVAL, "blocks_per_sm must be >= 0");

    cudaStream_t s = (cudaStream_t)stream;
    sta_ctx *x = new sta_ctx();
    Ctx *c = &x->c;
    c->n = n_nodes;
    c->T = n_tets;
    c->eps = o.eps;
    c->block_threads = o.block_threads ? o.block_threads : 128;
    c->blocks_per_sm = o.blocks_per_sm;
    int rc = STA_OK;
    auto bail = [&](int code) {
        free_ctx(x);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(fail(STA_ECUDA, "no CUDA device"));
    if (cudaEventCreateWithFlags(&x->h2d_done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(STA_ECUDA, "cudaEventCreate failed"));

    // inputs: nodes padded to double4_32a, tets as int4, materials as double2
    std::vector<double> X4(4 * (size_t)(n_nodes > 0 ? n_nodes : 1), 0.0);
    for (int64_t v = 0; v < n_nodes; ++v)
        for (int k = 0; k < 3; ++k) X4[4 * v + k] = nodes[3 * v + k];
    std::vector<double> M2(2 * (size_t)(n_tets > 0 ? n_tets : 1), 0.0);
    for (int64_t t = 0; t < n_tets; ++t) {
        M2[2 * t] = young[t];
        M2[2 * t + 1] = poisson[t];
    }
    if ((rc = dev_alloc(c, &c->X, n_nodes)) || (rc = dev_alloc(c, &c->tets, n_tets)) ||
        (rc = dev_alloc(c, &c->mat, n_tets)) || (rc = dev_alloc(c, &c->counters, 4)))
        return bail(rc);
    if (cudaMemcpyAsync(c->X, X4.data(), sizeof(double4_32a) * n_nodes, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(c->tets, tets, sizeof(int4) * n_tets, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(c->mat, M2.data(), sizeof(double2) * n_tets, cudaMemcpyHostToDevice, s))
        return bail(fail(STA_ECUDA, "input copy failed"));

    if ((rc = build_pattern(c, s))) return bail(rc);

    if ((rc = dev_alloc(c, &c->Ke, KE_STRIDE * n_tets)) || (rc = dev_alloc(c, &c->mask, n_tets)) ||
        (rc = dev_alloc(c, &c->val, c->nnz)))
        return bail(rc);
    unsigned long long init[4] = {0ull, 0ull, ~0ull, 0ull};
    if (cudaMemcpyAsync(c->counters, init, sizeof init, cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(c->mask, 0, (size_t)(n_tets > 0 ? n_tets : 1), s) ||
        cudaMemsetAsync(c->val, 0, sizeof(double) * (size_t)(c->nnz > 0 ? c->nnz : 1), s))
        return bail(fail(STA_ECUDA, "init failed"));
    if ((rc = launch_elements(c, false, s))) return bail(rc);
    unsigned long long back[4];
    if (cudaMemcpyAsync(back, c->counters, sizeof back, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return bail(fail(STA_ECUDA, std::string("element kernel failed: ") +
                                        cudaGetErrorString(cudaGetLastError())));
    if (back[0] != 0)
        return bail(fail(STA_EINVAL, std::to_string(back[0]) +
                                         " tetrahedra have det <= 0 (first: tet " +
                                         std::to_string(back[2]) + ")"));
    c->tstate.assign((size_t)n_tets, 0);
    c->seen.assign((size_t)n_tets, 0);
    c->last_counters = c->counters;
    if (cudaMallocHost((void **)&x->h_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void **)&x->h_mask, (size_t)(n_tets > 0 ? n_tets : 1)) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_count_mapped, sizeof(unsigned long long),
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_count_mapped, c->h_count_mapped, 0) != cudaSuccess)
        return bail(fail(STA_ENOMEM, "pinned host buffers"));
    *out = x;
    return STA_OK;
}

extern "C" int sta_proxy_create(int64_t n_nodes, const int32_t *tets, int64_t n_tets, double eps,
                                void *stream, sta_ctx **out) {
    if (!out) return fail(STA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_nodes < 0 || n_tets < 0) return fail(STA_EINVAL, "negative size");
    if (n_tets > 0 && !tets) return fail(STA_EINVAL, "NULL input array");
    if (n_tets >= (1LL << 27)) return fail(STA_ERANGE, "n_tets must be < 2^27");
    if (n_nodes + 1 > INT32_MAX) return fail(STA_ERANGE, "n_nodes + 1 exceeds int32");
    for (int64_t t = 0; t < n_tets; ++t) {
        const int32_t *q = tets + 4 * t;
        for (int a = 0; a < 4; ++a) {
            if (q[a] < 0 || q[a] >= n_nodes)
                return fail(STA_EINVAL, "tet " + std::to_string(t) + ": node id out of range");
            for (int b = 0; b < a; ++b)
                if (q[a] == q[b])
                    return fail(STA_EINVAL, "tet " + std::to_string(t) + ": repeated node");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    sta_ctx *x = new sta_ctx();
    Ctx *c = &x->c;
    c->op = STA_OP_PROXY;
    c->policy = STA_POLICY_FIXED;  // the maintained-count update; REFOLD recounts touched entries
    c->n = n_nodes;
    c->T = n_tets;
    c->eps = eps;
    int rc = STA_OK;
    auto bail = [&](int code) {
        free_ctx(x);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(fail(STA_ECUDA, "no CUDA device"));
    if (cudaEventCreateWithFlags(&x->h2d_done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(STA_ECUDA, "cudaEventCreate failed"));
    if ((rc = dev_alloc(c, &c->tets, n_tets)) || (rc = dev_alloc(c, &c->counters, 4)))
        return bail(rc);
    if (cudaMemcpyAsync(c->tets, tets, sizeof(int4) * n_tets, cudaMemcpyHostToDevice, s))
        return bail(fail(STA_ECUDA, "input copy failed"));
    if ((rc = build_pattern(c, s))) return bail(rc);
    if ((rc = dev_alloc(c, &c->mask, n_tets)) || (rc = dev_alloc(c, &c->val, c->nnz))) return bail(rc);
    unsigned long long init[4] = {0ull, 0ull, ~0ull, 0ull};
    if (cudaMemcpyAsync(c->counters, init, sizeof init, cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(c->mask, 0, (size_t)(n_tets > 0 ? n_tets : 1), s))
        return bail(fail(STA_ECUDA, "init failed"));
    if ((rc = launch_proxy_rebuild(c, s))) return bail(rc);  // all inactive: A = eps I
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return bail(fail(STA_ECUDA, std::string("proxy create: ") +
                                        cudaGetErrorString(cudaGetLastError())));
    c->tstate.assign((size_t)n_tets, 0);
    c->seen.assign((size_t)n_tets, 0);
    c->last_counters = c->counters;
    if (cudaMallocHost((void **)&x->h_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void **)&x->h_mask, (size_t)(n_tets > 0 ? n_tets : 1)) != cudaSuccess)
        return bail(fail(STA_ENOMEM, "pinned mask buffer"));
    *out = x;
    return STA_OK;
}

extern "C" {

int sta_destroy(sta_ctx *x) {
    if (!x) return STA_OK;
    cudaDeviceSynchronize();
    free_ctx(x);
    return STA_OK;
}

int sta_full_rebuild(sta_ctx *x, const uint8_t *mask, int mask_on_device, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (c->T > 0 && !mask) return fail(STA_EINVAL, "mask is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->T > 0) {
        STA_TRY(wait_staging(x));
        if (mask_on_device) {  // read back for the host mirror; the device copy is the 0/1 one
            std::vector<uint8_t> hm((size_t)c->T);
            STA_CUDA_TRY(cudaMemcpyAsync(hm.data(), mask, (size_t)c->T, cudaMemcpyDeviceToHost, s));
            STA_CUDA_TRY(cudaStreamSynchronize(s));
            c->n_active = set_host_mask(c, hm.data(), x->h_mask);
        } else {
            c->n_active = set_host_mask(c, mask, x->h_mask);
        }
        STA_CUDA_TRY(cudaMemcpyAsync(c->mask, x->h_mask, (size_t)c->T, cudaMemcpyHostToDevice, s));
        STA_CUDA_TRY(cudaEventRecord(x->h2d_done, s));
        x->h2d_pending = true;
    }
    if (c->graph_on) {
        STA_CUDA_TRY(cudaGraphLaunch(c->g_rebuild, s));
        return STA_OK;
    }
    STA_TRY(launch_mask_bits(c, s));
    return launch_values(c, s);
}

int sta_set_launch(sta_ctx *x, int32_t block_threads, int32_t blocks_per_sm) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (block_threads != 0 && block_threads != 64 && block_threads != 128 && block_threads != 256)
        return fail(STA_EINVAL, "block_threads must be 0, 64, 128 or 256");
    if (blocks_per_sm < 0) return fail(STA_EINVAL, "blocks_per_sm must be >= 0");
    if (x->c.graph_on) return fail(STA_ESTATE, "disable graph mode before changing the launch shape");
    x->c.block_threads = block_threads ? block_threads : 128;
    x->c.blocks_per_sm = blocks_per_sm;
    return STA_OK;
}

int sta_set_fold_depth(sta_ctx *x, int32_t operands_in_flight) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (operands_in_flight != 4 && operands_in_flight != 6)
        return fail(STA_EINVAL, "operands_in_flight must be 4 or 6");
    if (x->c.graph_on) return fail(STA_ESTATE, "disable graph mode before changing the fold depth");
    x->c.fold_depth = operands_in_flight;
    return STA_OK;
}

int sta_set_rebuild_form(sta_ctx *x, int32_t form) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (form != STA_REBUILD_AUTO && form != STA_REBUILD_FUSED && form != STA_REBUILD_ZERO_FILL)
        return fail(STA_EINVAL, "form must be STA_REBUILD_AUTO, _FUSED or _ZERO_FILL");
    if (x->c.graph_on) return fail(STA_ESTATE, "disable graph mode before changing the rebuild form");
    x->c.rebuild_form = form;
    return STA_OK;
}

int sta_get_rebuild_form(const sta_ctx *x, int32_t *form) {
    if (!x || !form) return fail(STA_EINVAL, "NULL argument");
    *form = rebuild_form_of(&x->c);
    return STA_OK;
}

int sta_refold(sta_ctx *x, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (x->c.graph_on) {
        STA_CUDA_TRY(cudaGraphLaunch(x->c.g_refold, (cudaStream_t)stream));
        return STA_OK;
    }
    return launch_values(&x->c, (cudaStream_t)stream);
}

int sta_apply_edits(sta_ctx *x, const sta_edit *edits, int64_t n_edits, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (n_edits < 0 || (n_edits > 0 && !edits)) return fail(STA_EINVAL, "bad edit list");
    if (n_edits > (INT32_MAX / 32)) return fail(STA_ERANGE, "too many edits in one call");
    cudaStream_t s = (cudaStream_t)stream;
    // edited tetrahedra (a swap edits two): 2 n_edits bounds them, which is all graph mode needs
    // to know when it is within the capacity; otherwise they are counted first.  Staging
    // counts them exactly either way.
    int64_t m = 2 * n_edits;
    if (!c->graph_on || m > c->gcap) {
        m = n_edits;
        for (int64_t e = 0; e < n_edits; ++e) m += edits[e].op == STA_SWAP;
    }

    // the frame block to stage into: one of the graph mode's two host-mapped blocks (fixed
    // capacity), or the context's pinned block (grown on demand)
    const bool use_graph = c->graph_on && m <= c->gcap;
    FrameHeader *h = nullptr, *d = nullptr;
    int gb = 0;
    if (use_graph) {  // the staging block last used two frames ago: its kernels are done
        gb = c->g_next;
        if (c->g_pending[gb]) {
            STA_CUDA_TRY(cudaEventSynchronize(c->g_done[gb]));
            c->g_pending[gb] = false;
        }
        h = c->h_gframe[gb];
        d = c->m_gframe[gb];
    } else {
        STA_TRY(wait_staging(x));
        if (m > c->edit_cap || !c->h_frame) {
            const int64_t cap = m < 1024 ? 1024 : m + m / 2;
            if (c->h_frame) cudaFreeHost(c->h_frame);
            c->h_frame = nullptr;
            if (c->d_frame) {
                if (c->last_counters == frame_counters(c->d_frame)) {
                    STA_CUDA_TRY(cudaMemcpyAsync(c->counters + 1, c->last_counters + 1,
                                                 3 * sizeof(unsigned long long),
                                                 cudaMemcpyDeviceToDevice, s));
                    c->last_counters = c->counters;
                }
                cudaFree(c->d_frame);  // implicit device synchronisation
                c->device_bytes -= (int64_t)frame_bytes(c->edit_cap);
            }
            c->d_frame = nullptr;
            c->edit_cap = 0;
            if (cudaMallocHost((void **)&c->h_frame, frame_bytes(cap)) != cudaSuccess)
                return fail(STA_ENOMEM, "pinned edit buffer");
            if (cudaMalloc((void **)&c->d_frame, frame_bytes(cap)) != cudaSuccess)
                return fail(STA_ENOMEM, "device edit buffer");
            c->device_bytes += (int64_t)frame_bytes(cap);
            c->edit_cap = cap;
        }
        h = c->h_frame;
        d = c->d_frame;
    }

    // one pass: validate each edit against the host mirror of the mask, stage it and apply it
    // to the mirror; on a bad edit, undo the mirror changes made so far and change nothing
    if (++c->stamp_gen > TS_STAMP) {  // stamps wrapped (every 127 calls): clear them
        for (auto &b : c->tstate) b &= TS_ACTIVE;
        c->stamp_gen = 1;
    }
    const uint8_t gen = c->stamp_gen;
    uint8_t *ts = c->tstate.data();
    int32_t *stage = frame_edited(h);
    int64_t k = 0, e = 0, dact = 0;  // dact: change of the active count
    const char *why = nullptr;
    for (; e < n_edits; ++e) {
        if (e + 16 < n_edits) {  // the per-tet state is accessed at random: fetch it ahead
            // (a prefetch never faults, so an unchecked id -- tet2 of a non-swap is -1 -- costs
            // at most a useless prefetch; the address is formed as an integer)
            const sta_edit &F = edits[e + 16];
            const uintptr_t base = (uintptr_t)ts;
            __builtin_prefetch((const void *)(base + (uintptr_t)(intptr_t)F.tet), 1);
            __builtin_prefetch((const void *)(base + (uintptr_t)(intptr_t)F.tet2), 1);
        }
        const sta_edit &E = edits[e];
        if (E.op < 0 || E.op > 2) { why = "bad op"; break; }
        if (E.tet < 0 || E.tet >= c->T) { why = "tet out of range"; break; }
        const uint8_t s1 = ts[E.tet];
        if ((s1 & TS_STAMP) == gen) { why = "tet named twice"; break; }
        if (E.op == STA_DEACTIVATE) {
            if (!(s1 & TS_ACTIVE)) { why = "deactivating an inactive tet"; break; }
            ts[E.tet] = gen;
            stage[k++] = E.tet;
            --dact;
        } else if (E.op == STA_ACTIVATE) {
            if (s1 & TS_ACTIVE) { why = "activating an active tet"; break; }
            ts[E.tet] = (uint8_t)(TS_ACTIVE | gen);
            stage[k++] = (int32_t)((uint32_t)E.tet | 0x80000000u);
            ++dact;
        } else {
            if (E.tet2 < 0 || E.tet2 >= c->T) { why = "tet2 out of range"; break; }
            const uint8_t s2 = ts[E.tet2];
            if (E.tet2 == E.tet || (s2 & TS_STAMP) == gen) { why = "tet2 named twice"; break; }
            if (!(s1 & TS_ACTIVE) || (s2 & TS_ACTIVE)) { why = "swap needs an active tet and an inactive tet2"; break; }
            ts[E.tet] = gen;
            ts[E.tet2] = (uint8_t)(TS_ACTIVE | gen);
            stage[k++] = E.tet;
            stage[k++] = (int32_t)((uint32_t)E.tet2 | 0x80000000u);
        }
    }
    if (why) {
        for (int64_t r = 0; r < e; ++r) {  // undo (each tet appears once, so this is exact)
            const sta_edit &E = edits[r];
            if (E.op == STA_DEACTIVATE) ts_set_active(c, E.tet, true);
            else if (E.op == STA_ACTIVATE) ts_set_active(c, E.tet, false);
            else { ts_set_active(c, E.tet, true); ts_set_active(c, E.tet2, false); }
        }
        return fail(STA_EINVAL, "edit " + std::to_string(e) + ": " + why);
    }
    c->n_active += dact;
    m = k;

    // header (count, zeroed counters) before the list: in graph mode the captured kernels read
    // the host-mapped block itself; otherwise block and list go to the device in one copy
    h->m = m;
    h->cnt[0] = h->cnt[1] = h->cnt[2] = 0ull;
    c->last_edited = m;
    // the fold kernel stores the frame's touched count into the host-mapped word (a frame
    // without edits launches no kernel outside graph mode)
    c->count_on_host = frame_counts_to_host(c) && (use_graph || m > 0);
    if (use_graph) {  // the captured sequence reads the host-mapped block itself: no copy call
        c->last_counters = c->d_gcnt + 4 * gb;
        std::atomic_thread_fence(std::memory_order_seq_cst);  // the block before the launch
        STA_CUDA_TRY(cudaGraphLaunch(c->g_streams[gb], s));
        STA_CUDA_TRY(cudaEventRecord(c->g_done[gb], s));
        c->g_pending[gb] = true;
        c->g_next = gb ^ 1;
        return STA_OK;
    }
    c->last_counters = frame_counters(d);
    STA_CUDA_TRY(cudaMemcpyAsync(d, h, frame_bytes(m), cudaMemcpyHostToDevice, s));
    STA_CUDA_TRY(cudaEventRecord(x->h2d_done, s));
    x->h2d_pending = true;
    if (m == 0) return STA_OK;  // the copy has zeroed the frame's counters
    return launch_stream_frame(c, d, m, s);
}

int sta_last_touched(sta_ctx *x, int64_t *touched_nnz, void *stream) {
    if (!x || !touched_nnz) return fail(STA_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (x->c.count_on_host) {  // the frame's fold kernel stored it in host-mapped memory
        STA_CUDA_TRY(cudaStreamSynchronize(s));
        *touched_nnz = (int64_t)*reinterpret_cast<volatile unsigned long long *>(x->c.h_count_mapped);
        return STA_OK;
    }
    // into a pinned word: a plain asynchronous copy (a pageable target is staged, and slower)
    STA_CUDA_TRY(cudaMemcpyAsync(x->h_count, x->c.last_counters + 3, sizeof *x->h_count,
                                 cudaMemcpyDeviceToHost, s));
    STA_CUDA_TRY(cudaStreamSynchronize(s));
    *touched_nnz = (int64_t)*x->h_count;
    return STA_OK;
}

int sta_csr(const sta_ctx *x, const int32_t **row_ptr, const int32_t **col, const double **val,
            int64_t *n_rows, int64_t *nnz) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (row_ptr) *row_ptr = x->c.row_ptr;
    if (col) *col = x->c.col;
    if (val) *val = x->c.val;
    if (n_rows) *n_rows = x->c.nrows;
    if (nnz) *nnz = x->c.nnz;
    return STA_OK;
}

int sta_scatter_map(const sta_ctx *x, const int32_t **scat) {
    if (!x || !scat) return fail(STA_EINVAL, "NULL argument");
    if (x->c.op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    *scat = x->c.scat;
    return STA_OK;
}

int sta_mask(const sta_ctx *x, const uint8_t **mask) {
    if (!x || !mask) return fail(STA_EINVAL, "NULL argument");
    *mask = x->c.mask;
    return STA_OK;
}

int sta_sizes(const sta_ctx *x, int64_t *n_nodes, int64_t *n_tets, int64_t *n_blocks,
              int64_t *device_bytes) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (n_nodes) *n_nodes = x->c.n;
    if (n_tets) *n_tets = x->c.T;
    if (n_blocks) *n_blocks = x->c.nblocks;
    if (device_bytes) *device_bytes = x->c.device_bytes;
    return STA_OK;
}

int sta_recompute_elements(sta_ctx *x, int active_only, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (x->c.op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    STA_TRY(launch_elements(&x->c, active_only != 0, (cudaStream_t)stream));
    if (x->c.policy == STA_POLICY_FIXED) STA_TRY(launch_fx_prepare(&x->c, (cudaStream_t)stream));
    return STA_OK;
}

int sta_set_policy(sta_ctx *x, int32_t policy, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (policy != STA_POLICY_REFOLD && policy != STA_POLICY_FIXED)
        return fail(STA_EINVAL, "policy must be STA_POLICY_REFOLD or STA_POLICY_FIXED");
    Ctx *c = &x->c;
    if (c->graph_on) return fail(STA_ESTATE, "disable graph mode before changing the policy");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->op == STA_OP_PROXY) {  // integer state either way: nothing to prepare
        c->policy = policy;
        return launch_values(c, s);
    }
    if (policy == STA_POLICY_FIXED) STA_TRY(launch_fx_prepare(c, s));
    c->policy = policy;
    return launch_rebuild(c, s);  // every value under the new policy, from the current mask
}

int sta_set_params(sta_ctx *x, const double *nodes, const double *young, const double *poisson,
                   int on_device, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (x->c.op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    Ctx *c = &x->c;
    cudaStream_t s = (cudaStream_t)stream;
    if (nodes) {
        if (on_device) {
            STA_CUDA_TRY(cudaMemcpy2DAsync(c->X, sizeof(double4_32a), nodes, 3 * sizeof(double),
                                           3 * sizeof(double), (size_t)c->n,
                                           cudaMemcpyDeviceToDevice, s));
        } else {
            std::vector<double> X4(4 * (size_t)(c->n > 0 ? c->n : 1), 0.0);
            for (int64_t v = 0; v < c->n; ++v)
                for (int k = 0; k < 3; ++k) X4[4 * v + k] = nodes[3 * v + k];
            STA_CUDA_TRY(cudaMemcpyAsync(c->X, X4.data(), sizeof(double4_32a) * c->n,
                                         cudaMemcpyHostToDevice, s));
            STA_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (young)
        STA_CUDA_TRY(cudaMemcpy2DAsync(c->mat, sizeof(double2), young, sizeof(double),
                                       sizeof(double), (size_t)c->T, kind, s));
    if (poisson)
        STA_CUDA_TRY(cudaMemcpy2DAsync((double *)c->mat + 1, sizeof(double2), poisson,
                                       sizeof(double), sizeof(double), (size_t)c->T, kind, s));
    unsigned long long init[2] = {0ull, 0ull};
    STA_CUDA_TRY(cudaMemcpyAsync(c->counters, init, sizeof init, cudaMemcpyHostToDevice, s));
    unsigned long long mx = ~0ull;
    STA_CUDA_TRY(cudaMemcpyAsync(c->counters + 2, &mx, sizeof mx, cudaMemcpyHostToDevice, s));
    STA_TRY(launch_elements(c, false, s));
    unsigned long long back[4];
    STA_CUDA_TRY(cudaMemcpyAsync(back, c->counters, sizeof back, cudaMemcpyDeviceToHost, s));
    STA_CUDA_TRY(cudaStreamSynchronize(s));
    if (back[0] != 0)
        return fail(STA_EINVAL, std::to_string(back[0]) + " tetrahedra have det <= 0 (first: tet " +
                                    std::to_string(back[2]) + ")");
    if (c->policy == STA_POLICY_FIXED) STA_TRY(launch_fx_prepare(c, s));
    if (nodes) {  // the tetrahedra's volumes, hence the lumped mass, follow the positions
        STA_TRY(launch_dyn_qmass(c, s));
        STA_TRY(launch_dyn_mass_all(c, s));
    }
    return STA_OK;
}

int sta_adjoint(sta_ctx *x, const double *grad_val, double *dE, double *dnu, double *dX,
                void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    const Ctx *c = &x->c;
    if (x->c.op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    if ((c->nnz > 0 && !grad_val) || (c->T > 0 && (!dE || !dnu)) || (c->n > 0 && !dX))
        return fail(STA_EINVAL, "NULL argument");
    return launch_adjoint(&x->c, grad_val, dE, dnu, dX, (cudaStream_t)stream);
}

int sta_spmv(sta_ctx *x, const double *val, const double *xv, double *y, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (x->c.nrows > 0 && (!xv || !y)) return fail(STA_EINVAL, "NULL argument");
    return launch_spmv(&x->c, val ? val : x->c.val, xv, y, (cudaStream_t)stream);
}

int sta_element_matrices(sta_ctx *x, const int32_t *tet_ids, int64_t n, double *out, void *stream) {
    if (!x || n < 0 || (n > 0 && (!tet_ids || !out))) return fail(STA_EINVAL, "bad argument");
    if (x->c.op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    return launch_expand_elements(&x->c, tet_ids, n, out, (cudaStream_t)stream);
}

}  // extern "C"
