// Streaming update (a3 of Algorithm 1, Sec. 3.2; the local_recompute policy of Sec. 3.5 made
// bitwise): apply a frame's mask changes, collect the fold units its edits touch, and re-fold
// exactly those with the rebuild's operands, order and operations.  Also the mask-to-activity
// pass of a full rebuild with a new mask.  Fold definition and shared device code:
// sta_fold.cuh.
#include "sta_fold.cuh"

namespace sta {
namespace {

// ------------------------------------------------------------------------------------------
// Entry-parallel fold of a list of units (streaming).  A frame's touched list is short and its
// longest folds (diagonal units, ~24 contributions) set the latency, so here each lane folds ONE
// matrix entry: a warp takes 3 listed units, lanes 9g .. 9g+8 fold the 9 entries (i, j) of
// unit g (6 of them for a diagonal unit), and one FP64 instruction per step advances all 27
// folds.  The unit's active codes are compacted (in list order) into shared memory first, 27
// codes per step (three loads in flight per lane).  Then the element-cache runs of the active
// contributors (48 B for a diagonal unit, 80 B for a pair; 16-byte aligned) are copied into
// shared memory with 16-byte cp.async copies, all in flight at once, so a unit costs one round
// trip for its operands however long its list; the fold reads them from there.  A unit with
// more than ENT_SCAP active contributions loads its operands from global memory instead (4
// steps in flight).  Operands, order and operations are those of k_fold_flat, so the values are
// the same bits.
// ------------------------------------------------------------------------------------------
constexpr int ENT_UNITS = 3;    // units per warp round (27 lanes)
constexpr int ENT_CAP = 96;     // active contributions listed per unit; larger units fold directly
constexpr int ENT_SCAP = 24;    // active contributions whose runs are staged in shared memory
constexpr int ENT_WARPS = 4;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(ENT_WARPS * 32)
k_fold_entries(FoldArgs A, const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
               int32_t *__restrict__ owner, unsigned long long *host_count) {
    __shared__ uint32_t sop_all[ENT_WARPS][ENT_UNITS][ENT_CAP];
    __shared__ __align__(16) double stage_all[ENT_WARPS][ENT_UNITS][ENT_SCAP * 10];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / 9, q = lane % 9;  // g == 3: lanes 27..31 idle
    const int qi = q / 3, qj = q % 3;
    uint32_t *sop = sop_all[wid][g < ENT_UNITS ? g : 0];
    double *stage = stage_all[wid][g < ENT_UNITS ? g : 0];  // run j at stage[10 j]
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = (int64_t)*count;
    const bool has_eps = A.eps != 0.0;
    // the frame's touched-entry count (count[2], final since the claim kernel ended) into the
    // host-mapped word sta_last_touched reads
    if (host_count && blockIdx.x == 0 && threadIdx.x == 0) *host_count = count[2];
    for (int64_t base = warp * ENT_UNITS; base < nitems; base += nwarps * ENT_UNITS) {  // warp-uniform
        const int64_t item = base + g;
        const bool valid = g < ENT_UNITS && item < nitems;
        int4 bm = make_int4(0, 0, 0, 0);
        int2 mir = make_int2(0, 0);
        if (valid) {
            const int32_t u = __ldg(list + item);
            bm = __ldg(A.bmeta + u);
            mir = __ldg(A.bmirror + u);
            if (q == 0) owner[u] = INT32_MAX;  // release the claim (all claims are done)
        }
        // compact the unit's active contributors (as operand bases), 9 lanes striding over its
        // list, three 9-code chunks loaded together and taken in list order
        int nact = 0;
        const int span = valid ? bm.w - bm.z : 0;
        const int max_span = __reduce_max_sync(FULL, span);
        const unsigned below_q = (1u << q) - 1u;
        for (int c0 = 0; c0 < max_span; c0 += 27) {
            int32_t k[3];
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const int c = c0 + 9 * h + q;
                k[h] = (valid && c < span) ? __ldg(A.ccode + bm.z + c) : 0;
            }
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const unsigned m = __ballot_sync(FULL, k[h] < 0);
                const unsigned gm = (m >> (9 * g)) & 0x1ffu;
                const int pos = nact + __popc(gm & below_q);
                if (k[h] < 0 && pos < ENT_CAP) sop[pos] = word_offset((uint32_t)k[h]);
                nact += __popc(gm);
            }
        }
        __syncwarp();
        const bool big = valid && nact > ENT_CAP;
        if (big && q == 0) fold_direct(A, bm, mir);  // rare: more active contributions than listed
        const bool diag = (bm.y & 1) != 0;
        const bool mine = valid && !big && (!diag || q < 6);  // a diagonal unit folds 6 entries
        // stage the runs of the unit's active contributors (16-byte pieces: 3 of a 48-byte
        // diagonal run, 5 of an 80-byte pair run), the unit's 9 lanes sharing the copies
        const bool staged = valid && !big && nact <= ENT_SCAP;
        if (staged) {
            const int cpr = diag ? 3 : 5;
            for (int kk = q; kk < nact * cpr; kk += 9) {
                const int j = kk / cpr, p = kk - j * cpr;
                cp_async16(stage + 10 * j + 2 * p, A.Ke + sop[j] + 2 * p);
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        double acc = 0.0;
        const int ns = mine && staged ? nact : 0;
        const int maxs = __reduce_max_sync(FULL, ns);
        if (maxs > 0) {  // warp-uniform; the same operands in the same order as below
            if (ns > 0) acc = plus_zero(stage[q]);  // the first contribution: +0.0 + v
            for (int j = 1; j < maxs; ++j)
                if (j < ns) acc += stage[10 * j + q];
        }
        const int n = mine && !staged ? nact : 0;  // longer lists: operands from global memory
        const int maxn = __reduce_max_sync(FULL, n);
#define STA_LD(j) ((j) < n ? __ldg(A.Ke + sop[(j)] + q) : 0.0)
        if (maxn > 0) {  // warp-uniform guards, as in k_fold_flat
            if (n > 0) acc = plus_zero(STA_LD(0));  // the first contribution: +0.0 + v
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            if (maxn > 1) v0 = STA_LD(1);
            if (maxn > 2) v1 = STA_LD(2);
            if (maxn > 3) v2 = STA_LD(3);
            if (maxn > 4) v3 = STA_LD(4);
            int j = 1;
            for (; j + 4 <= maxn; j += 4) {  // next 4 operands in flight
                double x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
                if (j + 4 < maxn) x0 = STA_LD(j + 4);
                if (j + 5 < maxn) x1 = STA_LD(j + 5);
                if (j + 6 < maxn) x2 = STA_LD(j + 6);
                if (j + 7 < maxn) x3 = STA_LD(j + 7);
                if (j < n) acc += v0;
                if (j + 1 < n) acc += v1;
                if (j + 2 < n) acc += v2;
                if (j + 3 < n) acc += v3;
                v0 = x0;
                v1 = x1;
                v2 = x2;
                v3 = x3;
            }
            if (j < maxn && j < n) acc += v0;
            if (j + 1 < maxn && j + 1 < n) acc += v1;
            if (j + 2 < maxn && j + 2 < n) acc += v2;
        }
#undef STA_LD
        if (mine) {
            if (diag) {
                // 6-run entry q = (i, j), i <= j
                const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
                double a = acc;
                if (i == j && has_eps) a += A.eps;
                double *out = A.val + bm.x;
                const int rs = bm.y >> 1;
                out[i * rs + j] = a;
                if (i != j) out[j * rs + i] = a;
            } else {
                A.val[bm.x + qi * (bm.y >> 1) + qj] = acc;
                A.val[mir.x + qj * mir.y + qi] = acc;
            }
        }
        __syncwarp();
    }
}

// Streaming, phase 1: apply the frame's mask changes and collect the touched fold units.  One
// thread per (edited tet k, unit slot s): it writes the contributor's new activity bit, and
// claims the slot's unit with a compare-and-swap on its owner word (INT32_MAX = free); the
// thread that wins appends the unit to the fold list (warp-aggregated) and counts its entries
// (9 for a diagonal unit, 18 = both blocks for a pair).  The fold releases the claims.  The
// list order depends on scheduling, the values do not (each unit folds independently).
// edited[k] = tet id | (new state << 31); the edited count is *m_dev if m_dev, else m;
// counters[1] (units) and counters[3] (entries) start at zero.
__global__ void k_stream_claim(const int32_t *__restrict__ edited, int64_t m,
                               const int64_t *__restrict__ m_dev, int64_t T,
                               const int32_t *__restrict__ tunit,
                               const int32_t *__restrict__ cslot, int32_t *__restrict__ ccode,
                               uint8_t *__restrict__ mask, int32_t *__restrict__ owner,
                               int32_t *__restrict__ list, unsigned long long *counters) {
    const int64_t n = 10 * (m_dev ? *m_dev : m);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // warp-uniform
        const int64_t i = i0 + threadIdx.x;
        bool won = false, diag = false;
        int32_t u = 0;
        if (i < n) {
            const uint32_t w = (uint32_t)edited[i / 10];
            const int32_t t = (int32_t)(w & 0x7fffffffu);
            const uint32_t on = w >> 31;
            const int s = (int)(i % 10);
            if (s == 0) mask[t] = (uint8_t)on;
            const int32_t slot = cslot[10 * (int64_t)t + s];
            u = tunit[10 * (int64_t)t + s];
            // the word is (t, s)'s run offset | activity: written without reading it back
            ccode[slot] = (int32_t)((uint32_t)ke_slot_at(T, t, s) | (on << 31));
            diag = s < 4;
            won = atomicCAS(&owner[u], INT32_MAX, 0) == INT32_MAX;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, won);
        const unsigned dball = __ballot_sync(0xffffffffu, won && diag);
        unsigned long long base = 0;
        if (lane == 0 && ball) {
            base = atomicAdd(&counters[1], (unsigned long long)__popc(ball));
            atomicAdd(&counters[3], (unsigned long long)(18 * __popc(ball) - 9 * __popc(dball)));
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (won) list[base + __popc(ball & ((1u << lane) - 1u))] = u;
    }
}

// Activity bits of all contributor codes from the mask (full rebuild with a new mask).
__global__ void k_mask_bits(int32_t *__restrict__ ccode, int64_t n, int64_t T,
                            const uint8_t *__restrict__ mask) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t code = (uint32_t)ccode[k];
        const uint32_t on = mask[word_tet(code, T)] ? CODE_ACTIVE : 0u;
        ccode[k] = (int32_t)((code & ~CODE_ACTIVE) | on);
    }
}

}  // namespace

int persistent_grid(const Ctx *c, const void *kernel, int threads, int64_t items, bool tuned) {
    int per_sm = tuned ? c->blocks_per_sm : 0;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int64_t need = (items + threads - 1) / threads;
    int64_t cap = (int64_t)per_sm * c->num_sms;
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

int launch_fold_list(Ctx *c, const int32_t *list, const unsigned long long *count,
                     int64_t max_items, cudaStream_t s, unsigned long long *host_count) {
    const int threads = ENT_WARPS * 32;
    // one unit per 9 lanes (3 per warp) for the largest possible list, at most the resident CTAs
    const int grid = persistent_grid(c, (const void *)k_fold_entries, threads,
                                     (max_items + ENT_UNITS - 1) / ENT_UNITS * 32);
    k_fold_entries<<<grid, threads, 0, s>>>(fold_args(c), list, count, c->owner, host_count);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_mask_bits(Ctx *c, cudaStream_t s) {
    if (c->T == 0 || c->op == STA_OP_PROXY) return STA_OK;  // the proxy reads the mask itself
    const int64_t n = 10 * c->T;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = (int64_t)c->num_sms * 8;
    if (grid > cap) grid = cap;
    k_mask_bits<<<(unsigned)grid, 256, 0, s>>>(c->ccode, n, c->T, c->mask);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

// Every value from the current mask: the operator's full rebuild.
int launch_values(Ctx *c, cudaStream_t s) {
    if (c->op == STA_OP_PROXY) return launch_proxy_rebuild(c, s);
    STA_TRY(launch_rebuild(c, s));
    return launch_dyn_mass_all(c, s);  // the lumped mass, when the dynamics are set up
}

// One streaming frame: claim kernel, then the fold of the touched units.  `frame` is a device
// frame block (FrameHeader + edited list) already holding the frame; the count is read from
// it, grids are sized for `cap` edited tetrahedra (so the sequence can be captured once and
// replayed for any frame up to `cap`).
int launch_stream_frame(Ctx *c, const int32_t *edited, const int64_t *m_dev,
                        unsigned long long *cnt, int64_t cap, cudaStream_t s) {
    if (c->op == STA_OP_PROXY)
        return launch_proxy_frame(c, edited, 0, m_dev, cap, c->plist, cnt, s);
    if (c->policy == STA_POLICY_FIXED) {
        STA_TRY(launch_fx_frame(c, edited, 0, m_dev, cap, c->touched, cnt, s));
        return launch_dyn_mass_edited(c, edited, 0, m_dev, cap, s);
    }
    const int threads = 256;
    int64_t g = (10 * cap + threads - 1) / threads;
    const int64_t gmax = (int64_t)c->num_sms * 16;
    g = g < 1 ? 1 : (g > gmax ? gmax : g);
    k_stream_claim<<<(unsigned)g, threads, 0, s>>>(edited, 0, m_dev, c->T, c->tunit, c->cslot,
                                                   c->ccode, c->mask, c->owner, c->touched, cnt);
    STA_CUDA_TRY(cudaGetLastError());
    STA_TRY(launch_fold_list(c, c->touched, cnt + 1, 10 * (cap > 0 ? cap : 1), s, c->d_count_mapped));
    return launch_dyn_mass_edited(c, edited, 0, m_dev, cap, s);
}

bool frame_counts_to_host(const Ctx *c) {
    return c->op == STA_OP_ELASTICITY && c->policy == STA_POLICY_REFOLD && c->d_count_mapped;
}

int launch_stream_frame(Ctx *c, FrameHeader *frame, int64_t cap, cudaStream_t s) {
    return launch_stream_frame(c, frame_edited(frame), &frame->m, frame_counters(frame), cap, s);
}

// Streaming update with caller-chosen scratch (the allocation-free entry point): the same two
// kernels, with the edited-tet list, the touched-unit list and the counters at the given
// addresses; the touched counts are copied to the context's counters afterwards so that
// sta_last_touched reports them.
int launch_stream_scratch(Ctx *c, int64_t m, const int32_t *d_edited, int32_t *touched,
                          unsigned long long *counters, cudaStream_t s) {
    STA_CUDA_TRY(cudaMemsetAsync(counters + 1, 0, 3 * sizeof(unsigned long long), s));
    if (m > 0 && c->op == STA_OP_PROXY) {
        STA_TRY(launch_proxy_frame(c, d_edited, m, nullptr, m, touched, counters, s));
    } else if (m > 0 && c->policy == STA_POLICY_FIXED) {
        STA_TRY(launch_fx_frame(c, d_edited, m, nullptr, m, touched, counters, s));
    } else if (m > 0) {
        const int threads = 256;
        const int64_t g = (10 * m + threads - 1) / threads;
        k_stream_claim<<<(unsigned)g, threads, 0, s>>>(d_edited, m, nullptr, c->T, c->tunit, c->cslot,
                                                       c->ccode, c->mask, c->owner, touched,
                                                       counters);
        STA_CUDA_TRY(cudaGetLastError());
        STA_TRY(launch_fold_list(c, touched, counters + 1, 10 * m, s, nullptr));
    }
    if (m > 0) STA_TRY(launch_dyn_mass_edited(c, d_edited, m, nullptr, m, s));
    // touched units and touched entries, for sta_last_touched
    STA_CUDA_TRY(cudaMemcpyAsync(c->counters + 1, counters + 1, 3 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s));
    c->last_counters = c->counters;
    c->count_on_host = false;  // read back from the device counters
    return STA_OK;
}

}  // namespace sta
