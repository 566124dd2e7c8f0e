// Streaming update (Sec. 3.2, Algorithm 1; the local_recompute policy of Sec. 3.5 made
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
// matrix entry, and one FP64 instruction per step advances a whole warp of folds.  The claim
// kernel lists the two kinds of unit apart (diagonal units from the front of the list, pair
// units from the back), so that a warp folds units of one kind: 5 diagonal units (lanes
// 6g .. 6g+5 fold the 6 entries i <= j of unit g) or 3 pair units (lanes 9g .. 9g+8 fold the
// 9 entries (i, j)).  A warp's step count is its longest fold, and on GB300 an FP64 warp
// instruction holds the SM's FP64 pipe for about 16 cycles: mixing a ~24-contribution diagonal
// unit with ~6-contribution pair units would leave most of those steps idle.
// The unit's active codes are compacted (in list order) into shared memory first, three codes
// per lane and step.  Then the element-cache runs of the active contributors (48 B for a
// diagonal unit, 80 B for a pair; 16-byte aligned) are copied into shared memory with 16-byte
// cp.async copies, all in flight at once, so a unit costs one round trip for its operands
// however long its list; the fold reads them from there.  A unit with more than ENT_SCAP
// active contributions loads its operands from global memory instead (4 steps in flight).
// Operands, order and operations are those of k_fold_flat, so the values are the same bits.
// ------------------------------------------------------------------------------------------
constexpr int ENT_DG = 5;      // diagonal units per warp round (6 lanes each: 30 lanes)
constexpr int ENT_PG = 3;      // pair units per warp round (9 lanes each: 27 lanes)
constexpr int ENT_DCAP = 64;   // listed active contributions of a diagonal unit (larger: direct)
constexpr int ENT_PCAP = 96;   // the same for a pair unit
constexpr int ENT_SCAP = 24;   // active contributions whose runs are staged in shared memory
constexpr int ENT_WARPS = 4;
constexpr int ENT_SOP = ENT_DG * ENT_DCAP > ENT_PG * ENT_PCAP ? ENT_DG * ENT_DCAP : ENT_PG * ENT_PCAP;
constexpr int ENT_STAGE = ENT_DG * ENT_SCAP * 6;  // doubles per warp: = ENT_PG * ENT_SCAP * 10
static_assert(ENT_DG * ENT_SCAP * 6 == ENT_PG * ENT_SCAP * 10, "stage shared by both kinds");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// One warp round over units first .. first+NG-1 of one kind (k-th diagonal unit at list[k],
// k-th pair unit at list[cap - 1 - k]); `sop`, `stage` are the warp's shared buffers.
template <bool DIAG>
__device__ __forceinline__ void fold_units(const FoldArgs &A, const int32_t *__restrict__ list,
                                           int64_t first, int64_t n_units, int64_t cap,
                                           int32_t *__restrict__ owner, uint32_t *sop_w,
                                           double *stage_w, int lane, bool has_eps) {
    constexpr int GW = DIAG ? 6 : 9;                 // lanes (entries) per unit
    constexpr int NG = DIAG ? ENT_DG : ENT_PG;       // units per warp round
    constexpr int CAP = DIAG ? ENT_DCAP : ENT_PCAP;  // listed active contributions
    constexpr int RUN = DIAG ? 6 : 10;               // staged doubles per run (48 B, 80 B)
    constexpr int CPR = DIAG ? 3 : 5;                // 16-byte copies per run
    const unsigned FULL = 0xffffffffu;
    const int g = lane / GW, q = lane % GW;          // g == NG: idle lanes
    const int64_t k = first + g;
    const bool valid = g < NG && k < n_units;
    uint32_t *sop = sop_w + (g < NG ? g : 0) * CAP;
    double *stage = stage_w + (g < NG ? g : 0) * (ENT_SCAP * RUN);  // run j at stage[RUN j]
    int4 bm = make_int4(0, 0, 0, 0);
    int2 mir = make_int2(0, 0);
    if (valid) {
        const int32_t u = __ldg(list + (DIAG ? k : cap - 1 - k));
        bm = __ldg(A.bmeta + u);
        if (!DIAG) mir = __ldg(A.bmirror + u);
        if (q == 0) owner[u] = INT32_MAX;  // release the claim (all claims are done)
    }
    // compact the unit's active contributors (as operand bases), its GW lanes striding over its
    // list, three GW-code chunks loaded together and taken in list order
    int nact = 0;
    const int span = valid ? bm.w - bm.z : 0;
    const int max_span = __reduce_max_sync(FULL, span);
    const unsigned below_q = (1u << q) - 1u;
    for (int c0 = 0; c0 < max_span; c0 += 3 * GW) {
        int32_t kc[3];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const int c = c0 + GW * h + q;
            kc[h] = (valid && c < span) ? __ldg(A.ccode + bm.z + c) : 0;
        }
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const unsigned m = __ballot_sync(FULL, kc[h] < 0);
            const unsigned gm = (m >> (GW * g)) & ((1u << GW) - 1u);
            const int pos = nact + __popc(gm & below_q);
            if (kc[h] < 0 && pos < CAP) sop[pos] = word_offset((uint32_t)kc[h]);
            nact += __popc(gm);
        }
    }
    __syncwarp();
    const bool big = valid && nact > CAP;
    if (big && q == 0) fold_direct(A, bm, mir);  // rare: more active contributions than listed
    const bool mine = valid && !big;
    // stage the runs of the unit's active contributors, the unit's GW lanes sharing the copies
    const bool staged = mine && nact <= ENT_SCAP;
    if (staged) {
        for (int kk = q; kk < nact * CPR; kk += GW) {
            const int j = kk / CPR, p = kk - j * CPR;
            cp_async16(stage + RUN * j + 2 * p, A.Ke + sop[j] + 2 * p);
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    double acc = 0.0;
    const int ns = staged ? nact : 0;
    const int maxs = __reduce_max_sync(FULL, ns);
    if (maxs > 0) {  // warp-uniform; the same operands in the same order as below
        if (ns > 0) acc = plus_zero(stage[q]);  // the first contribution: +0.0 + v
        for (int j = 1; j < maxs; ++j)
            if (j < ns) acc += stage[RUN * j + q];
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
        if (DIAG) {
            // 6-run entry q = (i, j), i <= j
            const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
            double a = acc;
            if (i == j && has_eps) a += A.eps;
            double *out = A.val + bm.x;
            const int rs = bm.y >> 1;
            out[i * rs + j] = a;
            if (i != j) out[j * rs + i] = a;
        } else {
            const int qi = q / 3, qj = q % 3;
            A.val[bm.x + qi * (bm.y >> 1) + qj] = acc;
            A.val[mir.x + qj * mir.y + qi] = acc;
        }
    }
    __syncwarp();
}

// count[0]: diagonal units | pair units << 32 (the claim kernel's); count[2] gets the frame's
// touched CSR entries (9 per diagonal unit, 18 = both blocks per pair unit), also stored into
// the host-mapped word `host_count` when given.  `cap`: the list's length.  `next_count`, when
// given, is the count pair of the next frame (graph mode alternates two), zeroed here so that
// the captured frame needs no memset node of its own.
__global__ void __launch_bounds__(ENT_WARPS * 32)
k_fold_entries(FoldArgs A, const int32_t *__restrict__ list, unsigned long long *count, int64_t cap,
               int32_t *__restrict__ owner, unsigned long long *host_count,
               unsigned long long *next_count) {
    __shared__ uint32_t sop_all[ENT_WARPS][ENT_SOP];
    __shared__ __align__(16) double stage_all[ENT_WARPS][ENT_STAGE];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long packed = *count;  // final: the claim kernel has ended
    const int64_t nd = (int64_t)(packed & 0xffffffffull), np = (int64_t)(packed >> 32);
    const int64_t gd = (nd + ENT_DG - 1) / ENT_DG, gp = (np + ENT_PG - 1) / ENT_PG;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long entries = 9ull * (unsigned long long)nd + 18ull * (unsigned long long)np;
        count[2] = entries;
        if (host_count) *host_count = entries;
        if (next_count) {
            next_count[0] = 0;
            next_count[2] = 0;
        }
    }
    const bool has_eps = A.eps != 0.0;
    for (int64_t item = warp; item < gd + gp; item += nwarps) {  // warp-uniform
        if (item < gd)
            fold_units<true>(A, list, item * ENT_DG, nd, cap, owner, sop_all[wid], stage_all[wid],
                             lane, has_eps);
        else
            fold_units<false>(A, list, (item - gd) * ENT_PG, np, cap, owner, sop_all[wid],
                              stage_all[wid], lane, has_eps);
    }
}

// Streaming, phase 1: apply the frame's mask changes and collect the touched fold units.  One
// thread per (edited tet k, unit slot s): it writes the contributor's new activity bit, and
// claims the slot's unit with a compare-and-swap on its owner word (INT32_MAX = free); the
// thread that wins appends the unit to the fold list, a diagonal unit (slots 0-3) at the front
// and a pair unit at the back of the `cap` entries, both counted by one CTA-aggregated atomic
// on counters[1] = diagonal units | pair units << 32 (a large frame's warps all appending to
// that one word serialise at the L2; per CTA there are 8 times fewer).  The fold releases the claims and counts
// the touched entries.  The list order depends on scheduling, the values do not (each unit
// folds independently).  edited[k] = tet id | (new state << 31); the edited count is *m_dev if
// m_dev, else m; counters[1] starts at zero; a frame lists at most 10 units per edited tet and
// at most every unit once, so the two ends never meet when cap >= min(10 m, units).
constexpr int CLAIM_THREADS = 256;

__global__ void __launch_bounds__(CLAIM_THREADS)
k_stream_claim(const int32_t *__restrict__ edited, int64_t m,
                               const int64_t *__restrict__ m_dev, int64_t T,
                               const int32_t *__restrict__ tunit,
                               const int32_t *__restrict__ cslot, int32_t *__restrict__ ccode,
                               uint8_t *__restrict__ mask, int32_t *__restrict__ owner,
                               int32_t *__restrict__ list, int64_t cap,
                               unsigned long long *counters) {
    // per warp of the CTA: its packed winner counts, then its offset; the CTA's base
    __shared__ unsigned long long s_cnt[CLAIM_THREADS / 32];
    __shared__ unsigned long long s_base;
    const int64_t n = 10 * (m_dev ? *m_dev : m);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // CTA-uniform
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
        const unsigned dball = __ballot_sync(0xffffffffu, won && diag);
        const unsigned pball = __ballot_sync(0xffffffffu, won && !diag);
        // packed counts add without carries: each half stays below 2^32
        if (lane == 0)
            s_cnt[wid] = (unsigned long long)__popc(dball) | ((unsigned long long)__popc(pball) << 32);
        __syncthreads();
        if (threadIdx.x == 0) {  // exclusive prefix over the CTA's warps, one atomic for all
            unsigned long long tot = 0;
            for (int w = 0; w < CLAIM_THREADS / 32; ++w) {
                const unsigned long long v = s_cnt[w];
                s_cnt[w] = tot;
                tot += v;
            }
            s_base = tot ? atomicAdd(&counters[1], tot) : 0ull;
        }
        __syncthreads();
        const unsigned long long base = s_base + s_cnt[wid];
        __syncthreads();  // s_cnt and s_base are rewritten in the next round
        const unsigned below = (1u << lane) - 1u;
        if (won && diag) list[(base & 0xffffffffull) + __popc(dball & below)] = u;
        if (won && !diag) list[cap - 1 - (int64_t)((base >> 32) + __popc(pball & below))] = u;
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

int launch_fold_list(Ctx *c, const int32_t *list, int64_t cap, unsigned long long *count,
                     int64_t max_items, cudaStream_t s, unsigned long long *host_count,
                     unsigned long long *next_count) {
    const int threads = ENT_WARPS * 32;
    // a warp round per 3 units for the largest possible list (all pair units), at most the
    // resident CTAs
    const int grid = persistent_grid(c, (const void *)k_fold_entries, threads,
                                     (max_items + ENT_PG - 1) / ENT_PG * 32);
    k_fold_entries<<<grid, threads, 0, s>>>(fold_args(c), list, count, cap, c->owner, host_count,
                                            next_count);
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
// replayed for any frame up to `cap`).  `next_cnt`: the counters of the next frame, which the
// frame's last kernel zeroes (graph mode), or nullptr.
int launch_stream_frame(Ctx *c, const int32_t *edited, const int64_t *m_dev,
                        unsigned long long *cnt, int64_t cap, cudaStream_t s,
                        unsigned long long *next_cnt) {
    if (c->op == STA_OP_PROXY)
        return launch_proxy_frame(c, edited, 0, m_dev, cap, c->plist, cnt, s, next_cnt);
    if (c->policy == STA_POLICY_FIXED) {
        STA_TRY(launch_fx_frame(c, edited, 0, m_dev, cap, c->touched, cnt, s, next_cnt));
        return launch_dyn_mass_edited(c, edited, 0, m_dev, cap, s);
    }
    const int threads = CLAIM_THREADS;
    int64_t g = (10 * cap + threads - 1) / threads;
    const int64_t gmax = (int64_t)c->num_sms * 16;
    g = g < 1 ? 1 : (g > gmax ? gmax : g);
    k_stream_claim<<<(unsigned)g, threads, 0, s>>>(edited, 0, m_dev, c->T, c->tunit, c->cslot,
                                                   c->ccode, c->mask, c->owner, c->touched,
                                                   c->nunits, cnt);
    STA_CUDA_TRY(cudaGetLastError());
    STA_TRY(launch_fold_list(c, c->touched, c->nunits, cnt + 1, 10 * (cap > 0 ? cap : 1), s,
                             c->d_count_mapped, next_cnt ? next_cnt + 1 : nullptr));
    return launch_dyn_mass_edited(c, edited, 0, m_dev, cap, s);
}

bool frame_counts_to_host(const Ctx *c) {
    return c->op == STA_OP_ELASTICITY && c->policy == STA_POLICY_REFOLD && c->d_count_mapped;
}

int launch_stream_frame(Ctx *c, FrameHeader *frame, int64_t cap, cudaStream_t s) {
    return launch_stream_frame(c, frame_edited(frame), &frame->m, frame_counters(frame), cap, s,
                               nullptr);
}

// Streaming update with caller-chosen scratch (the allocation-free entry point): the same two
// kernels, with the edited-tet list, the touched-unit list and the counters at the given
// addresses; the touched counts are copied to the context's counters afterwards so that
// sta_last_touched reports them.
int launch_stream_scratch(Ctx *c, int64_t m, const int32_t *d_edited, int32_t *touched,
                          unsigned long long *counters, cudaStream_t s) {
    STA_CUDA_TRY(cudaMemsetAsync(counters + 1, 0, 3 * sizeof(unsigned long long), s));
    if (m > 0 && c->op == STA_OP_PROXY) {
        STA_TRY(launch_proxy_frame(c, d_edited, m, nullptr, m, touched, counters, s, nullptr));
    } else if (m > 0 && c->policy == STA_POLICY_FIXED) {
        STA_TRY(launch_fx_frame(c, d_edited, m, nullptr, m, touched, counters, s, nullptr));
    } else if (m > 0) {
        const int threads = CLAIM_THREADS;
        const int64_t g = (10 * m + threads - 1) / threads;
        // the touched list holds 10 m units (at most 10 per edited tet)
        k_stream_claim<<<(unsigned)g, threads, 0, s>>>(d_edited, m, nullptr, c->T, c->tunit, c->cslot,
                                                       c->ccode, c->mask, c->owner, touched,
                                                       10 * m, counters);
        STA_CUDA_TRY(cudaGetLastError());
        STA_TRY(launch_fold_list(c, touched, 10 * m, counters + 1, 10 * m, s, nullptr, nullptr));
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
