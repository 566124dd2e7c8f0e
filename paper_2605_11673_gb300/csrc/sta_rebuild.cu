// Full rebuild (a2 of Algorithm 1; the full_rebuild policy of Sec. 3.5): every value of the
// superset pattern folded from the element cache over the active mask, one lane per fold
// entry (k_fold_flat), in FP64 or, under STA_POLICY_FIXED, as the fixed-point integer sum.
// Fold definition and shared device code: sta_fold.cuh.
#include <type_traits>

#include "sta_fold.cuh"

namespace sta {
namespace {

// ------------------------------------------------------------------------------------------
// Flat entry-parallel rebuild.  Every fold entry of the pattern gets a lane: 6 per diagonal
// unit, 9 per off-diagonal unit.  A warp tile is 32 consecutive entries of units of one kind
// (tile records built at create: first unit, entry offset, kind, entry count, and the code
// range of its units (up to 7), which is contiguous).  The warp compacts the active codes of that range into
// shared memory with ballots (list order kept, so each unit's active codes form one segment),
// each lane locates its unit's segment from the same ballots, and every FP64 add instruction
// then advances up to 32 folds.  Units are ordered so that a tile's lists have equal length.
//
// Each tile needs two dependent loads before its first add (tile record -> unit records and
// codes), so the persistent warps run them as a software pipeline: while tile w folds, the
// first three code chunks of tile w+W (96 codes: most tiles' whole range), the unit records of
// tile w+2W and the tile record of tile w+3W are in flight (W = warps in the grid).  Operands, order and operations are those of
// fold_direct and k_fold_entries.
// ------------------------------------------------------------------------------------------
constexpr int FLAT_CAP = 448;  // staged active codes per tile; a larger tile folds from the list


struct FlatLane {
    int32_t u;  // unit
    int q;      // entry of the unit
    bool dgl, valid;
    int nv;     // entries in the tile (lanes 0 .. nv-1 valid)
};

__device__ __forceinline__ FlatLane flat_lane(int4 r, int lane) {
    FlatLane L;
    L.dgl = (r.y >> 4) & 1;
    L.nv = r.y >> 5;
    L.valid = lane < L.nv;
    const int e = (r.y & 15) + lane;
    const int du = L.dgl ? e / FOLD_TASKS_DIAG : e / FOLD_TASKS_PAIR;
    L.u = r.x + du;
    L.q = e - (L.dgl ? FOLD_TASKS_DIAG : FOLD_TASKS_PAIR) * du;
    return L;
}

__device__ __forceinline__ int4 flat_rec(const int4 *__restrict__ trec, int64_t w, int64_t ntiles) {
    return w < ntiles ? __ldg(trec + w) : make_int4(0, 0, 0, 0);  // no valid lane, no codes
}

// Fixed-point operands of the fold (policy STA_POLICY_FIXED, sta_fixed.cu): the quantised
// contributions at the element-cache offsets, the exponent of each entry and the integer sums,
// keyed by the value index of the entry's upper block.
struct FxArgs {
    const long long *Kq;
    const int16_t *e;
    long long *S;
};

// FX = false: the canonical FP64 fold.  FX = true: the same tiles, compaction and operand
// order over the quantised contributions with int64 adds (integer pipe), then S_k stored and
// converted once, val = double(S_k) 2^e_k (+ eps on the diagonal).
template <int WARPS, bool FX>  // warps per CTA: 2, 4 or 8 (at most 64 registers a thread)
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS)
k_fold_flat(FoldArgs A, const int4 *__restrict__ trec, int64_t ntiles, FxArgs X) {
    using V = typename std::conditional<FX, long long, double>::type;
    const V *__restrict__ src;
    if constexpr (FX) src = X.Kq; else src = A.Ke;
    __shared__ int32_t sbuf[WARPS][FLAT_CAP];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int32_t *scode = sbuf[threadIdx.x >> 5];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int4 Z4 = make_int4(0, 0, 0, 0);
    const bool has_eps = A.eps != 0.0;

    // pipeline prologue: records of tiles w, w+W, w+2W; unit records of w, w+W; codes of w
    int64_t w = warp;
    const int4 r0 = flat_rec(trec, w, ntiles), r1 = flat_rec(trec, w + W, ntiles);
    int4 r2 = flat_rec(trec, w + 2 * W, ntiles);
    FlatLane L = flat_lane(r0, lane);
    int4 bm0 = L.valid ? __ldg(A.bmeta + L.u) : Z4;
    int2 mir0 = L.valid && !L.dgl ? __ldg(A.bmirror + L.u) : make_int2(0, 0);
    FlatLane L1 = flat_lane(r1, lane);
    int4 bm1 = L1.valid ? __ldg(A.bmeta + L1.u) : Z4;
    int32_t cr0 = r0.z, cr1 = r0.w;  // the tile's code range
    int32_t code0 = cr0 + lane < cr1 ? __ldg(A.ccode + cr0 + lane) : 0;
    int32_t code0b = cr0 + 32 + lane < cr1 ? __ldg(A.ccode + cr0 + 32 + lane) : 0;
    int32_t code0c = cr0 + 64 + lane < cr1 ? __ldg(A.ccode + cr0 + 64 + lane) : 0;
    int32_t nr0 = r1.z, nr1 = r1.w;

    for (; w < ntiles; w += W) {  // warp-uniform
        // stage 0: tile record of w + 3W
        const int4 r3 = flat_rec(trec, w + 3 * W, ntiles);
        // stage 1: unit records of w + 2W
        const FlatLane L2 = flat_lane(r2, lane);
        const int4 bm2 = L2.valid ? __ldg(A.bmeta + L2.u) : Z4;
        // stage 2: first three code chunks and mirror records of w + W
        const int32_t code1 = nr0 + lane < nr1 ? __ldg(A.ccode + nr0 + lane) : 0;
        const int32_t code1b = nr0 + 32 + lane < nr1 ? __ldg(A.ccode + nr0 + 32 + lane) : 0;
        const int32_t code1c = nr0 + 64 + lane < nr1 ? __ldg(A.ccode + nr0 + 64 + lane) : 0;
        const int2 mir1 = L1.valid && !L1.dgl ? __ldg(A.bmirror + L1.u) : make_int2(0, 0);

        // stage 3: tile w -- compact its active codes
        int base = 0, lo = 0, hi = 0;
        for (int32_t c0 = cr0; c0 < cr1; c0 += 32) {  // warp-uniform
            const int32_t c = c0 + lane;
            const int32_t code = c0 == cr0        ? code0
                                 : c0 == cr0 + 32 ? code0b
                                 : c0 == cr0 + 64 ? code0c
                                                  : (c < cr1 ? __ldg(A.ccode + c) : 0);
            const unsigned m = __ballot_sync(FULL, code < 0);
            const int pos = base + __popc(m & below);
            if (code < 0 && pos < FLAT_CAP) scode[pos] = (int32_t)word_offset((uint32_t)code);
            const int dz = bm0.z - c0, dw = bm0.w - c0;
            if (dz >= 0 && dz < 32) lo = base + __popc(m & ((1u << dz) - 1u));
            if (dw >= 0 && dw < 32) hi = base + __popc(m & ((1u << dw) - 1u));
            base += __popc(m);
        }
        if (bm0.z >= cr1) lo = base;
        if (bm0.w >= cr1) hi = base;
        __syncwarp();
        const int n = L.valid ? hi - lo : 0;
        const bool dgl = L.dgl;
        const int q = L.q;
        // 6-run entry q = (i, j), i <= j, of a diagonal unit; 3x3 row-major of a pair unit
        const int ei = dgl ? (q < 3 ? 0 : (q < 5 ? 1 : 2)) : q / 3;
        const int ej = dgl ? (q < 3 ? q : (q < 5 ? q - 2 : 2)) : q % 3;
        const int32_t key = bm0.x + ei * (bm0.y >> 1) + ej;
        int ex = 0;  // the entry's fixed-point exponent, loaded before the fold
        if constexpr (FX) ex = L.valid ? (int)__ldg(X.e + key) : 0;
        V acc = V(0);
        if (base <= FLAT_CAP) {
            const int maxn = __reduce_max_sync(FULL, n);
            // staged entries are element-cache offsets of the contributors' runs
            const uint32_t *sc = reinterpret_cast<const uint32_t *>(scode) + lo;
            // every guard on maxn is warp-uniform: a tile issues no operand work past its
            // longest fold (a tile of units without active contributors issues none at all)
#define STA_LD(j) ((j) < n ? __ldg(src + sc[(j)] + q) : V(0))
            if (maxn > 0) {
                if constexpr (FX) acc = STA_LD(0);
                else acc = plus_zero(STA_LD(0));  // the first contribution: +0.0 + v, no FP64 add
                V v0 = V(0), v1 = V(0), v2 = V(0), v3 = V(0);
                if (maxn > 1) v0 = STA_LD(1);
                if (maxn > 2) v1 = STA_LD(2);
                if (maxn > 3) v2 = STA_LD(3);
                if (maxn > 4) v3 = STA_LD(4);
                int j = 1;
                for (; j + 4 <= maxn; j += 4) {  // next 4 operands in flight
                    V x0 = V(0), x1 = V(0), x2 = V(0), x3 = V(0);
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
        } else if (L.valid) {  // rare: more active codes than staged; fold from the list itself
            int j = 0;
            for (int32_t c = bm0.z; c < bm0.w; ++c) {
                const int32_t code = __ldg(A.ccode + c);
                if (code >= 0) continue;
                const V v = __ldg(src + word_offset((uint32_t)code) + q);
                if constexpr (FX) acc += v;
                else acc = j == 0 ? plus_zero(v) : acc + v;
                ++j;
            }
        }
        if (L.valid) {
            double a;
            if constexpr (FX) {
                X.S[key] = acc;
                a = __ll2double_rn(acc) * pow2i(ex);
            } else {
                a = acc;
            }
            if (dgl) {  // mirrored inside the block; eps on the diagonal
                if (ei == ej && has_eps) a += A.eps;
                A.val[key] = a;
                if (ei != ej) A.val[bm0.x + ej * (bm0.y >> 1) + ei] = a;
            } else {
                A.val[key] = a;
                A.val[mir0.x + ej * mir0.y + ei] = a;
            }
        }
        __syncwarp();
        // advance the pipeline
        L = L1;
        bm0 = bm1;
        mir0 = mir1;
        cr0 = nr0;
        cr1 = nr1;
        code0 = code1;
        code0b = code1b;
        code0c = code1c;
        L1 = L2;
        bm1 = bm2;
        nr0 = r2.z;
        nr1 = r2.w;
        r2 = r3;
    }
}

}  // namespace

// Full rebuild: the flat entry-parallel fold over all tiles, with the context's CTA shape
// (block_threads 64, 128 or 256; blocks_per_sm 0 = occupancy maximum).
int launch_rebuild(Ctx *c, cudaStream_t s) {
    if (c->ntiles == 0) return STA_OK;
    const bool fx = c->policy == STA_POLICY_FIXED;
    const FxArgs X{c->fx_q, c->fx_e, c->fx_s};
    const int threads = c->block_threads == 64 || c->block_threads == 256 ? c->block_threads : 128;
    const void *kern = threads == 64    ? (fx ? (const void *)k_fold_flat<2, true>
                                              : (const void *)k_fold_flat<2, false>)
                       : threads == 256 ? (fx ? (const void *)k_fold_flat<8, true>
                                              : (const void *)k_fold_flat<8, false>)
                                        : (fx ? (const void *)k_fold_flat<4, true>
                                              : (const void *)k_fold_flat<4, false>);
    const int grid = persistent_grid(c, kern, threads, c->ntiles * 32, true);
    const FoldArgs A = fold_args(c);
    if (threads == 64) {
        if (fx) k_fold_flat<2, true><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
        else k_fold_flat<2, false><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
    } else if (threads == 256) {
        if (fx) k_fold_flat<8, true><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
        else k_fold_flat<8, false><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
    } else {
        if (fx) k_fold_flat<4, true><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
        else k_fold_flat<4, false><<<grid, threads, 0, s>>>(A, c->ftile, c->ntiles, X);
    }
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace sta
