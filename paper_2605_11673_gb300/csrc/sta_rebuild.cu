// Full rebuild (the full_rebuild policy of Sec. 3.5): every value of the
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

// One tile of the flat fold: compact the active codes of the tile's code range into shared
// memory, fold each lane's entry, write it and its mirror.  `code0..2` are the first three
// 32-code chunks of the range (already loaded), `bm`, `mir` the lane's unit records.  A tile
// that is not `live` (a code range of at most 96 codes, none active) folds nothing: every
// entry is the empty fold +0.0 (+ eps on the diagonal), written only if `write_dead`.
template <bool FX, int PF, typename V>
__device__ __forceinline__ void flat_tile(const FoldArgs &A, const FxArgs &X, const V *__restrict__ src,
                                          int32_t *scode, int lane, const FlatLane &L, int4 bm,
                                          int2 mir, int32_t cr0, int32_t cr1, int32_t code0,
                                          int32_t code0b, int32_t code0c, bool live,
                                          bool write_dead) {
    const unsigned FULL = 0xffffffffu;
    const unsigned below = (1u << lane) - 1u;
    int base = 0, lo = 0, hi = 0;
    if (live) {
        for (int32_t c0 = cr0; c0 < cr1; c0 += 32) {  // warp-uniform
            const int32_t c = c0 + lane;
            const int32_t code = c0 == cr0        ? code0
                                 : c0 == cr0 + 32 ? code0b
                                 : c0 == cr0 + 64 ? code0c
                                                  : (c < cr1 ? __ldg(A.ccode + c) : 0);
            const unsigned m = __ballot_sync(FULL, code < 0);
            const int pos = base + __popc(m & below);
            if (code < 0 && pos < FLAT_CAP) scode[pos] = (int32_t)word_offset((uint32_t)code);
            const int dz = bm.z - c0, dw = bm.w - c0;
            if (dz >= 0 && dz < 32) lo = base + __popc(m & ((1u << dz) - 1u));
            if (dw >= 0 && dw < 32) hi = base + __popc(m & ((1u << dw) - 1u));
            base += __popc(m);
        }
        if (bm.z >= cr1) lo = base;
        if (bm.w >= cr1) hi = base;
    }
    __syncwarp();
    const int n = L.valid ? hi - lo : 0;
    const bool dgl = L.dgl;
    const int q = L.q;
    // 6-run entry q = (i, j), i <= j, of a diagonal unit; 3x3 row-major of a pair unit
    const int ei = dgl ? (q < 3 ? 0 : (q < 5 ? 1 : 2)) : q / 3;
    const int ej = dgl ? (q < 3 ? q : (q < 5 ? q - 2 : 2)) : q % 3;
    const int32_t key = bm.x + ei * (bm.y >> 1) + ej;
    int ex = 0;  // the entry's fixed-point exponent, loaded before the fold
    if constexpr (FX) ex = L.valid && (live || write_dead) ? (int)__ldg(X.e + key) : 0;
    V acc = V(0);
    if (!live) {
        // no active contributor in the tile: every fold is the empty fold
    } else if (base <= FLAT_CAP) {
        const int maxn = __reduce_max_sync(FULL, n);
        // staged entries are element-cache offsets of the contributors' runs
        const uint32_t *sc = reinterpret_cast<const uint32_t *>(scode) + lo;
        // every guard on maxn is warp-uniform: a tile issues no operand work past its
        // longest fold (a tile of units without active contributors issues none at all)
#define STA_LD(j) ((j) < n ? __ldg(src + sc[(j)] + q) : V(0))
        if (maxn > 0 && PF != 4) {  // PF operands in flight, in registers v[]
            if constexpr (FX) acc = STA_LD(0);
            else acc = plus_zero(STA_LD(0));  // the first contribution: +0.0 + v, no FP64 add
            V v[PF];
#pragma unroll
            for (int k = 0; k < PF; ++k) v[k] = maxn > 1 + k ? STA_LD(1 + k) : V(0);
            int j = 1;
            for (; j + PF <= maxn; j += PF) {  // next PF operands in flight
                V x[PF];
#pragma unroll
                for (int k = 0; k < PF; ++k) x[k] = j + PF + k < maxn ? STA_LD(j + PF + k) : V(0);
#pragma unroll
                for (int k = 0; k < PF; ++k)
                    if (j + k < n) acc += v[k];
#pragma unroll
                for (int k = 0; k < PF; ++k) v[k] = x[k];
            }
#pragma unroll
            for (int k = 0; k < PF - 1; ++k)
                if (j + k < maxn && j + k < n) acc += v[k];
        } else if (maxn > 0) {  // PF == 4, written out (the array form spills in one instance)
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
        for (int32_t c = bm.z; c < bm.w; ++c) {
            const int32_t code = __ldg(A.ccode + c);
            if (code >= 0) continue;
            const V v = __ldg(src + word_offset((uint32_t)code) + q);
            if constexpr (FX) acc += v;
            else acc = j == 0 ? plus_zero(v) : acc + v;
            ++j;
        }
    }
    if (L.valid && (live || write_dead)) {
        double a;
        if constexpr (FX) {
            X.S[key] = acc;
            a = __ll2double_rn(acc) * pow2i(ex);
        } else {
            a = acc;
        }
        if (dgl) {  // mirrored inside the block; eps on the diagonal
            if (ei == ej && A.eps != 0.0) a += A.eps;
            A.val[key] = a;
            if (ei != ej) A.val[bm.x + ej * (bm.y >> 1) + ei] = a;
        } else {
            A.val[key] = a;
            A.val[mir.x + ej * mir.y + ei] = a;
        }
    }
    __syncwarp();
}

// whether a tile must be folded: its code range is longer than the three chunks in registers,
// or one of them holds an active code (bit 31; lanes past the range hold 0)
__device__ __forceinline__ bool tile_live(int32_t cr0, int32_t cr1, int32_t c0, int32_t c1,
                                          int32_t c2) {
    return (cr1 - cr0 > 96) || __any_sync(0xffffffffu, (c0 | c1 | c2) < 0);
}

// The zero-fill form's tiles of one warp: the positions k = 0, 1, ... of its stripe (tile
// w + k W) whose flag is set.  The flags of 32 positions are read at once (one per lane),
// those of the next 32 one step ahead, and handed out from a ballot.  Every flag is read by
// the one warp whose stripe holds it, and that lane clears it: once the fold has run, all
// flags are zero again for the next rebuild's flag pass.
struct FlagStream {
    int32_t base;    // stripe position of bit 0 of `mask`
    unsigned mask;   // set flags of positions base .. base+31 not yet handed out
    uint8_t ahead;   // this lane's flag of position base + 32 + lane
    __device__ __forceinline__ void load_ahead(uint8_t *__restrict__ flags, int32_t w,
                                               int32_t W, int32_t ntiles, int lane) {
        const int64_t t = w + (int64_t)(base + 32 + lane) * W;
        ahead = t < ntiles ? flags[t] : 0;
        if (ahead) flags[t] = 0;
    }
    // the next flagged tile, or ntiles past the end of the stripe
    __device__ __forceinline__ int32_t next(uint8_t *__restrict__ flags, int32_t w,
                                            int32_t W, int32_t ntiles, int lane) {
        while (mask == 0) {  // warp-uniform
            base += 32;
            if (w + (int64_t)base * W >= ntiles) return ntiles;
            mask = __ballot_sync(0xffffffffu, ahead != 0);
            load_ahead(flags, w, W, ntiles, lane);
        }
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        return w + (base + b) * W;
    }
};

// FX = false: the canonical FP64 fold.  FX = true: the same tiles, compaction and operand
// order over the quantised contributions with int64 adds (integer pipe), then S_k stored and
// converted once, val = double(S_k) 2^e_k (+ eps on the diagonal).
// ZF = false (fused form): every tile, each writing all its entries, +0.0 for the tiles
// without an active code.  ZF = true (zero-fill form): the values were set to zero and the
// tiles to fold flagged by k_tile_flags; the warp visits only the flagged tiles of its stripe.
// PF: operand loads in flight per lane, 4 (at most 64 registers a thread: 32 resident warps per
// SM) or 6 (at most 80: 24 warps).  The fold is bound by load latency; which of the two hides
// it better depends on the workload (the autotuner chooses).
template <int WARPS, bool FX, bool ZF, int PF>  // warps per CTA: 2, 4 or 8
__global__ void __launch_bounds__(WARPS * 32, (PF == 4 ? 32 : 24) / WARPS)
k_fold_flat(FoldArgs A, const int4 *__restrict__ trec, int64_t ntiles, FxArgs X,
            uint8_t *__restrict__ tflag) {
    using V = typename std::conditional<FX, long long, double>::type;
    const V *__restrict__ src;
    if constexpr (FX) src = X.Kq; else src = A.Ke;
    __shared__ int32_t sbuf[WARPS][FLAT_CAP];
    const int lane = threadIdx.x & 31;
    int32_t *scode = sbuf[threadIdx.x >> 5];
    // tile indices fit int32: the pattern has fewer than 2^31 entries, 32 per tile
    const int32_t nt = (int32_t)ntiles;
    const int32_t warp = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t W = (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int4 Z4 = make_int4(0, 0, 0, 0);

    // the warp's tiles: w, w+W, w+2W, ... (fused) or the flagged ones among them (zero fill);
    // past the end, nt (a tile index with the empty record)
    FlagStream fs{-32, 0u, 0};
    if constexpr (ZF) fs.load_ahead(tflag, warp, W, nt, lane);
    auto next_tile = [&](int32_t t) -> int32_t {
        if constexpr (ZF) return fs.next(tflag, warp, W, nt, lane);
        else return t < nt - W ? t + W : nt;
    };
    // pipeline prologue: records of tiles t0, t1, t2; unit records of t0, t1; codes of t0
    const int32_t t0 = ZF ? next_tile(0) : (warp < nt ? warp : nt);
    const int32_t t1 = next_tile(t0);
    int32_t t2 = next_tile(t1);
    const int4 r0 = flat_rec(trec, t0, ntiles), r1 = flat_rec(trec, t1, ntiles);
    int4 r2 = flat_rec(trec, t2, ntiles);
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

    // a warp's tiles increase; past the end of its stripe the record is the empty one
    while (L.nv > 0) {  // warp-uniform
        // stage 0: tile record of t3
        t2 = next_tile(t2);  // now t3
        const int4 r3 = flat_rec(trec, t2, ntiles);
        // stage 1: unit records of t2
        const FlatLane L2 = flat_lane(r2, lane);
        const int4 bm2 = L2.valid ? __ldg(A.bmeta + L2.u) : Z4;
        // stage 2: first three code chunks and mirror records of t1
        const int32_t code1 = nr0 + lane < nr1 ? __ldg(A.ccode + nr0 + lane) : 0;
        const int32_t code1b = nr0 + 32 + lane < nr1 ? __ldg(A.ccode + nr0 + 32 + lane) : 0;
        const int32_t code1c = nr0 + 64 + lane < nr1 ? __ldg(A.ccode + nr0 + 64 + lane) : 0;
        const int2 mir1 = L1.valid && !L1.dgl ? __ldg(A.bmirror + L1.u) : make_int2(0, 0);
        // stage 3: tile t0 (a tile without an active code skips the compaction and the fold)
        flat_tile<FX, PF, V>(A, X, src, scode, lane, L, bm0, mir0, cr0, cr1, code0, code0b, code0c,
                         tile_live(cr0, cr1, code0, code0b, code0c), true);
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

// Zero-fill form, first pass.  Flags the tiles the fold must visit -- every tile holding a fold
// entry of a unit with an active contributor, and with eps != 0 every diagonal tile (`tdiag`,
// else null) -- into `tflag`, which is all zero at launch (the previous fold cleared what it
// read), and sets every value (and, for the fixed-point fold, every integer sum) to zero with
// 16-byte stores.  The flags come from the mask: each active
// tetrahedron's 10 units, each in one tile or two consecutive ones; a thread reads the mask of 4
// tetrahedra at once and an active tetrahedron's 10 unit words together.  The flags are plain
// byte stores of 1 (any order, no atomics).  Flags first: the warps with active tetrahedra wait
// on their loads while the others are already filling.
__global__ void k_tile_flags(const uint8_t *__restrict__ mask, const int32_t *__restrict__ tunit,
                             const int32_t *__restrict__ utile, int64_t T, uint8_t *__restrict__ tflag,
                             const uint8_t *__restrict__ tdiag, int64_t ntiles,
                             double *__restrict__ val, long long *__restrict__ S, int64_t nnz) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    if (tdiag)  // eps on the diagonal: every diagonal tile is folded
        for (int64_t t = tid; t < ntiles; t += nthreads)
            if (__ldg(tdiag + t)) tflag[t] = 1;
    // tile flags: tetrahedra 4q .. 4q+3 per step (the mask is cudaMalloc'd, so its 4-byte
    // words are aligned; the last word may be partial)
    for (int64_t q = tid; 4 * q < T; q += nthreads) {
        uint32_t m4;
        if (4 * q + 4 <= T) {
            m4 = __ldg(reinterpret_cast<const uint32_t *>(mask) + q);
        } else {
            m4 = 0;
            for (int64_t t = 4 * q; t < T; ++t) m4 |= (uint32_t)__ldg(mask + t) << (8 * (t - 4 * q));
        }
        if (!m4) continue;
        for (int k = 0; k < 4; ++k) {
            if (!((m4 >> (8 * k)) & 0xffu)) continue;
            const int64_t t = 4 * q + k;
            // the tet's 10 unit words (40 bytes at 10 t of a cudaMalloc'd array: 8-byte aligned)
            const int2 *tu2 = reinterpret_cast<const int2 *>(tunit + 10 * t);
            int32_t uu[10], ut[10];
#pragma unroll
            for (int h = 0; h < 5; ++h) {
                const int2 v = __ldg(tu2 + h);
                uu[2 * h] = v.x;
                uu[2 * h + 1] = v.y;
            }
#pragma unroll
            for (int sl = 0; sl < 10; ++sl) ut[sl] = __ldg(utile + uu[sl]);
#pragma unroll
            for (int sl = 0; sl < 10; ++sl) {
                const int32_t t0 = ut[sl] & INT32_MAX;
                tflag[t0] = 1;
                if (ut[sl] < 0) tflag[t0 + 1] = 1;  // the unit reaches into the next tile
            }
        }
    }
    // zero fill (both arrays are cudaMalloc'd, 256-byte aligned; an odd last word alone)
    for (int64_t i = tid; i < (nnz >> 1); i += nthreads) {
        reinterpret_cast<double2 *>(val)[i] = make_double2(0.0, 0.0);
        if (S) reinterpret_cast<longlong2 *>(S)[i] = make_longlong2(0, 0);
    }
    if (tid == 0 && (nnz & 1)) {
        val[nnz - 1] = 0.0;
        if (S) S[nnz - 1] = 0;
    }
}

template <int WARPS, bool FX, bool ZF, int PF>
int launch_flat(Ctx *c, const FoldArgs &A, const FxArgs &X, cudaStream_t s) {
    const void *kern = (const void *)k_fold_flat<WARPS, FX, ZF, PF>;
    const int grid = persistent_grid(c, kern, WARPS * 32, c->ntiles * 32, true);
    k_fold_flat<WARPS, FX, ZF, PF><<<grid, WARPS * 32, 0, s>>>(A, c->ftile, c->ntiles, X, c->tflag);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

template <bool FX, bool ZF, int PF>
int launch_flat_shape(Ctx *c, const FoldArgs &A, const FxArgs &X, cudaStream_t s) {
    if (c->block_threads == 64) return launch_flat<2, FX, ZF, PF>(c, A, X, s);
    if (c->block_threads == 256) return launch_flat<8, FX, ZF, PF>(c, A, X, s);
    return launch_flat<4, FX, ZF, PF>(c, A, X, s);
}

template <bool FX, bool ZF>
int launch_fold(Ctx *c, cudaStream_t s) {
    const FxArgs X{c->fx_q, c->fx_e, c->fx_s};
    const FoldArgs A = fold_args(c);
    if (ZF) {  // the flags are all zero here: the previous zero-fill fold cleared them
        k_tile_flags<<<c->num_sms * 8, 256, 0, s>>>(c->mask, c->tunit, c->utile, c->T, c->tflag,
                                                    c->eps != 0.0 ? c->tdiag : nullptr, c->ntiles,
                                                    c->val, FX ? c->fx_s : nullptr, c->nnz);
        STA_CUDA_TRY(cudaGetLastError());
    }
    return c->fold_depth == 6 ? launch_flat_shape<FX, ZF, 6>(c, A, X, s)
                              : launch_flat_shape<FX, ZF, 4>(c, A, X, s);
}

}  // namespace

// AUTO: the zero-fill form while fewer than 40% of the tetrahedra are active.  Measured on
// GB300: a refinement hierarchy with 12% of its superset active rebuilds in about a third of
// the fused form's time; a pre-fractured block with 66% active is faster fused.
int rebuild_form_of(const Ctx *c) {
    if (c->rebuild_form != STA_REBUILD_AUTO) return c->rebuild_form;
    return c->n_active * 5 < c->T * 2 ? STA_REBUILD_ZERO_FILL : STA_REBUILD_FUSED;
}

// Full rebuild: the flat entry-parallel fold over all tiles, with the context's launch shape
// (block_threads 64, 128 or 256; blocks_per_sm 0 = occupancy maximum; fold_depth 4 or 6
// operand loads in flight) and rebuild form (rebuild_form_of: fused, or zero fill + fold of the
// tiles with an active contributor).
int launch_rebuild(Ctx *c, cudaStream_t s) {
    if (c->ntiles == 0) return STA_OK;
    const bool fx = c->policy == STA_POLICY_FIXED;
    if (rebuild_form_of(c) == STA_REBUILD_ZERO_FILL)
        return fx ? launch_fold<true, true>(c, s) : launch_fold<false, true>(c, s);
    return fx ? launch_fold<true, false>(c, s) : launch_fold<false, false>(c, s);
}

}  // namespace sta
