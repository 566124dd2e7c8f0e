// Fold kernels: full rebuild (a2) and streaming update (a3).
//
// Both evaluate, for a node-pair block (a, b) of the superset pattern, the 9 CSR values
//   A[3a+i][3b+j] = fold_{tau active, ascending id} K^(tau)[3 la + i][3 lb + j]   (+ eps)
// i.e. Eq. 8 of STA-FEM restricted to one block, with the fold starting at +0.0 and eps
// added afterwards on the diagonal.  The work unit is an unordered node pair {a <= b}: the
// element matrices are stored exactly symmetric, so block (b, a) folds the same operands in
// the same order as (a, b) and one fold writes both.  The streaming pass (Sec. 3.2,
// Algorithm 1; the local_recompute policy of Sec. 3.5) folds the units touched by the frame's
// edits only, with the same operands, order and operations, so its values are bit-identical
// to the rebuild's.
//
// No atomics touch values: each entry is folded by exactly one lane, and the summation order
// is the order of the unit's contributor list (ascending tetrahedron id), independent of the
// kernel and the launch configuration.  Every fold starts with (+0.0 + c1) formed without an
// FP64 operation (plus_zero) and continues with one FP64 add per further contribution.
#include <climits>

#include "sta_internal.cuh"

namespace sta {
namespace {

struct FoldArgs {
    const int4 *__restrict__ bmeta;     // per unit: value offset of (a,b), rs_a << 1 | diag, c0, c1
    const int2 *__restrict__ bmirror;   // per unit: value offset of (b,a), rs_b
    const int32_t *__restrict__ ccode;  // contributor words: element-cache offset | active << 31
    const double *__restrict__ Ke;
    double *__restrict__ val;
    double eps;
};

// +0.0 + v without an FP64 operation: identical except that -0.0 becomes +0.0.
__device__ __forceinline__ double plus_zero(double v) {
    long long bits = __double_as_longlong(v);
    return __longlong_as_double(bits == (long long)0x8000000000000000ULL ? 0LL : bits);
}

// The operands one contributor (word w) supplies to a fold unit {a, b}, id(a) <= id(b): its
// run of the element cache read row-major, with 16-byte loads --
//   diagonal unit:     the 6-run of (a, a): v[0..5] = (0,0) (0,1) (0,2) (1,1) (1,2) (2,2); the
//                      mirrored entries (j, i) fold the same operands;
//   off-diagonal unit: the 9-run, v[3i+j] = K[3la+i][3lb+j] (runs are stored oriented by id).
// The mirror block (b, a) folds exactly the same operand sequence (K is stored exactly
// symmetric), so one fold per unit gives both blocks' values bit for bit.
__device__ __forceinline__ void load_contrib(const FoldArgs &A, int32_t w, bool diag, double v[9]) {
    const double2 *r = reinterpret_cast<const double2 *>(A.Ke + word_offset((uint32_t)w));
    const double2 p0 = __ldg(r), p1 = __ldg(r + 1), p2 = __ldg(r + 2);
    v[0] = p0.x; v[1] = p0.y; v[2] = p1.x;
    v[3] = p1.y; v[4] = p2.x; v[5] = p2.y;
    if (diag) {
        v[6] = 0.0; v[7] = 0.0; v[8] = 0.0;
    } else {
        const double2 p3 = __ldg(r + 3), p4 = __ldg(r + 4);
        v[6] = p3.x; v[7] = p3.y; v[8] = p4.x;
    }
}

// first position >= c in [c, ce) whose contributor is active (code bit 31 set)
__device__ __forceinline__ int32_t next_active(const FoldArgs &A, int32_t c, int32_t ce) {
    while (c < ce && __ldg(A.ccode + c) >= 0) ++c;
    return c;
}

struct BlockOut {
    double *out;   // block (a, b)
    double *out2;  // its mirror (b, a)
    int rs, rs2;
    bool diag;
};

__device__ __forceinline__ BlockOut unit_out(const FoldArgs &A, int4 bm, int2 mir) {
    return BlockOut{A.val + bm.x, A.val + mir.x, bm.y >> 1, mir.y, (bm.y & 1) != 0};
}

// Writes a unit's folds: a diagonal unit's 6 folds to the 9 entries of its block (mirrored,
// eps added to the diagonal entries last); an off-diagonal unit's 9 folds to (a, b) and,
// transposed, to (b, a).
__device__ __forceinline__ void write_block(const FoldArgs &A, const BlockOut &o, double acc[9]) {
    if (o.diag) {
        if (A.eps != 0.0) {
            acc[0] += A.eps;
            acc[3] += A.eps;
            acc[5] += A.eps;
        }
        const int tri[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) o.out[i * o.rs + j] = acc[tri[i][j]];
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                o.out[i * o.rs + j] = acc[3 * i + j];
                o.out2[j * o.rs2 + i] = acc[3 * i + j];
            }
    }
}

// One lane folds a whole unit from global memory (units larger than the shared buffers).
__device__ void fold_direct(const FoldArgs &A, const int4 bm, const int2 mir) {
    const bool diag = (bm.y & 1) != 0;
    double acc[9], v[9];
    int32_t c = next_active(A, bm.z, bm.w);
    if (c == bm.w) {
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    } else {
        load_contrib(A, __ldg(A.ccode + c), diag, acc);
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = plus_zero(acc[q]);
        for (c = next_active(A, c + 1, bm.w); c < bm.w; c = next_active(A, c + 1, bm.w)) {
            load_contrib(A, __ldg(A.ccode + c), diag, v);
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] += v[q];  // (diagonal: entries 6..8 unused)
        }
    }
    write_block(A, unit_out(A, bm, mir), acc);
}

// ------------------------------------------------------------------------------------------
// Entry-parallel fold of a list of units (streaming).  A frame's touched list is short and its
// longest folds (diagonal units, ~24 contributions) set the latency, so here each lane folds ONE
// matrix entry: a warp takes 3 listed units, lanes 9g .. 9g+8 fold the 9 entries (i, j) of
// unit g (6 of them for a diagonal unit), and one FP64 instruction per step advances all 27
// folds.  The unit's active codes are compacted (in list order) into shared memory first; each
// step then loads one operand per lane (4 steps of loads in flight).  Operands, order and
// operations are those of k_fold_flat, so the values are the same bits.
// ------------------------------------------------------------------------------------------
constexpr int ENT_UNITS = 3;    // units per warp round (27 lanes)
constexpr int ENT_CAP = 96;     // active contributions staged per unit; larger units fold directly
constexpr int ENT_WARPS = 4;

__global__ void __launch_bounds__(ENT_WARPS * 32)
k_fold_entries(FoldArgs A, const int32_t *__restrict__ list, const unsigned long long *__restrict__ count) {
    __shared__ uint32_t sop_all[ENT_WARPS][ENT_UNITS][ENT_CAP];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / 9, q = lane % 9;  // g == 3: lanes 27..31 idle
    const int qi = q / 3, qj = q % 3;
    uint32_t *sop = sop_all[wid][g < ENT_UNITS ? g : 0];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = (int64_t)*count;
    const bool has_eps = A.eps != 0.0;
    for (int64_t base = warp * ENT_UNITS; base < nitems; base += nwarps * ENT_UNITS) {  // warp-uniform
        const int64_t item = base + g;
        const bool valid = g < ENT_UNITS && item < nitems;
        int4 bm = make_int4(0, 0, 0, 0);
        int2 mir = make_int2(0, 0);
        if (valid) {
            const int32_t u = __ldg(list + item);
            bm = __ldg(A.bmeta + u);
            mir = __ldg(A.bmirror + u);
        }
        // compact the unit's active contributors (as operand bases), 9 lanes striding over its list
        int nact = 0;
        const int span = valid ? bm.w - bm.z : 0;
        const int max_span = __reduce_max_sync(FULL, span);
        for (int c0 = 0; c0 < max_span; c0 += 9) {
            const int c = c0 + q;
            const int32_t code = (valid && c < span) ? __ldg(A.ccode + bm.z + c) : 0;
            const unsigned m = __ballot_sync(FULL, code < 0);
            const unsigned gm = (m >> (9 * g)) & 0x1ffu;
            const int pos = nact + __popc(gm & ((1u << q) - 1u));
            if (code < 0 && pos < ENT_CAP) sop[pos] = word_offset((uint32_t)code);
            nact += __popc(gm);
        }
        __syncwarp();
        const bool big = valid && nact > ENT_CAP;
        if (big && q == 0) fold_direct(A, bm, mir);  // rare: more active contributions than staged
        const bool diag = (bm.y & 1) != 0;
        const bool mine = valid && !big && (!diag || q < 6);  // a diagonal unit folds 6 entries
        const int n = mine ? nact : 0;
        double acc = 0.0;
        const int maxn = __reduce_max_sync(FULL, n);
#define STA_LD(j) ((j) < n ? __ldg(A.Ke + sop[(j)] + q) : 0.0)
        if (maxn > 0) {  // warp-uniform guards, as in k_fold_flat
            acc = plus_zero(STA_LD(0));  // the first contribution: +0.0 + v, no FP64 add
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

// ------------------------------------------------------------------------------------------
// Flat entry-parallel rebuild.  Every fold entry of the pattern gets a lane: 6 per diagonal
// unit, 9 per off-diagonal unit.  A warp tile is 32 consecutive entries of units of one kind
// (tile records built at create: first unit, entry offset, kind, entry count); its units (up to
// 7) have contiguous contributor codes.  The warp compacts the active codes of that range into
// shared memory with ballots (list order kept, so each unit's active codes form one segment),
// each lane locates its unit's segment from the same ballots, and every FP64 add instruction
// then advances up to 32 folds.  Units are ordered so that a tile's lists have equal length.
//
// Each tile needs three dependent loads before its first add (tile record -> unit record ->
// codes), so the persistent warps run them as a software pipeline: while tile w folds, the
// first code chunk of tile w+W, the unit records of tile w+2W and the tile record of tile w+3W
// are in flight (W = warps in the grid).  Operands, order and operations are those of
// fold_direct and k_fold_entries.
// ------------------------------------------------------------------------------------------
constexpr int FLAT_CAP = 448;  // staged active codes per tile; a larger tile folds from the list


struct FlatLane {
    int32_t u;  // unit
    int q;      // entry of the unit
    bool dgl, valid;
    int nv;     // entries in the tile (lanes 0 .. nv-1 valid)
};

__device__ __forceinline__ FlatLane flat_lane(int2 r, int lane) {
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

__device__ __forceinline__ int2 flat_rec(const int2 *__restrict__ trec, int64_t w, int64_t ntiles) {
    return w < ntiles ? __ldg(trec + w) : make_int2(0, 0);  // nv = 0: no valid lane
}

template <int WARPS>  // warps per CTA: 2, 4 or 8 (at most 64 registers a thread)
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS)
k_fold_flat(FoldArgs A, const int2 *__restrict__ trec, int64_t ntiles) {
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
    int2 r0 = flat_rec(trec, w, ntiles), r1 = flat_rec(trec, w + W, ntiles),
         r2 = flat_rec(trec, w + 2 * W, ntiles);
    FlatLane L = flat_lane(r0, lane);
    int4 bm0 = L.valid ? __ldg(A.bmeta + L.u) : Z4;
    int2 mir0 = L.valid && !L.dgl ? __ldg(A.bmirror + L.u) : make_int2(0, 0);
    FlatLane L1 = flat_lane(r1, lane);
    int4 bm1 = L1.valid ? __ldg(A.bmeta + L1.u) : Z4;
    int32_t cr0 = __shfl_sync(FULL, bm0.z, 0), cr1 = __shfl_sync(FULL, bm0.w, L.nv > 0 ? L.nv - 1 : 0);
    if (L.nv == 0) cr0 = cr1 = 0;
    int32_t code0 = cr0 + lane < cr1 ? __ldg(A.ccode + cr0 + lane) : 0;

    for (; w < ntiles; w += W) {  // warp-uniform
        // stage 0: tile record of w + 3W
        const int2 r3 = flat_rec(trec, w + 3 * W, ntiles);
        // stage 1: unit records of w + 2W
        const FlatLane L2 = flat_lane(r2, lane);
        const int4 bm2 = L2.valid ? __ldg(A.bmeta + L2.u) : Z4;
        // stage 2: first code chunk and mirror records of w + W
        int32_t nr0 = __shfl_sync(FULL, bm1.z, 0), nr1 = __shfl_sync(FULL, bm1.w, L1.nv > 0 ? L1.nv - 1 : 0);
        if (L1.nv == 0) nr0 = nr1 = 0;
        const int32_t code1 = nr0 + lane < nr1 ? __ldg(A.ccode + nr0 + lane) : 0;
        const int2 mir1 = L1.valid && !L1.dgl ? __ldg(A.bmirror + L1.u) : make_int2(0, 0);

        // stage 3: tile w -- compact its active codes
        int base = 0, lo = 0, hi = 0;
        for (int32_t c0 = cr0; c0 < cr1; c0 += 32) {  // warp-uniform
            const int32_t c = c0 + lane;
            const int32_t code = c0 == cr0 ? code0 : (c < cr1 ? __ldg(A.ccode + c) : 0);
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
        double acc = 0.0;
        if (base <= FLAT_CAP) {
            const int maxn = __reduce_max_sync(FULL, n);
            // staged entries are element-cache offsets of the contributors' runs
            const uint32_t *sc = reinterpret_cast<const uint32_t *>(scode) + lo;
            // every guard on maxn is warp-uniform: a tile issues no operand work past its
            // longest fold (a tile of units without active contributors issues none at all)
#define STA_LD(j) ((j) < n ? __ldg(A.Ke + sc[(j)] + q) : 0.0)
            if (maxn > 0) {
                acc = plus_zero(STA_LD(0));  // the first contribution: +0.0 + v, no FP64 add
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
        } else if (L.valid) {  // rare: more active codes than staged; fold from the list itself
            int j = 0;
            for (int32_t c = bm0.z; c < bm0.w; ++c) {
                const int32_t code = __ldg(A.ccode + c);
                if (code >= 0) continue;
                const double v = __ldg(A.Ke + word_offset((uint32_t)code) + q);
                acc = j == 0 ? plus_zero(v) : acc + v;
                ++j;
            }
        }
        if (L.valid) {
            const int rs = bm0.y >> 1;
            if (dgl) {  // 6-run entry q = (i, j), i <= j, mirrored; eps on the diagonal
                const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
                double a = acc;
                if (i == j && has_eps) a += A.eps;
                A.val[bm0.x + i * rs + j] = a;
                if (i != j) A.val[bm0.x + j * rs + i] = a;
            } else {
                const int qi = q / 3, qj = q % 3;
                A.val[bm0.x + qi * rs + qj] = acc;
                A.val[mir0.x + qj * mir0.y + qi] = acc;
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
        L1 = L2;
        bm1 = bm2;
        r2 = r3;
    }
}

// Streaming, phase 1: apply the frame's mask changes and claim each touched block for the
// lowest candidate index (edited tet k, local pair s -> candidate 16 k + s).
// edited[k] = tet id | (new state << 31).
__global__ void k_stream_apply(const int32_t *__restrict__ edited, int64_t m,
                               const int32_t *__restrict__ tunit, const int32_t *__restrict__ cslot,
                               int32_t *__restrict__ ccode, uint8_t *__restrict__ mask,
                               int32_t *__restrict__ owner, unsigned long long *counters) {
    // one thread per (edited tet k, unit slot s): candidate 10 k + s
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        counters[1] = 0ull;
        counters[3] = 0ull;
    }
    if (i >= 10 * m) return;
    const uint32_t w = (uint32_t)edited[i / 10];
    const int32_t t = (int32_t)(w & 0x7fffffffu);
    const uint32_t on = w >> 31;
    const int s = (int)(i % 10);
    if (s == 0) mask[t] = (uint8_t)on;
    const int32_t slot = cslot[10 * (int64_t)t + s];
    ccode[slot] = (int32_t)(((uint32_t)ccode[slot] & ~CODE_ACTIVE) | (on << 31));
    atomicMin(&owner[tunit[10 * (int64_t)t + s]], (int32_t)i);
}

// Activity bits of all contributor codes from the mask (full rebuild with a new mask).
__global__ void k_mask_bits(int32_t *__restrict__ ccode, int64_t n, const uint8_t *__restrict__ mask) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t code = (uint32_t)ccode[k];
        const uint32_t on = mask[word_tet(code)] ? CODE_ACTIVE : 0u;
        ccode[k] = (int32_t)((code & ~CODE_ACTIVE) | on);
    }
}

// Streaming, phase 2: the owner of each touched block appends it to the fold list and
// releases the claim.  A non-owner reads either the owner's index or INT32_MAX, never its
// own index, so the release does not race with the ownership test.  The list order depends
// on scheduling; the values do not (each block is folded independently).
__device__ __forceinline__ void compact_one(int64_t i, int64_t n, const int32_t *__restrict__ edited,
                                            const int32_t *__restrict__ tunit,
                                            int32_t *__restrict__ owner, int32_t *__restrict__ list,
                                            unsigned long long *counters) {
    bool mine = false, diag = false;
    int32_t g = 0;
    if (i < n) {
        const int32_t t = (int32_t)((uint32_t)edited[i / 10] & 0x7fffffffu);
        const int s = (int)(i % 10);
        g = tunit[10 * (int64_t)t + s];
        diag = s < 4;
        mine = owner[g] == (int32_t)i;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, mine);
    const unsigned dball = __ballot_sync(0xffffffffu, mine && diag);
    unsigned long long base = 0;
    const int lane = threadIdx.x & 31;
    if (lane == 0 && ball) {
        base = atomicAdd(&counters[1], (unsigned long long)__popc(ball));
        // touched CSR entries: 9 for a diagonal unit, 18 (both blocks) for a pair
        atomicAdd(&counters[3], (unsigned long long)(18 * __popc(ball) - 9 * __popc(dball)));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (mine) {
        list[base + __popc(ball & ((1u << lane) - 1u))] = g;
        owner[g] = INT32_MAX;
    }
}

__global__ void k_stream_compact(const int32_t *__restrict__ edited, int64_t m,
                                 const int32_t *__restrict__ tunit, int32_t *__restrict__ owner,
                                 int32_t *__restrict__ list, unsigned long long *counters) {
    compact_one((int64_t)blockIdx.x * blockDim.x + threadIdx.x, 10 * m, edited, tunit, owner, list,
                counters);
}

// Device-count variants of the two streaming kernels for CUDA-graph replay: the number of
// edited tetrahedra is read from device memory, the grid is fixed and strides over it.
__global__ void k_stream_apply_dc(const int32_t *__restrict__ edited, const int64_t *__restrict__ m_dev,
                                  const int32_t *__restrict__ tunit, const int32_t *__restrict__ cslot,
                                  int32_t *__restrict__ ccode, uint8_t *__restrict__ mask,
                                  int32_t *__restrict__ owner, unsigned long long *counters) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[1] = 0ull;
        counters[3] = 0ull;
    }
    const int64_t n = 10 * *m_dev;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)edited[i / 10];
        const int32_t t = (int32_t)(w & 0x7fffffffu);
        const uint32_t on = w >> 31;
        const int s = (int)(i % 10);
        if (s == 0) mask[t] = (uint8_t)on;
        const int32_t slot = cslot[10 * (int64_t)t + s];
        ccode[slot] = (int32_t)(((uint32_t)ccode[slot] & ~CODE_ACTIVE) | (on << 31));
        atomicMin(&owner[tunit[10 * (int64_t)t + s]], (int32_t)i);
    }
}

__global__ void k_stream_compact_dc(const int32_t *__restrict__ edited, const int64_t *__restrict__ m_dev,
                                    const int32_t *__restrict__ tunit, int32_t *__restrict__ owner,
                                    int32_t *__restrict__ list, unsigned long long *counters) {
    const int64_t n = 10 * *m_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride)  // warp-uniform
        compact_one(i0 + threadIdx.x, n, edited, tunit, owner, list, counters);
}


}  // namespace


namespace {

FoldArgs fold_args(const Ctx *c) {
    return FoldArgs{c->bmeta, c->bmirror, c->ccode, c->Ke, c->val, c->eps};
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
                     int64_t max_items, cudaStream_t s) {
    const int threads = ENT_WARPS * 32;
    // one unit per 9 lanes (3 per warp) for the largest possible list, at most the resident CTAs
    const int grid = persistent_grid(c, (const void *)k_fold_entries, threads,
                                     (max_items + ENT_UNITS - 1) / ENT_UNITS * 32);
    k_fold_entries<<<grid, threads, 0, s>>>(fold_args(c), list, count);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

// Full rebuild: the flat entry-parallel fold over all tiles, with the context's CTA shape
// (block_threads 64, 128 or 256; blocks_per_sm 0 = occupancy maximum).
int launch_rebuild(Ctx *c, cudaStream_t s) {
    if (c->ntiles == 0) return STA_OK;
    const int threads = c->block_threads == 64 || c->block_threads == 256 ? c->block_threads : 128;
    const void *kern = threads == 64    ? (const void *)k_fold_flat<2>
                       : threads == 256 ? (const void *)k_fold_flat<8>
                                        : (const void *)k_fold_flat<4>;
    const int grid = persistent_grid(c, kern, threads, c->ntiles * 32, true);
    if (threads == 64)
        k_fold_flat<2><<<grid, threads, 0, s>>>(fold_args(c), c->ftile, c->ntiles);
    else if (threads == 256)
        k_fold_flat<8><<<grid, threads, 0, s>>>(fold_args(c), c->ftile, c->ntiles);
    else
        k_fold_flat<4><<<grid, threads, 0, s>>>(fold_args(c), c->ftile, c->ntiles);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_mask_bits(Ctx *c, cudaStream_t s) {
    if (c->T == 0) return STA_OK;
    const int64_t n = 10 * c->T;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = (int64_t)c->num_sms * 8;
    if (grid > cap) grid = cap;
    k_mask_bits<<<(unsigned)grid, 256, 0, s>>>(c->ccode, n, c->mask);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_stream(Ctx *c, int64_t m, cudaStream_t s) {
    if (m == 0) {
        STA_CUDA_TRY(cudaMemsetAsync(c->counters + 1, 0, 3 * sizeof(unsigned long long), s));
        return STA_OK;
    }
    const int threads = 256;
    const int64_t g2 = (10 * m + threads - 1) / threads;
    k_stream_apply<<<(unsigned)g2, threads, 0, s>>>(c->d_edited, m, c->tunit, c->cslot, c->ccode,
                                                    c->mask, c->owner, c->counters);
    k_stream_compact<<<(unsigned)g2, threads, 0, s>>>(c->d_edited, m, c->tunit, c->owner,
                                                      c->touched, c->counters);
    // the touched count is only known on the device: size the grid for the upper bound
    return launch_fold_list(c, c->touched, c->counters + 1, 10 * m, s);
}

// Streaming update for graph capture: edited list and its length in device memory, fixed grids
// sized for `cap` edited tetrahedra.
int launch_stream_devcount(Ctx *c, const int32_t *d_edited, const int64_t *d_m, int64_t cap,
                           cudaStream_t s) {
    const int threads = 256;
    int64_t g1 = (10 * cap + threads - 1) / threads, g2 = (10 * cap + threads - 1) / threads;
    const int64_t c1 = (int64_t)c->num_sms * 16, c2 = (int64_t)c->num_sms * 16;
    g1 = g1 < 1 ? 1 : (g1 > c1 ? c1 : g1);
    g2 = g2 < 1 ? 1 : (g2 > c2 ? c2 : g2);
    k_stream_apply_dc<<<(unsigned)g1, threads, 0, s>>>(d_edited, d_m, c->tunit, c->cslot, c->ccode,
                                                       c->mask, c->owner, c->counters);
    k_stream_compact_dc<<<(unsigned)g2, threads, 0, s>>>(d_edited, d_m, c->tunit, c->owner,
                                                         c->touched, c->counters);
    return launch_fold_list(c, c->touched, c->counters + 1, 10 * (cap > 0 ? cap : 1), s);
}

// Streaming update with caller-chosen scratch: the same three kernels as launch_stream, with
// the edited-tet list, the touched-block list and the counters at the given addresses (used
// by the allocation-free entry point; the touched count is copied to the context's counter
// afterwards so that sta_last_touched reports it).
int launch_stream_scratch(Ctx *c, int64_t m, const int32_t *d_edited, int32_t *touched,
                          unsigned long long *counters, cudaStream_t s) {
    if (m == 0) {
        STA_CUDA_TRY(cudaMemsetAsync(c->counters + 1, 0, 3 * sizeof(unsigned long long), s));
        return STA_OK;
    }
    const int threads = 256;
    const int64_t g2 = (10 * m + threads - 1) / threads;
    k_stream_apply<<<(unsigned)g2, threads, 0, s>>>(d_edited, m, c->tunit, c->cslot, c->ccode,
                                                    c->mask, c->owner, counters);
    k_stream_compact<<<(unsigned)g2, threads, 0, s>>>(d_edited, m, c->tunit, c->owner, touched,
                                                      counters);
    STA_TRY(launch_fold_list(c, touched, counters + 1, 10 * m, s));
    // touched units and touched entries, for sta_last_touched
    STA_CUDA_TRY(cudaMemcpyAsync(c->counters + 1, counters + 1, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s));
    STA_CUDA_TRY(cudaMemcpyAsync(c->counters + 3, counters + 3, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s));
    return STA_OK;
}

}  // namespace sta
