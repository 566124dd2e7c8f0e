// Fold kernels: full rebuild (a2) and streaming update (a3).
//
// Both evaluate, for a node-pair block (a, b) of the superset pattern, the 9 CSR values
//   A[3a+i][3b+j] = fold_{tau active, ascending id} K^(tau)[3 la + i][3 lb + j]   (+ eps)
// i.e. Eq. 8 of STA-FEM restricted to one block, with the fold starting at +0.0 and eps
// added afterwards on the diagonal.  The streaming pass (Sec. 3.2, Algorithm 1; the
// local_recompute policy of Sec. 3.5) calls the same device function on the blocks touched
// by the frame's edits only, so its values are bit-identical to the rebuild's.
//
// No atomics touch values: each block is folded by exactly one thread, and the summation
// order is the order of the contributor list (ascending tetrahedron id), independent of the
// launch configuration.
#include <climits>

#include "softfloat.cuh"
#include "sta_internal.cuh"

// Number of the 9 accumulators of a fold step whose additions run on the integer pipes
// (int_add, bit-identical to the FP64 add); the rest use the FP64 pipe.  Build-time tuning;
// measured slower on the fold (its loop is latency- rather than FP64-issue-bound), so 0.
#ifndef STA_INT_ADDS
#define STA_INT_ADDS 0
#endif

namespace sta {
namespace {

struct FoldArgs {
    const int4 *__restrict__ bmeta;     // per unit: value offset of (a,b), rs_a << 1 | diag, c0, c1
    const int2 *__restrict__ bmirror;   // per unit: value offset of (b,a), rs_b
    const int32_t *__restrict__ ccode;  // contributor codes, bit 31 = active
    const double *__restrict__ Ke;
    double *__restrict__ val;
    double eps;
};

// +0.0 + v without an FP64 operation: identical except that -0.0 becomes +0.0.
__device__ __forceinline__ double plus_zero(double v) {
    long long bits = __double_as_longlong(v);
    return __longlong_as_double(bits == (long long)0x8000000000000000ULL ? 0LL : bits);
}

__device__ __forceinline__ int pair_index(int a, int b) {  // a < b
    return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// The operands one contributor supplies to a fold unit (node pair a <= b; la, lb the local
// indices of a and b in the contributing tetrahedron), read with 16-byte loads:
//   diagonal unit (la == lb): the 6-run of (la, la): v[0..5] = (0,0) (0,1) (0,2) (1,1) (1,2)
//                              (2,2); the mirrored entries (j, i) fold the same operands;
//   off-diagonal, la < lb:     the 9-run of (la, lb), row-major: v[3i+j] = K[3la+i][3lb+j];
//   off-diagonal, la > lb:     the 9-run of (lb, la), transposed.
// The mirror block (b, a) folds exactly the same operand sequence (K is stored exactly
// symmetric), so one fold per unit gives both blocks' values bit for bit.
__device__ __forceinline__ void load_contrib(const FoldArgs &A, int32_t code, double v[9]) {
    const int la = (code >> 2) & 3, lb = code & 3;
    const double *rec = A.Ke + (size_t)code_tet(code) * KE_STRIDE;
    if (la == lb) {
        const double2 *r = reinterpret_cast<const double2 *>(rec + 6 * la);
        const double2 x = __ldg(r), y = __ldg(r + 1), z = __ldg(r + 2);
        v[0] = x.x; v[1] = x.y; v[2] = y.x;
        v[3] = y.y; v[4] = z.x; v[5] = z.y;
        v[6] = 0.0; v[7] = 0.0; v[8] = 0.0;
    } else {
        const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
        const double2 *r = reinterpret_cast<const double2 *>(rec + 24 + 10 * pair_index(lo, hi));
        const double2 p0 = __ldg(r), p1 = __ldg(r + 1), p2 = __ldg(r + 2), p3 = __ldg(r + 3),
                      p4 = __ldg(r + 4);
        const double w[9] = {p0.x, p0.y, p1.x, p1.y, p2.x, p2.y, p3.x, p3.y, p4.x};
        const bool tr = la > lb;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) v[3 * i + j] = tr ? w[3 * j + i] : w[3 * i + j];
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

// Lockstep fold.  On GB300 a warp-wide FP64 instruction costs the same however many lanes
// are active, and FP64 issue is the scarcest resource, so every FP64 add instruction should
// carry 32 useful lanes.  Each warp works in two phases over its share of the blocks:
//
//  stage: blocks are taken in order; the active contributor codes of each block are
//         compacted, in list order, into the warp's shared buffer.  Blocks with no active
//         contributor are written (+0.0) and blocks with one are written (+0.0 + c) right
//         away, with no FP64 operation.  Integer and load work only.
//  fold:  lanes claim staged blocks in order as they become free.  A claim loads the
//         operands of the block's first contribution into v and of its second into the
//         accumulators; the next iteration forms (+0.0 + c1) + c2, and every later iteration
//         adds one more contribution while the loads of the following one are in flight.
//         Every iteration of a busy lane is one useful 9-wide FP64 add.
//
// Items are handed out in chunks of 32: warp w owns chunks w, w + W, w + 2W, ... (W warps in
// the grid).  MODE 0: item = block id (whole pattern) -- a chunk is 32 consecutive blocks
// whose codes are contiguous, staged with coalesced windows and ballots; MODE 1: item
// indexes a list of block ids whose length is read from device memory (streaming), staged
// one block per lane.
constexpr int FOLD_WARPS = 4;       // default warps per CTA (2, 4 or 8 selectable)
constexpr int STAGE_BLOCKS = 192;   // staged blocks per warp
constexpr int STAGE_CODES = 1280;   // staged active codes per warp (>= contributors of any block)
constexpr int STAGE_WIN = 8;        // 32-code windows of one staging round held in registers
constexpr int LONG_BLOCK = 8;       // staged blocks with this many contributors are claimed first
constexpr size_t FOLD_WARP_SMEM = sizeof(int4) * STAGE_BLOCKS + sizeof(int2) * STAGE_BLOCKS +
                                  sizeof(int32_t) * STAGE_CODES;

__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// bits of positions [0, n) of a 32-bit window (n clamped to [0, 32])
__device__ __forceinline__ unsigned below(int n) {
    return n <= 0 ? 0u : (n >= 32 ? 0xffffffffu : ((1u << n) - 1u));
}

// A block with at most one active contributor: written directly (+0.0, or +0.0 + c).
__device__ __forceinline__ void write_small_block(const FoldArgs &A, const int4 bm, int2 mir,
                                                  int cnt, int32_t code) {
    double acc[9];
    if (cnt == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    } else {
        load_contrib(A, code, acc);
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = plus_zero(acc[q]);
    }
    write_block(A, unit_out(A, bm, mir), acc);
}

template <int MODE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_fold(FoldArgs A, const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
       int64_t nitems_static) {
    // per warp: STAGE_BLOCKS int4 block records, then STAGE_CODES int32 codes (dynamic)
    extern __shared__ int4 fold_smem[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 *sblk = fold_smem + (size_t)wid * (FOLD_WARP_SMEM / sizeof(int4));
    int2 *smir = reinterpret_cast<int2 *>(sblk + STAGE_BLOCKS);
    int32_t *scode = reinterpret_cast<int32_t *>(smir + STAGE_BLOCKS);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = MODE == 0 ? nitems_static : (int64_t)*count;
    const unsigned lt_mask = (1u << lane) - 1u;

    int64_t p_base = 0;  // warp-uniform position in this warp's item sequence
    bool more = true;
    while (more) {
        // ------------------------------------------------------------ stage
        int nlong = 0, nshort = 0, nc = 0;
        while (nlong + nshort + 32 <= STAGE_BLOCKS) {
            if (MODE == 0) {
                // the rest of the current chunk: consecutive blocks, contiguous codes
                const int off = (int)(p_base & 31);
                const int64_t chunk_first = ((p_base >> 5) * nwarps + warp) * 32;
                const int64_t g = chunk_first + off + lane;
                const bool valid = lane < 32 - off && g < nitems;
                const unsigned validm = __ballot_sync(FULL, valid);
                if (!validm) {
                    more = false;
                    break;
                }
                const int nv = __popc(validm);  // valid lanes form a prefix
                int4 bm = make_int4(0, 0, 0, 0);
                int2 mir = make_int2(0, 0);
                if (valid) {
                    bm = __ldg(A.bmeta + g);
                    mir = __ldg(A.bmirror + g);
                }
                const int32_t r0 = __shfl_sync(FULL, bm.z, 0);
                const int32_t r1 = __shfl_sync(FULL, bm.w, nv - 1);
                const int nwin = (r1 - r0 + 31) >> 5;
                // all windows' code loads issued before any is used
                int32_t cw[STAGE_WIN];
#pragma unroll
                for (int w = 0; w < STAGE_WIN; ++w) {
                    const int32_t c = r0 + 32 * w + lane;
                    cw[w] = (w < nwin && c < r1) ? __ldg(A.ccode + c) : 0;
                }
                // pass 1: active codes before each block start (lo) and in the whole range
                int lo = 0, total = 0;
#pragma unroll
                for (int w = 0; w < STAGE_WIN; ++w) {
                    if (w < nwin) {
                        const unsigned m = __ballot_sync(FULL, cw[w] < 0);
                        lo += __popc(m & below(bm.z - (r0 + 32 * w)));
                        total += __popc(m);
                    }
                }
                for (int w = STAGE_WIN; w < nwin; ++w) {
                    const int32_t c = r0 + 32 * w + lane;
                    const unsigned m = __ballot_sync(FULL, c < r1 && __ldg(A.ccode + c) < 0);
                    lo += __popc(m & below(bm.z - (r0 + 32 * w)));
                    total += __popc(m);
                }
                int hi = __shfl_down_sync(FULL, lo, 1);
                if (lane == nv - 1) hi = total;
                const int cnt = valid ? hi - lo : 0;
                // blocks that fit: lo + cnt within the free code space (a prefix of lanes)
                const bool fits = valid && nc + hi <= STAGE_CODES;
                const unsigned fitm = __ballot_sync(FULL, fits);
                const int nfit = __popc(fitm);
                if (nfit > 0) {
                    // pass 2: compact the active codes of the fitting blocks, in list order
                    const int32_t f1 = __shfl_sync(FULL, bm.w, nfit - 1);
                    int run = nc;
#pragma unroll
                    for (int w = 0; w < STAGE_WIN; ++w) {
                        if (w < nwin) {
                            const int32_t c = r0 + 32 * w + lane;
                            const bool act = c < f1 && cw[w] < 0;
                            const unsigned m = __ballot_sync(FULL, act);
                            if (act) scode[run + __popc(m & lt_mask)] = cw[w];
                            run += __popc(m);
                        }
                    }
                    for (int w = STAGE_WIN; w < nwin; ++w) {
                        const int32_t c = r0 + 32 * w + lane;
                        int32_t code = 0;
                        const bool act = c < f1 && (code = __ldg(A.ccode + c)) < 0;
                        const unsigned m = __ballot_sync(FULL, act);
                        if (act) scode[run + __popc(m & lt_mask)] = code;
                        run += __popc(m);
                    }
                    __syncwarp();
                    // long blocks fill the staging list from the front, short ones from the
                    // back: claims take long blocks first (longest-processing-time order)
                    const unsigned longm = __ballot_sync(FULL, fits && cnt >= LONG_BLOCK);
                    const unsigned shortm = __ballot_sync(FULL, fits && cnt >= 2 && cnt < LONG_BLOCK);
                    if (fits) {
                        if (cnt < 2) {
                            write_small_block(A, bm, mir, cnt, cnt ? scode[nc + lo] : 0);
                        } else {
                            const int at = cnt >= LONG_BLOCK
                                               ? nlong + __popc(longm & lt_mask)
                                               : STAGE_BLOCKS - 1 - nshort - __popc(shortm & lt_mask);
                            sblk[at] = make_int4(bm.x, bm.y, nc + lo, cnt);
                            smir[at] = mir;
                        }
                    }
                    nlong += __popc(longm);
                    nshort += __popc(shortm);
                    nc += __shfl_sync(FULL, hi, nfit - 1);
                    p_base += nfit;
                }
                if (nfit < nv) break;  // code space full: fold, then continue this chunk
            } else {
                const int64_t p = p_base + lane;
                const int64_t item = ((p >> 5) * nwarps + warp) * 32 + (p & 31);
                const bool valid = item < nitems;
                int4 bm = make_int4(0, 0, 0, 0);
                int2 mir = make_int2(0, 0);
                int cnt = 0;
                if (valid) {
                    const int32_t u = __ldg(list + item);
                    bm = __ldg(A.bmeta + u);
                    mir = __ldg(A.bmirror + u);
                    for (int32_t c = bm.z; c < bm.w; ++c) cnt += __ldg(A.ccode + c) < 0;
                }
                const int inc = warp_inclusive_scan(cnt, lane);
                const bool fits = valid && nc + inc <= STAGE_CODES;
                const unsigned fitm = __ballot_sync(FULL, fits);
                const unsigned longm = __ballot_sync(FULL, fits && cnt >= LONG_BLOCK);
                const unsigned shortm = __ballot_sync(FULL, fits && cnt >= 2 && cnt < LONG_BLOCK);
                if (fits) {
                    const int at = nc + inc - cnt;
                    int j = 0;
                    for (int32_t c = bm.z; c < bm.w; ++c) {
                        const int32_t code = __ldg(A.ccode + c);
                        if (code < 0) scode[at + j++] = code;
                    }
                    if (cnt < 2) {
                        write_small_block(A, bm, mir, cnt, cnt ? scode[at] : 0);
                    } else {
                        const int idx = cnt >= LONG_BLOCK
                                            ? nlong + __popc(longm & lt_mask)
                                            : STAGE_BLOCKS - 1 - nshort - __popc(shortm & lt_mask);
                        sblk[idx] = make_int4(bm.x, bm.y, at, cnt);
                        smir[idx] = mir;
                    }
                }
                const int nfit = __popc(fitm);  // fitting lanes form a prefix
                if (nfit > 0) nc += __shfl_sync(FULL, inc, nfit - 1);
                nlong += __popc(longm);
                nshort += __popc(shortm);
                p_base += nfit;
                if (nfit < 32) {
                    more = __any_sync(FULL, valid);
                    break;
                }
            }
        }
        __syncwarp();
        // ------------------------------------------------------------ fold
        int next_blk = 0;  // warp-uniform: staged blocks claimed so far
        bool busy = false;
        int k = 0, kend = 0;
        BlockOut o{nullptr, nullptr, 0, 0, false};
        // acc: accumulators; v: operands of the next contribution to add; w: of the one after
        // (two contributions in flight per lane).  Right after a claim, acc holds the raw
        // operands of contribution 2 and v those of contribution 1 (fresh).
        double acc[9], v[9], w[9];
        bool fresh = false, have_w = false;
        // Claims come right after a block is written, so the operand loads of a newly
        // claimed block are in flight for a whole iteration, like every other prefetch.
        auto claim_blocks = [&]() {
            const unsigned claim = __ballot_sync(FULL, !busy);
            if (!busy) {
                const int b = next_blk + __popc(claim & lt_mask);
                if (b < nlong + nshort) {
                    const int at = b < nlong ? b : STAGE_BLOCKS - 1 - (b - nlong);
                    const int4 sb = sblk[at];
                    o = unit_out(A, sb, smir[at]);
                    k = sb.z;
                    kend = sb.z + sb.w;
                    load_contrib(A, scode[k], v);
                    load_contrib(A, scode[k + 1], acc);
                    k += 2;
                    have_w = k < kend;
                    if (have_w) load_contrib(A, scode[k++], w);
                    busy = true;
                    fresh = true;
                }
            }
            next_blk += __popc(claim);
        };
        claim_blocks();
        while (__any_sync(FULL, busy)) {
            if (busy) {
                if (fresh) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = plus_zero(v[q]);
                    fresh = false;
                }
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    acc[q] = q < STA_INT_ADDS ? int_add(acc[q], v[q]) : acc[q] + v[q];
                if (!o.diag) {  // a diagonal unit folds 6 entries
#pragma unroll
                    for (int q = 6; q < 9; ++q)
                        acc[q] = q < STA_INT_ADDS ? int_add(acc[q], v[q]) : acc[q] + v[q];
                }
                if (have_w) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = w[q];
                    have_w = k < kend;
                    if (have_w) load_contrib(A, scode[k++], w);
                } else {
                    write_block(A, o, acc);
                    busy = false;
                }
            }
            if (__any_sync(FULL, !busy)) claim_blocks();
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Fold of a list of blocks (streaming).  A frame touches few blocks (thousands to tens of
// thousands), so here latency rules, not FP64 issue: each warp takes up to 32 listed blocks
// per round (one per lane), counts their active contributors with batched code loads,
// compacts the active codes into its shared memory and copies their operand runs there with
// asynchronous 16-byte copies (cp.async, all in flight together), then folds the blocks from
// shared memory, lanes claiming the staged blocks longest first.  Same fold order and
// operations as k_fold, so the values are the same bits.
// ------------------------------------------------------------------------------------------
constexpr int LIST_WARPS = 4;
constexpr int LIST_BLOCKS = 64;     // staged blocks per warp
constexpr int LIST_CONTRIB = 256;   // staged operand runs per warp
constexpr int LIST_RUN = 10;        // doubles per staged run (80 bytes, 16-byte aligned)
constexpr size_t LIST_WARP_SMEM = sizeof(int4) * LIST_BLOCKS + sizeof(int2) * LIST_BLOCKS +
                                  sizeof(int32_t) * LIST_CONTRIB +
                                  sizeof(double) * LIST_RUN * LIST_CONTRIB;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// copy a contribution's operand run (48 or 80 bytes) into shared memory
__device__ __forceinline__ void stage_run(const FoldArgs &A, int32_t code, double *dst) {
    const int la = (code >> 2) & 3, lb = code & 3;
    const double *rec = A.Ke + (size_t)code_tet(code) * KE_STRIDE;
    if (la == lb) {
        const double *src = rec + 6 * la;
#pragma unroll
        for (int q = 0; q < 3; ++q) cp_async16(dst + 2 * q, src + 2 * q);
    } else {
        const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
        const double *src = rec + 24 + 10 * pair_index(lo, hi);
#pragma unroll
        for (int q = 0; q < 5; ++q) cp_async16(dst + 2 * q, src + 2 * q);
    }
}

// the 9 operands of a staged run (same three layouts as load_contrib)
__device__ __forceinline__ void smem_operands(const double *r, int32_t code, double v[9]) {
    const int la = (code >> 2) & 3, lb = code & 3;
    const double2 *p = reinterpret_cast<const double2 *>(r);
    const double2 p0 = p[0], p1 = p[1], p2 = p[2];
    if (la == lb) {
        v[0] = p0.x; v[1] = p0.y; v[2] = p1.x;
        v[3] = p1.y; v[4] = p2.x; v[5] = p2.y;
        v[6] = 0.0; v[7] = 0.0; v[8] = 0.0;
    } else {
        const double2 p3 = p[3], p4 = p[4];
        const double w[9] = {p0.x, p0.y, p1.x, p1.y, p2.x, p2.y, p3.x, p3.y, p4.x};
        const bool tr = la > lb;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) v[3 * i + j] = tr ? w[3 * j + i] : w[3 * i + j];
    }
}

// One lane folds a whole unit from global memory (units larger than the shared buffers).
__device__ void fold_direct(const FoldArgs &A, const int4 bm, const int2 mir) {
    double acc[9], v[9];
    int32_t c = next_active(A, bm.z, bm.w);
    if (c == bm.w) {
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    } else {
        load_contrib(A, __ldg(A.ccode + c), acc);
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = plus_zero(acc[q]);
        for (c = next_active(A, c + 1, bm.w); c < bm.w; c = next_active(A, c + 1, bm.w)) {
            load_contrib(A, __ldg(A.ccode + c), v);
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] += v[q];  // (diagonal: entries 6..8 unused)
        }
    }
    write_block(A, unit_out(A, bm, mir), acc);
}

__global__ void __launch_bounds__(LIST_WARPS * 32)
k_fold_list(FoldArgs A, const int32_t *__restrict__ list, const unsigned long long *__restrict__ count) {
    extern __shared__ int4 list_smem[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 *sblk = list_smem + (size_t)wid * (LIST_WARP_SMEM / sizeof(int4));
    int2 *smir = reinterpret_cast<int2 *>(sblk + LIST_BLOCKS);
    int32_t *scode = reinterpret_cast<int32_t *>(smir + LIST_BLOCKS);
    double *sop = reinterpret_cast<double *>(scode + LIST_CONTRIB);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = (int64_t)*count;
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t p_base = 0;
    bool more = true;
    while (more) {
        // ------------------------------------------------------------ stage
        int nlong = 0, nshort = 0, nc = 0;
        while (true) {
            const int nb = nlong + nshort;
            const int64_t p = p_base + lane;
            const int64_t item = ((p >> 5) * nwarps + warp) * 32 + (p & 31);
            const bool valid = item < nitems;
            int4 bm = make_int4(0, 0, 0, 0);
            int2 mir = make_int2(0, 0);
            if (valid) {
                const int32_t u = __ldg(list + item);
                bm = __ldg(A.bmeta + u);
                mir = __ldg(A.bmirror + u);
            }
            const unsigned validm = __ballot_sync(FULL, valid);
            if (!validm) {
                more = false;
                break;
            }
            const int nv = __popc(validm);
            int cnt = 0;
            for (int32_t c0 = bm.z; c0 < bm.w; c0 += 8) {  // 8 code loads in flight
                int32_t cb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) cb[u] = c0 + u < bm.w ? __ldg(A.ccode + c0 + u) : 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) cnt += cb[u] < 0;
            }
            const int hi = warp_inclusive_scan(cnt, lane), lo = hi - cnt;
            const unsigned nzm = __ballot_sync(FULL, valid && cnt > 0);
            const int blk_upto = nb + __popc(nzm & (lt_mask | (1u << lane)));
            const bool fits = valid && nc + hi <= LIST_CONTRIB && blk_upto <= LIST_BLOCKS;
            const unsigned fitm = __ballot_sync(FULL, fits);
            const int nfit = __popc(fitm);
            if (nfit == 0) {
                if (nc == 0 && nb == 0) {  // one block larger than the buffers
                    if (lane == 0) fold_direct(A, bm, mir);
                    p_base += 1;
                    continue;
                }
                break;
            }
            if (fits) {
                int j = nc + lo;
                for (int32_t c = bm.z; c < bm.w; ++c) {
                    const int32_t code = __ldg(A.ccode + c);
                    if (code < 0) {
                        scode[j] = code;
                        stage_run(A, code, sop + LIST_RUN * j);
                        ++j;
                    }
                }
            }
            const unsigned longm = __ballot_sync(FULL, fits && cnt >= LONG_BLOCK);
            const unsigned shortm = __ballot_sync(FULL, fits && cnt > 0 && cnt < LONG_BLOCK);
            if (fits) {
                if (cnt == 0) {
                    double acc[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) acc[q] = 0.0;
                    write_block(A, unit_out(A, bm, mir), acc);
                } else {
                    const int at = cnt >= LONG_BLOCK ? nlong + __popc(longm & lt_mask)
                                                     : LIST_BLOCKS - 1 - nshort - __popc(shortm & lt_mask);
                    sblk[at] = make_int4(bm.x, bm.y, nc + lo, cnt);
                    smir[at] = mir;
                }
            }
            nlong += __popc(longm);
            nshort += __popc(shortm);
            nc += __shfl_sync(FULL, hi, nfit - 1);
            p_base += nfit;
            if (nfit < nv) break;
        }
        cp_async_wait_all();
        __syncwarp();
        // ------------------------------------------------------------ fold
        const int nstaged = nlong + nshort;
        int next_blk = 0;
        bool busy = false, parked = false;
        int k = 0, kend = 0;
        BlockOut o{nullptr, nullptr, 0, 0, false};
        double acc[9], v[9];
        auto claim_blocks = [&]() {
            while (true) {
                const unsigned need = __ballot_sync(FULL, !busy && !parked);
                if (!need) break;
                const int b = next_blk + __popc(need & lt_mask);
                next_blk += __popc(need);
                if (!busy && !parked) {
                    if (b >= nstaged) {
                        parked = true;
                    } else {
                        const int at = b < nlong ? b : LIST_BLOCKS - 1 - (b - nlong);
                        const int4 sb = sblk[at];
                        o = unit_out(A, sb, smir[at]);
                        k = sb.z;
                        kend = sb.z + sb.w;
                        smem_operands(sop + LIST_RUN * k, scode[k], v);
#pragma unroll
                        for (int q = 0; q < 9; ++q) acc[q] = plus_zero(v[q]);
                        ++k;
                        if (k == kend) {
                            write_block(A, o, acc);
                        } else {
                            smem_operands(sop + LIST_RUN * k, scode[k], v);
                            busy = true;
                        }
                    }
                }
            }
        };
        claim_blocks();
        while (__any_sync(FULL, busy)) {
            if (busy) {
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[q] += v[q];
                if (!o.diag) {
#pragma unroll
                    for (int q = 6; q < 9; ++q) acc[q] += v[q];
                }
                ++k;
                if (k < kend) {
                    smem_operands(sop + LIST_RUN * k, scode[k], v);
                } else {
                    write_block(A, o, acc);
                    busy = false;
                }
            }
            if (__any_sync(FULL, !busy && !parked)) claim_blocks();
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Entry-parallel fold of a list of units (streaming).  A frame's touched list is short and its
// longest folds (diagonal units, ~24 contributions) set the latency, so here each lane folds ONE
// matrix entry: a warp takes 3 listed units, lanes 9g .. 9g+8 fold the 9 entries (i, j) of
// unit g (6 of them for a diagonal unit), and one FP64 instruction per step advances all 27
// folds.  The unit's active codes are compacted (in list order) into shared memory first; each
// step then loads one operand per lane (4 steps of loads in flight).  Operands, order and
// operations are those of k_fold, so the values are the same bits.
// ------------------------------------------------------------------------------------------
constexpr int ENT_UNITS = 3;    // units per warp round (27 lanes)
constexpr int ENT_CAP = 96;     // active contributions staged per unit; larger units fold directly
constexpr int ENT_WARPS = 4;

template <int MODE>  // 0: units 0 .. nitems_static-1; 1: the listed units (count on the device)
__global__ void __launch_bounds__(ENT_WARPS * 32)
k_fold_entries(FoldArgs A, const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
               int64_t nitems_static) {
    __shared__ int32_t scode_all[ENT_WARPS][ENT_UNITS][ENT_CAP];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / 9, q = lane % 9;  // g == 3: lanes 27..31 idle
    const int qi = q / 3, qj = q % 3;
    int32_t *scode = scode_all[wid][g < ENT_UNITS ? g : 0];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = MODE == 0 ? nitems_static : (int64_t)*count;
    for (int64_t base = warp * ENT_UNITS; base < nitems; base += nwarps * ENT_UNITS) {  // warp-uniform
        const int64_t item = base + g;
        const bool valid = g < ENT_UNITS && item < nitems;
        int4 bm = make_int4(0, 0, 0, 0);
        int2 mir = make_int2(0, 0);
        if (valid) {
            const int32_t u = MODE == 0 ? (int32_t)item : __ldg(list + item);
            bm = __ldg(A.bmeta + u);
            mir = __ldg(A.bmirror + u);
        }
        // compact the unit's active codes, 9 lanes striding over its contributor list
        int nact = 0;
        const int span = valid ? bm.w - bm.z : 0;
        const int max_span = __reduce_max_sync(FULL, span);
        for (int c0 = 0; c0 < max_span; c0 += 9) {
            const int c = c0 + q;
            const int32_t code = (valid && c < span) ? __ldg(A.ccode + bm.z + c) : 0;
            const unsigned m = __ballot_sync(FULL, code < 0);
            const unsigned gm = (m >> (9 * g)) & 0x1ffu;
            const int pos = nact + __popc(gm & ((1u << q) - 1u));
            if (code < 0 && pos < ENT_CAP) scode[pos] = code;
            nact += __popc(gm);
        }
        __syncwarp();
        const bool big = valid && nact > ENT_CAP;
        if (big && q == 0) fold_direct(A, bm, mir);  // rare: more active contributions than staged
        const int n = valid && !big ? nact : 0;
        const bool diag = (bm.y & 1) != 0;
        const bool mine = n > 0 && (!diag || q < 6);  // a diagonal unit folds 6 entries
        double acc = 0.0;
        const int maxn = __reduce_max_sync(FULL, n);
        for (int j0 = 0; j0 < maxn; j0 += 4) {
            double v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                v[t] = 0.0;
                const int j = j0 + t;
                if (mine && j < n) {
                    const int32_t code = scode[j];
                    const int la = (code >> 2) & 3, lb = code & 3;
                    const double *rec = A.Ke + (size_t)code_tet(code) * KE_STRIDE;
                    if (la == lb) {
                        v[t] = __ldg(rec + 6 * la + q);
                    } else {
                        const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
                        v[t] = __ldg(rec + 24 + 10 * pair_index(lo, hi) + (la < lb ? q : 3 * qj + qi));
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = j0 + t;
                if (mine && j < n) acc = j == 0 ? plus_zero(v[t]) : acc + v[t];
            }
        }
        if (valid && !big) {
            if (diag) {
                if (q < 6) {
                    // 6-run entry q = (i, j), i <= j
                    const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
                    double a = acc;
                    if (i == j && A.eps != 0.0) a += A.eps;
                    double *out = A.val + bm.x;
                    const int rs = bm.y >> 1;
                    out[i * rs + j] = a;
                    if (i != j) out[j * rs + i] = a;
                }
            } else {
                A.val[bm.x + qi * (bm.y >> 1) + qj] = acc;
                A.val[mir.x + qj * mir.y + qi] = acc;
            }
        }
        __syncwarp();
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
        const uint32_t on = mask[code_tet((int32_t)code)] ? CODE_ACTIVE : 0u;
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

int max_block_contributors() { return STAGE_CODES; }

namespace {

FoldArgs fold_args(const Ctx *c) {
    return FoldArgs{c->bmeta, c->bmirror, c->ccode, c->Ke, c->val, c->eps};
}

}  // namespace

int persistent_grid(const Ctx *c, const void *kernel, int threads, int64_t items, size_t smem) {
    int per_sm = c->blocks_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int64_t need = (items + threads - 1) / threads;
    int64_t cap = (int64_t)per_sm * c->num_sms;
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

// Launch the fold with the context's CTA shape (block_threads 64, 128 or 256).
template <int MODE>
int launch_fold(Ctx *c, const int32_t *list, const unsigned long long *count, int64_t nitems,
                int64_t max_items, cudaStream_t s) {
    const int threads = c->block_threads == 64 || c->block_threads == 256 ? c->block_threads : 128;
    const void *kern = threads == 64    ? (const void *)k_fold<MODE, 2>
                       : threads == 256 ? (const void *)k_fold<MODE, 8>
                                        : (const void *)k_fold<MODE, 4>;
    const size_t smem = FOLD_WARP_SMEM * (threads / 32);
    const int grid = persistent_grid(c, kern, threads, max_items, smem);
    if (threads == 64)
        k_fold<MODE, 2><<<grid, threads, smem, s>>>(fold_args(c), list, count, nitems);
    else if (threads == 256)
        k_fold<MODE, 8><<<grid, threads, smem, s>>>(fold_args(c), list, count, nitems);
    else
        k_fold<MODE, 4><<<grid, threads, smem, s>>>(fold_args(c), list, count, nitems);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

// Dynamic shared memory limits of the fold instantiations (set once per context creation,
// outside any stream capture).
int init_fold_attributes() {
    const void *k[6] = {(const void *)k_fold<0, 2>, (const void *)k_fold<0, 4>,
                        (const void *)k_fold<0, 8>, (const void *)k_fold<1, 2>,
                        (const void *)k_fold<1, 4>, (const void *)k_fold<1, 8>};
    const int w[6] = {2, 4, 8, 2, 4, 8};
    for (int i = 0; i < 6; ++i)
        STA_CUDA_TRY(cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(FOLD_WARP_SMEM * w[i])));
    STA_CUDA_TRY(cudaFuncSetAttribute((const void *)k_fold_list,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(LIST_WARP_SMEM * LIST_WARPS)));
    return STA_OK;
}

int launch_fold_list(Ctx *c, const int32_t *list, const unsigned long long *count,
                     int64_t max_items, cudaStream_t s) {
    const int threads = ENT_WARPS * 32;
    // one unit per 9 lanes (3 per warp) for the largest possible list, at most the resident CTAs
    const int grid = persistent_grid(c, (const void *)k_fold_entries<1>, threads,
                                     (max_items + ENT_UNITS - 1) / ENT_UNITS * 32);
    k_fold_entries<1><<<grid, threads, 0, s>>>(fold_args(c), list, count, 0);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

#ifndef STA_REBUILD_ENTRIES
#define STA_REBUILD_ENTRIES 0
#endif

int launch_rebuild(Ctx *c, cudaStream_t s) {
    if (c->nunits == 0) return STA_OK;
    if (STA_REBUILD_ENTRIES) {
        const int threads = ENT_WARPS * 32;
        const int grid = persistent_grid(c, (const void *)k_fold_entries<0>, threads,
                                         (c->nunits + ENT_UNITS - 1) / ENT_UNITS * 32);
        k_fold_entries<0><<<grid, threads, 0, s>>>(fold_args(c), nullptr, nullptr, c->nunits);
        STA_CUDA_TRY(cudaGetLastError());
        return STA_OK;
    }
    return launch_fold<0>(c, nullptr, nullptr, c->nunits, c->nunits, s);
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
