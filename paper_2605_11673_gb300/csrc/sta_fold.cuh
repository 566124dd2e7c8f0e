// Fold kernels: the full rebuild and the streaming update.
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
//
// This header holds what both folds share: the arguments, the +0.0 start, the operand runs
// of one contributor, the block writer and the one-lane fold of a whole unit.
#pragma once

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
// 2^x for x in [-1022, 1023], exact (the fixed-point scale of an entry)
__device__ __forceinline__ double pow2i(int x) {
    return __longlong_as_double((long long)(x + 1023) << 52);
}

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

inline FoldArgs fold_args(const Ctx *c) {
    return FoldArgs{c->bmeta, c->bmirror, c->ccode, c->Ke, c->val, c->eps};
}

}  // namespace
}  // namespace sta
