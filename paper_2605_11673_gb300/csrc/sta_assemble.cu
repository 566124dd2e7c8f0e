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

#include "sta_internal.cuh"

namespace sta {
namespace {

struct FoldArgs {
    const int32_t *__restrict__ cptr;
    const int32_t *__restrict__ ccode;
    const uint8_t *__restrict__ mask;
    const double *__restrict__ Ke;
    const int32_t *__restrict__ adj_ptr;
    const int32_t *__restrict__ adj;
    const int32_t *__restrict__ block_node;
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

// Diagonal block (a, a): every contributor uses its own diagonal 3x3 block (la == lb), whose
// 6 stored entries are folded; the 9 outputs mirror them (the element matrices are exactly
// symmetric, so (i, j) and (j, i) folds are identical).
__device__ __forceinline__ void fold_diag(const FoldArgs &A, int32_t c, int32_t c1,
                                          double *__restrict__ out, int rs) {
    double acc[6];
    for (; c < c1; ++c)
        if (A.mask[A.ccode[c] >> 4]) break;
    if (c == c1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = 0.0;
    } else {
        int32_t code = A.ccode[c];
        const double *r = A.Ke + (size_t)(code >> 4) * KE_STRIDE + 6 * ((code >> 2) & 3);
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = plus_zero(r[k]);
        for (++c; c < c1; ++c) {
            code = A.ccode[c];
            if (!A.mask[code >> 4]) continue;
            r = A.Ke + (size_t)(code >> 4) * KE_STRIDE + 6 * ((code >> 2) & 3);
            double v[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = r[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] += v[k];
        }
    }
    if (A.eps != 0.0) {
        acc[0] += A.eps;
        acc[3] += A.eps;
        acc[5] += A.eps;
    }
    out[0] = acc[0];          out[1] = acc[1];          out[2] = acc[2];
    out[rs + 0] = acc[1];     out[rs + 1] = acc[3];     out[rs + 2] = acc[4];
    out[2 * rs + 0] = acc[2]; out[2 * rs + 1] = acc[4]; out[2 * rs + 2] = acc[5];
}

// Off-diagonal block: contributor (t, la, lb) supplies K^(t)[3la+i][3lb+j], stored as the
// 9-run of pair (min, max) read row-major when la < lb and transposed otherwise.
__device__ __forceinline__ const double *off_run(const FoldArgs &A, int32_t code, int &si, int &sj) {
    int la = (code >> 2) & 3, lb = code & 3;
    int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
    si = la < lb ? 3 : 1;
    sj = la < lb ? 1 : 3;
    return A.Ke + (size_t)(code >> 4) * KE_STRIDE + 24 + 9 * pair_index(lo, hi);
}

__device__ __forceinline__ void fold_off(const FoldArgs &A, int32_t c, int32_t c1,
                                         double *__restrict__ out, int rs) {
    double acc[9];
    for (; c < c1; ++c)
        if (A.mask[A.ccode[c] >> 4]) break;
    if (c == c1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    } else {
        int si, sj;
        const double *r = off_run(A, A.ccode[c], si, sj);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[3 * i + j] = plus_zero(r[si * i + sj * j]);
        for (++c; c < c1; ++c) {
            int32_t code = A.ccode[c];
            if (!A.mask[code >> 4]) continue;
            r = off_run(A, code, si, sj);
            double v[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) v[3 * i + j] = r[si * i + sj * j];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] += v[k];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) out[i * rs + j] = acc[3 * i + j];
}

__device__ __forceinline__ void fold_block(const FoldArgs &A, int32_t g) {
    const int32_t a = A.block_node[g], b = A.adj[g];
    const int32_t s = A.adj_ptr[a], d = A.adj_ptr[a + 1] - s;
    double *out = A.val + (9 * (int64_t)s + 3 * (int64_t)(g - s));
    const int rs = 3 * d;
    if (a == b)
        fold_diag(A, A.cptr[g], A.cptr[g + 1], out, rs);
    else
        fold_off(A, A.cptr[g], A.cptr[g + 1], out, rs);
}

__global__ void __launch_bounds__(256) k_rebuild(FoldArgs A, int64_t nblocks) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x)
        fold_block(A, (int32_t)g);
}

// Streaming, phase 1: apply the frame's mask changes and claim each touched block for the
// lowest candidate index (edited tet k, local pair s -> candidate 16 k + s).
// edited[k] = tet id | (new state << 31).
__global__ void k_stream_apply(const int32_t *__restrict__ edited, int64_t m,
                               const int32_t *__restrict__ tblk, uint8_t *__restrict__ mask,
                               int32_t *__restrict__ owner, unsigned long long *counters) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) counters[1] = 0ull;
    if (k >= m) return;
    uint32_t w = (uint32_t)edited[k];
    int32_t t = (int32_t)(w & 0x7fffffffu);
    mask[t] = (uint8_t)(w >> 31);
#pragma unroll
    for (int s = 0; s < 16; ++s) atomicMin(&owner[tblk[16 * (int64_t)t + s]], (int32_t)(16 * k + s));
}

// Streaming, phase 2: the owner of each touched block re-folds it and releases the claim.
// A non-owner reads either the owner's index or INT32_MAX, never its own index, so the
// release does not race with the ownership test.
__global__ void __launch_bounds__(256)
k_stream_fold(FoldArgs A, const int32_t *__restrict__ edited, int64_t m,
              const int32_t *__restrict__ tblk, int32_t *__restrict__ owner,
              unsigned long long *counters) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool mine = false;
    int32_t g = 0;
    if (i < 16 * m) {
        int32_t t = (int32_t)((uint32_t)edited[i >> 4] & 0x7fffffffu);
        g = tblk[16 * (int64_t)t + (i & 15)];
        mine = owner[g] == (int32_t)i;
    }
    unsigned ball = __ballot_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(&counters[1], (unsigned long long)__popc(ball));
    if (mine) {
        fold_block(A, g);
        owner[g] = INT32_MAX;
    }
}

FoldArgs fold_args(const Ctx *c) {
    return FoldArgs{c->cptr, c->ccode, c->mask, c->Ke, c->adj_ptr, c->adj, c->block_node,
                    c->val, c->eps};
}

}  // namespace

int persistent_grid(const Ctx *c, const void *kernel, int threads, int64_t items) {
    int per_sm = c->blocks_per_sm;
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

int launch_rebuild(Ctx *c, cudaStream_t s) {
    if (c->nblocks == 0) return STA_OK;
    int threads = 256;
    int grid = persistent_grid(c, (const void *)k_rebuild, threads, c->nblocks);
    k_rebuild<<<grid, threads, 0, s>>>(fold_args(c), c->nblocks);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_stream(Ctx *c, int64_t m, cudaStream_t s) {
    if (m == 0) {
        STA_CUDA_TRY(cudaMemsetAsync(c->counters + 1, 0, sizeof(unsigned long long), s));
        return STA_OK;
    }
    int64_t g1 = (m + 255) / 256, g2 = (16 * m + 255) / 256;
    k_stream_apply<<<(unsigned)g1, 256, 0, s>>>(c->d_edited, m, c->tblk, c->mask, c->owner,
                                                c->counters);
    k_stream_fold<<<(unsigned)g2, 256, 0, s>>>(fold_args(c), c->d_edited, m, c->tblk, c->owner,
                                               c->counters);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace sta
