// Exact additive streaming in fixed point (policy STA_POLICY_FIXED).
//
// The paper's streaming_update (Sec. 3.4, Sec. 3.5) adds or subtracts the element
// contributions of the edited tetrahedra, O(|Delta|), and is exact only up to rounding in
// floating point.  Here every CSR entry k has a fixed binary exponent e_k, every contribution
// c to k is quantised once to q = c 2^-e_k rounded to the nearest integer (ties to even), and
// the context keeps the exact integer sum S_k over the active contributors.  A frame adds and
// subtracts the q of its edited tetrahedra with integer atomics -- integer addition is
// associative, so the order does not matter -- and converts the touched entries once:
// val_k = double(S_k) 2^e_k (+ eps on the diagonal).  The result is bit-identical to the fixed
// point rebuild (the integer sum over the active set) on every frame.
//
// Exponent: E(x) = unbiased exponent field of x (-1023 for 0), m_k = max over the entry's
// superset contributions of E(c), L_k = ceil(log2 kappa_k) with kappa_k the number of superset
// contributions, e_k = m_k + 1 + L_k - 62 limited to [-1022, 1023], 0 when every contribution
// is 0.  Then |q| < 2^(62 - L_k), |S_k| < 2^62, and |val_k - sum c| <= kappa_k 2^(e_k - 1) plus
// the conversion's rounding: about 2^-56 of the entry's largest contribution.
//
// Entries are keyed by the value index of their upper block (unit (a, b), a <= b); the mirror
// block folds the same contributions and is written with the same value.
#include "sta_claim.cuh"
#include "sta_fold.cuh"

namespace sta {
namespace {

__device__ __forceinline__ int exp_field(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ int ceil_log2(int64_t k) {  // k >= 1
    int L = 0;
    while (((int64_t)1 << L) < k) ++L;
    return L;
}

// value index of entry q of a unit (6-run entries for a diagonal unit, row-major for a pair)
__device__ __forceinline__ int32_t unit_key(int4 bm, bool diag, int q) {
    const int rs = bm.y >> 1;
    if (diag) {
        const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
        return bm.x + i * rs + j;
    }
    return bm.x + (q / 3) * rs + q % 3;
}

// m_k: maximum exponent field over the superset contributions of every entry.
// One thread per (tet, unit slot).
__global__ void k_fx_emax(int64_t T, const int32_t *__restrict__ tunit, const int4 *__restrict__ bmeta,
                          const double *__restrict__ Ke, int32_t *__restrict__ emax) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 10 * T;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / 10;
        const int s = (int)(i % 10);
        const int4 bm = __ldg(bmeta + __ldg(tunit + i));
        const bool diag = s < 4;
        const double *run = Ke + ke_slot_at(T, t, s);
        for (int q = 0; q < (diag ? 6 : 9); ++q) atomicMax(&emax[unit_key(bm, diag, q)], exp_field(run[q]));
    }
}

// e_k from m_k and the unit's contributor count.  One thread per unit.
__global__ void k_fx_exponents(int64_t nunits, const int4 *__restrict__ bmeta,
                               const int32_t *__restrict__ emax, int16_t *__restrict__ e) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunits;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int4 bm = bmeta[u];
        const bool diag = bm.y & 1;
        const int L = ceil_log2(bm.w - bm.z > 0 ? bm.w - bm.z : 1);
        for (int q = 0; q < (diag ? 6 : 9); ++q) {
            const int32_t k = unit_key(bm, diag, q);
            const int m = emax[k];
            int ek = m + 1 + L - 62;
            ek = ek < -1022 ? -1022 : (ek > 1023 ? 1023 : ek);
            e[k] = (int16_t)(m == -1023 ? 0 : ek);
        }
    }
}

// q of every superset contribution, at the element-cache offsets of Ke.  One thread per
// (tet, unit slot).
__global__ void k_fx_quantize(int64_t T, const int32_t *__restrict__ tunit,
                              const int4 *__restrict__ bmeta, const double *__restrict__ Ke,
                              const int16_t *__restrict__ e, long long *__restrict__ Kq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 10 * T;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / 10;
        const int s = (int)(i % 10);
        const int4 bm = __ldg(bmeta + __ldg(tunit + i));
        const bool diag = s < 4;
        const int64_t off = ke_slot_at(T, t, s);
        for (int q = 0; q < (diag ? 6 : 9); ++q)
            Kq[off + q] = __double2ll_rn(Ke[off + q] * pow2i(-e[unit_key(bm, diag, q)]));
    }
}

// Value of an entry from its integer sum, written to the entry and (off the block diagonal, or
// for a pair unit) to its mirror.
__device__ __forceinline__ void fx_write(const FoldArgs &A, const int16_t *__restrict__ e,
                                         int4 bm, int2 mir, bool diag, int q, long long S) {
    const int32_t k = unit_key(bm, diag, q);
    double v = __ll2double_rn(S) * pow2i(e[k]);
    const int rs = bm.y >> 1;
    if (diag) {
        const int i = q < 3 ? 0 : (q < 5 ? 1 : 2), j = q < 3 ? q : (q < 5 ? q - 2 : 2);
        if (i == j && A.eps != 0.0) v += A.eps;
        A.val[k] = v;
        if (i != j) A.val[bm.x + j * rs + i] = v;
    } else {
        A.val[k] = v;
        A.val[mir.x + (q % 3) * mir.y + q / 3] = v;
    }
}

// Fixed-point frame, phase 1: as k_stream_claim (activity bits, mask, first-wins unit claims,
// fold list, entry counts), and each (edited tet, slot) thread adds its quantised contributions
// to the unit's integer sums (+q on activation, -q on deactivation).
constexpr int FX_CLAIM_THREADS = 256;

__global__ void __launch_bounds__(FX_CLAIM_THREADS)
k_fx_claim(const int32_t *__restrict__ edited, int64_t m,
                           const int64_t *__restrict__ m_dev, int64_t T,
                           const int32_t *__restrict__ tunit, const int32_t *__restrict__ cslot,
                           int32_t *__restrict__ ccode, uint8_t *__restrict__ mask,
                           int32_t *__restrict__ owner, int32_t *__restrict__ list,
                           unsigned long long *counters, const int4 *__restrict__ bmeta,
                           const long long *__restrict__ Kq, long long *__restrict__ S) {
    const int64_t n = 10 * (m_dev ? *m_dev : m);
    const int lane = threadIdx.x & 31;
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
            const int64_t off = ke_slot_at(T, t, s);
            ccode[slot] = (int32_t)((uint32_t)off | (on << 31));
            diag = s < 4;
            const int4 bm = __ldg(bmeta + u);
            for (int q = 0; q < (diag ? 6 : 9); ++q) {
                const long long v = __ldg(Kq + off + q);
                atomicAdd(reinterpret_cast<unsigned long long *>(&S[unit_key(bm, diag, q)]),
                          (unsigned long long)(on ? v : -v));
            }
            won = atomicCAS(&owner[u], INT32_MAX, 0) == INT32_MAX;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, won);
        const unsigned dball = __ballot_sync(0xffffffffu, won && diag);
        const unsigned long long base = cta_append<FX_CLAIM_THREADS>(
            counters, __popc(ball), 18 * __popc(ball) - 9 * __popc(dball));
        if (won) list[base + __popc(ball & ((1u << lane) - 1u))] = u;
    }
}

// Fixed-point frame, phase 2: convert the touched units' entries and release the claims.
// 9 lanes per listed unit (6 used by a diagonal unit), 3 units per warp.  `next_count`, when
// given, is the next frame's count pair (graph mode alternates two), zeroed here.
__global__ void k_fx_convert(FoldArgs A, const int32_t *__restrict__ list,
                             const unsigned long long *__restrict__ count,
                             const int16_t *__restrict__ e, const long long *__restrict__ S,
                             int32_t *__restrict__ owner, unsigned long long *next_count) {
    if (next_count && blockIdx.x == 0 && threadIdx.x == 0) {
        next_count[0] = 0;
        next_count[2] = 0;
    }
    const int lane = threadIdx.x & 31;
    const int g = lane / 9, q = lane % 9;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nitems = (int64_t)*count;
    for (int64_t base = warp * 3; base < nitems; base += nwarps * 3) {
        const int64_t item = base + g;
        if (g >= 3 || item >= nitems) continue;
        const int32_t u = __ldg(list + item);
        const int4 bm = __ldg(A.bmeta + u);
        const bool diag = bm.y & 1;
        if (diag && q >= 6) continue;
        const int2 mir = diag ? make_int2(0, 0) : __ldg(A.bmirror + u);
        fx_write(A, e, bm, mir, diag, q, S[unit_key(bm, diag, q)]);
        if (q == 0) owner[u] = INT32_MAX;
    }
}

int grid_cap(const Ctx *c, int64_t items, int threads) {
    int64_t g = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)c->num_sms * 16;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

// Exponents and quantised contributions from the current element cache (allocates the
// fixed-point arrays on first use).
int launch_fx_prepare(Ctx *c, cudaStream_t s) {
    if (!c->fx_q) {
        STA_TRY(dev_alloc(c, &c->fx_q, KE_STRIDE * (c->T > 0 ? c->T : 1)));
        STA_TRY(dev_alloc(c, &c->fx_e, c->nnz > 0 ? c->nnz : 1));
        STA_TRY(dev_alloc(c, &c->fx_s, c->nnz > 0 ? c->nnz : 1));
    }
    if (c->T == 0) return STA_OK;
    // m_k in the integer-sum array (rebuilt afterwards), as int32 starting very negative
    int32_t *emax = reinterpret_cast<int32_t *>(c->fx_s);
    STA_CUDA_TRY(cudaMemsetAsync(emax, 0x80, sizeof(int32_t) * c->nnz, s));
    k_fx_emax<<<grid_cap(c, 10 * c->T, 256), 256, 0, s>>>(c->T, c->tunit, c->bmeta, c->Ke, emax);
    STA_CUDA_TRY(cudaMemsetAsync(c->fx_e, 0, sizeof(int16_t) * c->nnz, s));
    k_fx_exponents<<<grid_cap(c, c->nunits, 256), 256, 0, s>>>(c->nunits, c->bmeta, emax, c->fx_e);
    STA_CUDA_TRY(cudaMemsetAsync(c->fx_q, 0, sizeof(long long) * KE_STRIDE * c->T, s));
    k_fx_quantize<<<grid_cap(c, 10 * c->T, 256), 256, 0, s>>>(c->T, c->tunit, c->bmeta, c->Ke,
                                                             c->fx_e, c->fx_q);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_fx_frame(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev, int64_t cap,
                    int32_t *touched, unsigned long long *counters, cudaStream_t s,
                    unsigned long long *next_cnt) {
    const int threads = FX_CLAIM_THREADS;
    k_fx_claim<<<grid_cap(c, 10 * cap, threads), threads, 0, s>>>(
        edited, m, m_dev, c->T, c->tunit, c->cslot, c->ccode, c->mask, c->owner, touched,
        counters, c->bmeta, c->fx_q, c->fx_s);
    k_fx_convert<<<grid_cap(c, (10 * (cap > 0 ? cap : 1) + 2) / 3 * 32, 128), 128, 0, s>>>(
        fold_args(c), touched, counters + 1, c->fx_e, c->fx_s, c->owner,
        next_cnt ? next_cnt + 1 : nullptr);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace sta
