// Append counting shared by the claim kernels of the fixed-point and proxy frames: each warp's
// winners are counted in one CTA-wide step, so a frame issues one atomic per CTA on each
// counter word instead of one per warp (a large frame's warps all appending to one word
// serialise at the L2).
#pragma once

#include "sta_internal.cuh"

namespace sta {
namespace {

// Called by every thread of a CTA of THREADS threads, the same number of times.  Lane 0 of
// each warp brings its warp's counts c1 (for counters[1]) and c3 (for counters[3]); returns,
// to every lane, the warp's first position in counters[1]'s sequence.
template <int THREADS>
__device__ __forceinline__ unsigned long long cta_append(unsigned long long *counters, unsigned c1,
                                                         unsigned c3) {
    __shared__ unsigned long long s_cnt[THREADS / 32];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_cnt[wid] = (unsigned long long)c1 | ((unsigned long long)c3 << 32);
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive prefix of c1 over the warps; totals of both
        unsigned long long t1 = 0, t3 = 0;
        for (int w = 0; w < THREADS / 32; ++w) {
            const unsigned long long v = s_cnt[w];
            s_cnt[w] = t1;
            t1 += v & 0xffffffffull;
            t3 += v >> 32;
        }
        s_base = t1 ? atomicAdd(&counters[1], t1) : 0ull;
        if (t3) atomicAdd(&counters[3], t3);
    }
    __syncthreads();
    const unsigned long long base = s_base + s_cnt[wid];
    __syncthreads();  // s_cnt and s_base are rewritten by the next call
    return base;
}

}  // namespace
}  // namespace sta
