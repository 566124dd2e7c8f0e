// Exact IEEE-754 binary64 addition (round to nearest, ties to even) in 64-bit integer
// arithmetic, for the fold kernels.
//
// Why: on GB300 the FP64 pipe issues about 0.5e12 lane operations per second while the
// integer pipes issue about 35e12, so moving part of a fold's additions to integer
// instructions raises the rate at which a fold can run.  The result of int_add(a, b) is the
// same bit pattern as the hardware's a + b for all inputs: the common case (both operands
// normal, result normal) is computed here with the textbook align / add-or-subtract /
// normalise / round-to-nearest-even steps on a significand widened by ten guard bits with a
// sticky bit; zero operands are resolved exactly; infinities, NaNs, subnormal operands or
// results and overflow fall back to the hardware addition.
//
// The header compiles as CUDA device code and as plain host C++ (so the host test suite can
// check it against the CPU's own IEEE addition).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define STA_HD __host__ __device__ __forceinline__
#else
#define STA_HD inline
#include <string.h>
#endif

namespace sta {

STA_HD uint64_t f64_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

STA_HD double f64_from(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

STA_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

STA_HD double int_add(double a, double b) {
    const uint64_t ABS = 0x7fffffffffffffffull, FRAC = 0x000fffffffffffffull;
    const uint64_t ua = f64_bits(a), ub = f64_bits(b);
    const uint64_t ma = ua & ABS, mb = ub & ABS;
    const bool sw = ma < mb;  // x: operand of larger magnitude
    const uint64_t x = sw ? ub : ua, y = sw ? ua : ub;
    const uint64_t mx = sw ? mb : ma, my = sw ? ma : mb;
    const int ex = (int)(mx >> 52), ey = (int)(my >> 52);
    if (ex == 0x7ff || (ey == 0 && my != 0)) return a + b;  // inf / NaN / subnormal operand
    if (my == 0) return f64_from(mx == 0 ? (ua & ub) : x);  // a zero operand: exact
    const int d = ex - ey;
    const uint64_t X = ((mx & FRAC) | (1ull << 52)) << 10;  // leading one at bit 62
    const uint64_t Y = ((my & FRAC) | (1ull << 52)) << 10;
    uint64_t Ya;
    if (d == 0)
        Ya = Y;
    else if (d < 63)
        Ya = (Y >> d) | (uint64_t)((Y << (64 - d)) != 0);  // sticky bit
    else
        Ya = 1;
    const bool same = ((x ^ y) >> 63) == 0;
    uint64_t S = same ? X + Ya : X - Ya;
    if (S == 0) return 0.0;  // exact cancellation rounds to +0
    const int lz = clz64(S);
    int e;
    if (lz == 0) {  // carry out of bit 62
        S = (S >> 1) | (S & 1);
        e = ex + 1;
    } else {
        S <<= (lz - 1);
        e = ex - (lz - 1);
    }
    if (e <= 0) return a + b;  // subnormal result
    uint64_t sig = S >> 10;
    const uint64_t rem = S & 0x3ff;
    if (rem > 0x200 || (rem == 0x200 && (sig & 1))) ++sig;
    if (sig >> 53) {
        sig >>= 1;
        ++e;
    }
    if (e >= 0x7ff) return a + b;  // overflow
    return f64_from((x & ~ABS) | ((uint64_t)e << 52) | (sig & FRAC));
}

}  // namespace sta
