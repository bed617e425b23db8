// Rounding of exact 128-bit integers to doubles in integer arithmetic (the
// exact filtration values are int128 rationals; on GB300 the FP64 pipe is
// narrow, so the conversion is done with integer shifts and the double's bits
// are assembled directly). Host and device: the CPU tests compile it with g++.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define AC_HD __host__ __device__ __forceinline__
#else
#define AC_HD inline
#endif

namespace ac {

AC_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

AC_HD double bits_to_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// x * 2^e2 rounded to the nearest double, ties to even. Requires |x| < 2^127
// and the result in the normal range (|x| * 2^e2 between 2^-1022 and 2^1023),
// which holds for every OrthoSize numerator and denominator here (e2 = -20 or 0).
AC_HD double i128_to_double_rn(__int128 x, int e2) {
    if (x == 0) return 0.0;
    const bool neg = x < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const int nbits = hi ? 128 - clz64(hi) : 64 - clz64(lo);
    uint64_t m;  // the value is m * 2^e, m below 2^53
    int e = 0;
    if (nbits <= 53) {
        m = lo;
    } else {
        const int sh = nbits - 53;
        const unsigned __int128 q = u >> sh;
        const unsigned __int128 rem = u - (q << sh), half = (unsigned __int128)1 << (sh - 1);
        m = (uint64_t)q;
        if (rem > half || (rem == half && (m & 1u))) m++;
        e = sh;
        if (m == (1ull << 53)) {
            m >>= 1;
            e++;
        }
    }
    const int lz = clz64(m) - 11;  // bring the leading bit to position 52
    m <<= lz;
    e -= lz;
    const uint64_t be = (uint64_t)(e + e2 + 52 + 1023);
    return bits_to_double(((uint64_t)neg << 63) | (be << 52) | (m & ((1ull << 52) - 1)));
}

}  // namespace ac
