// qmc_fp.cuh -- exact bit-level helpers that keep work off the FP64 pipe.
#pragma once
#include <cstdint>

namespace qmc {

// Non-negative double compare on the bit pattern.
__device__ __forceinline__ bool le_half(double u) {
    return (unsigned long long)__double_as_longlong(u) <= 0x3FE0000000000000ull;
}

// 1 - u for u in [1/2, 1], exact (Sterbenz), on the integer pipe.
__device__ __forceinline__ double one_minus_upper(double u) {
    uint64_t b = (uint64_t)__double_as_longlong(u);
    if (b >= 0x3FF0000000000000ull) return 0.0;             // u == 1
    uint64_t mant = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;  // u = mant 2^-53
    uint64_t x = 0x0020000000000000ull - mant;               // 1 - u = x 2^-53, 1 <= x <= 2^52
    int lz = __clzll(x);                                     // >= 11
    return __longlong_as_double((long long)(((uint64_t)(1032 - lz) << 52) + (x << (lz - 11))));
}

// 2 y for y = 0 or a positive normal double, exact, on the integer pipe.
__device__ __forceinline__ double twice(double y) {
    uint64_t b = (uint64_t)__double_as_longlong(y);
    return __longlong_as_double((long long)(b ? b + 0x0010000000000000ull : 0ull));
}

// x^e for a small non-negative integer e (uniform across the warp): left-to-right binary
// powering, floor(log2 e) squarings plus one multiply per further set bit.
__device__ __forceinline__ double ipow_u(double x, int e) {
    if (e <= 0) return 1.0;
    const int top = 31 - __clz(e);
    double r = x;
#pragma unroll 1
    for (int b = top - 1; b >= 0; --b) {
        r *= r;
        if ((e >> b) & 1) r *= x;
    }
    return r;
}

// Select between two doubles on the integer pipe.
__device__ __forceinline__ double sel(bool p, double a, double b) { return p ? a : b; }

}  // namespace qmc
