// qmc_cos.cuh -- cos(2 pi t) on the integer pipe for the oscillatory Genz integrand, whose
// phase arrives as a 64-bit fraction of a turn, T = t 2^64 (mod 2^64 is the periodicity).
//
//   * t = j/256 + r with j = round(t 256) mod 256 and |r| <= 1/512; y = 2 pi r, |y| < 0.0123.
//   * j = 64 q + i: the quadrant q and cos(2 pi i/256), sin(2 pi i/256) = cos(2 pi (64 - i)/256)
//     from a 65-entry table (2^62 scale, rounded to nearest, in shared memory) give
//     cos(2 pi t) = +-(P - P (1 - cos y) +- Q sin y) with (P, Q) the table pair in the
//     order the quadrant asks for (cos(a + y) for even q, sin(a + y) for odd q).
//   * sin|y| = |y| (1 - z/6 + z^2/120) and 1 - cos y = z (1/2 - z/24 + z^2/720), z = y^2
//     (Taylor; the omitted terms are below 9e-18 absolutely), in fixed point: |y| 2^69,
//     z 2^74, coefficients 2^64.
//   Products are truncated high words (mulhi_trunc); the result, a signed 2^62-scaled
//   integer, is within 1e-17 of cos(2 pi t) absolutely (random checks in exact arithmetic:
//   8.6e-18 at most), then rounded once to double.
#pragma once
#include <cstdint>

#include "qmc_fixed.cuh"

namespace qmc {

// cos(2 pi i/256) 2^62, i = 0..64, rounded to nearest (computed in 300-bit arithmetic).
static __constant__ uint64_t kCos256[65] = {
    0x4000000000000000ull, 0x3ffb10c1099a1976ull, 0x3fec43c6f2dafbc7ull, 0x3fd39b5a0310742aull,
    0x3fb11b47a24a4b3cull, 0x3f84c8e1c33fa68full, 0x3f4eaafe114a2d43ull, 0x3f0ec9f4e297526bull,
    0x3ec52f9feeb96056ull, 0x3e71e758c9cb118aull, 0x3e14fdf72461ae55ull, 0x3dae81ced092c67aull,
    0x3d3e82ad8c5bb4bbull, 0x3cc511d891c223ddull, 0x3c424209ed0dc97full, 0x3bb6276d998478c2ull,
    0x3b20d79e651a8c51ull, 0x3a8269a29b927359ull, 0x39daf5e8798ee5e2ull, 0x392a96426823e9edull,
    0x387165e3017b61a4ull, 0x37af8158df2a533full, 0x36e5068a32dc7b22ull, 0x361214b02a03ff37ull,
    0x3536cc521d434606ull, 0x34534f408c4f03bbull, 0x3367c08fe70e8168ull, 0x3274449324c7f69full,
    0x317900d62a2e816aull, 0x30761c17ff2edba4ull, 0x2f6bbe44d55f5dbcull, 0x2e5a106fdfff2c87ull,
    0x2d413cccfe779921ull, 0x2c216eaa3a59bdb7ull, 0x2afad26919d93f45ull, 0x29cd9577c7cbd228ull,
    0x2899e64a123bac30ull, 0x275ff45240a17279ull, 0x261feff9c2e069c2ull, 0x24da0a99ba25bd51ull,
    0x238e76735cd190d9ull, 0x223d66a836964508ull, 0x20e70f3245ffdb2dull, 0x1f8ba4dbf89ab9fbull,
    0x1e2b5d3806f63b1eull, 0x1cc66e9931c45e17ull, 0x1b5d1009e15cc02bull, 0x19ef7943a8ed8a2eull,
    0x187de2a6aea962d2ull, 0x17088530fa459eafull, 0x158f9a75ab1fdcfeull, 0x14135c9417660143ull,
    0x1294062ed59f05a9ull, 0x1111d262b1f67761ull, 0x0f8cfcbd90af8d58ull, 0x0e05c1353f27b17eull,
    0x0c7c5c1e34d3055bull, 0x0af10a22459fe32aull, 0x0964083747309d11ull, 0x07d59395aa5cc38dull,
    0x0645e9af0a6d0af8ull, 0x04b54824b3867d73ull, 0x0323ecbe21bb027dull, 0x0192155f7a3667e0ull,
    0x0000000000000000ull,
};

// cos(2 pi T 2^-64) rounded to double; tab: kCos256 staged in shared memory.
__device__ __forceinline__ double cos_turns_fixed(uint64_t T, const uint64_t *tab) {
    constexpr uint64_t k2Pi = 0xc90fdaa22168c235ull;    // 2 pi 2^61
    constexpr uint64_t kC6 = 0x2aaaaaaaaaaaaaabull;     // 2^64 / 6
    constexpr uint64_t kC24 = 0x0aaaaaaaaaaaaaabull;    // 2^64 / 24
    constexpr uint64_t kK120 = 0x0000888888888889ull;   // 2^54 / 120
    constexpr uint64_t kK720 = 0x000016c16c16c16cull;   // 2^54 / 720
    const uint64_t u = T + (1ull << 55);
    const int j = (int)(u >> 56);
    const long long r = (long long)(u & ((1ull << 56) - 1)) - (1ll << 55);
    const bool neg = r < 0;
    const uint64_t a = (uint64_t)(neg ? -r : r);                 // |r| 2^64 turns, < 2^55
    const uint64_t Y = mulhi_trunc(a << 8, k2Pi);                // |y| 2^69
    const uint64_t Z = sqhi_trunc(Y);                        // z 2^74
    const uint64_t Ps = mulhi_trunc(Z, kC6 - mulhi_trunc(Z, kK120));            // z (1/6 - z/120) 2^74
    const uint64_t Sy = Y - (mulhi_trunc(Y, Ps) >> 10);                         // sin|y| 2^69
    const uint64_t Q2 = 0x8000000000000000ull - (mulhi_trunc(Z, kC24 - mulhi_trunc(Z, kK720)) >> 10);
    const uint64_t Cm = mulhi_trunc(Z, Q2);                                     // (1 - cos y) 2^74
    const int q = j >> 6, i = j & 63;
    const uint64_t ca = tab[i], sa = tab[64 - i];
    const bool even = !(q & 1);
    const uint64_t P = even ? ca : sa, Q = even ? sa : ca;
    // cos(a + y) = cos a - cos a (1 - cos y) - sin a sin y; sin(a + y) = sin a - ... + cos a sin y
    const long long ysin = (long long)(mulhi_trunc(Q, Sy) >> 5);               // Q sin|y| 2^62
    const bool minus = even != neg;                                              // sign of that term is -
    long long v = (long long)P - (long long)(mulhi_trunc(P, Cm) >> 10) + (minus ? -ysin : ysin);
    if (q == 1 || q == 2) v = -v;
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(b ? b - (62ll << 52) : 0ll);
}

}  // namespace qmc
