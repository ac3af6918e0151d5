// qmc_fixed.cuh -- the symmetric Korobov map (Sec. 2.3, Eq. (korobov)) on the integer pipe.
//
// For Korobov<r,r> the map is phi(v) = v^(r+1) P(v) on v = min(u, 1 - u) in [0, 1/2]
// (phi(u) = 1 - phi(1 - u) above 1/2), with P(v) = sum_k A_k v^k,
// A_k = C (-1)^k binom(r,k) / (r+1+k), and the weight is C (v (1 - v))^r.  For r <= 4 every
// A_k is an integer (3 -2 | 10 -15 6 | 35 -84 70 -20 | 126 -420 540 -315 70), so the map is
// evaluated with 64-bit integer multiplies and a single rounding to double at the end:
//
//   * P(v) by Horner in signed fixed point with F fractional bits (F = 59, 57, 55, 52 for
//     r = 1..4), chosen on the host so that every Horner intermediate, bounded by
//     max_k sum_{j>=k} |A_j| 2^(k-j) on [0, 1/2], stays below 2^62; each step truncates by
//     at most 2^-F and P >= 2^r on [0, 1/2], so P has relative error < 2^-54.
//   * v^(r+1), t = v (1 - v), the product of the t_j over the dimensions, its r-th power and
//     the factor C^d are carried in the format Fx (a 64-bit mantissa and an exponent), each
//     product truncating at the mantissa's last bit: relative error < 2^-56 overall.
//   * phi and the weight are rounded once to double (to nearest on the truncated value).
//
// v enters as a 0.64 fixed-point number taken straight from the lattice state: the top 64
// bits X of the shifted fraction x give v = X 2^-64 (x < 1/2) or (2^64 - 1 - X) 2^-64, each
// within 2^-64 of the exact min(x, 1 - x).  That moves phi by at most 2.2 2^-64 absolutely
// (below half an ulp of phi for v > 2^-11); for smaller v, phi and the weight are below
// C v^r and their absolute change is below 2^-50 C^d of the largest term of the sum.
//
// GB300 runs ~2 FP64 fused multiply-adds per clock per SM but ~32x as many 32-bit integer
// multiply-adds; the ~8 FP64 instructions per dimension of the FP64 form become ~100
// integer instructions, which cost about a third of the time.  No step rounds more
// coarsely than the FP64 form: results agree with it to a few ulp.
#pragma once
#include <cstdint>

#include "qmc_params.cuh"

namespace qmc {

// value = m 2^(e - 64); m == 0 encodes zero.  Normalized: m >= 2^63.
struct Fx {
    uint64_t m;
    int e;
};

// v >= 0, zero or normal.
__device__ __forceinline__ Fx fx_of_double(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return {b ? ((b << 11) | 0x8000000000000000ull) : 0ull, (int)(b >> 52) - 1022};
}

// Truncated product; exponents add.
__device__ __forceinline__ Fx fx_mul(Fx a, Fx b) { return {__umul64hi(a.m, b.m), a.e + b.e}; }

// Normalize a mantissa that is zero or >= 2^32 (shift 0..32; zero stays zero).
__device__ __forceinline__ Fx fx_norm(Fx a) {
    const int lz = __clz((unsigned)(a.m >> 32));
    return {a.m << lz, a.e - lz};
}

// Round to the nearest double (ties to even on the truncated mantissa).  Zero, and values
// below the normal range, give 0.
__device__ __forceinline__ double fx_to_double(Fx a) {
    a = fx_norm(a);
    const int be = a.e + 1021;   // biased exponent minus one
    if (!a.m || be < 0) return 0.0;
    uint64_t mant = a.m >> 11;
    const uint64_t rb = (a.m >> 10) & 1u;
    const uint64_t sticky = a.m & 0x3FFull;
    mant += rb & ((sticky != 0) | (mant & 1u));
    // adding the mantissa with its leading one to (exponent - 1) << 52 carries correctly
    return __longlong_as_double((long long)(((uint64_t)be << 52) + mant));
}

// 0.64 fixed point of a value in [0, 1): floor(value 2^64).
__device__ __forceinline__ uint64_t fx_to_fixed(Fx a) {
    a = fx_norm(a);
    const int sh = -a.e;   // >= 0 for values below 1
    return sh < 64 ? (a.m >> sh) : 0ull;
}

// phi(v) for v = min(x, 1 - x) as Fx (mantissa >= 2^58), and the weight factor
// t = v (1 - v) folded into Wp (a normalized running product).  V = v 2^64 in 0.64 fixed
// point (V <= 2^63).
__device__ __forceinline__ Fx korobov_int_phi(uint64_t V, const TransformParams &t, Fx &Wp) {
    const int r = t.r0;
    const int lz = __clzll(V);   // 64 for V == 0
    const Fx fv = {V ? (V << (lz & 63)) : 0ull, -lz};
    // Horner in signed fixed point: p <- floor(p V / 2^64) + A_k 2^F.  For signed p,
    // hi(p_unsigned V) = floor(p V / 2^64) + V [p < 0].
    long long p = t.kfix[r];
#pragma unroll 1
    for (int k = r - 1; k >= 0; --k) {
        const uint64_t hi = __umul64hi((uint64_t)p, V) - (p < 0 ? V : 0ull);
        p = (long long)hi + t.kfix[k];
    }
    // P = p 2^-F >= 2: p >= 2^(F+1) >= 2^54, so its high word is non-zero
    const Fx P = fx_norm(Fx{(uint64_t)p, 64 - t.kfix_F});
    // v^(r+1): mantissas stay >= 2^58, relative error < 2^-57
    Fx pw = fx_mul(fv, fv);
    if (r == 2) {
        pw = fx_mul(pw, fv);
    } else if (r >= 3) {
        pw = fx_mul(pw, pw);
        if (r == 4) pw = fx_mul(pw, fv);
    }
    // t = v (1 - v), with 1 - v ~ (2^64 - 1 - V) 2^-64 (error <= 2^-63 relative)
    Wp = fx_norm(fx_mul(Wp, fx_mul(fv, Fx{~V, 0})));
    return fx_mul(pw, P);
}

__device__ __forceinline__ double korobov_int(uint64_t V, const TransformParams &t, Fx &Wp) {
    return fx_to_double(korobov_int_phi(V, t, Wp));
}

// C^d (prod_j t_j)^r rounded to double; cdx = C^d as Fx.
__device__ __forceinline__ double korobov_int_weight(Fx Wp, int r, Fx cdx) {
    Fx w = Wp;
    if (r >= 2) {
        w = fx_norm(fx_mul(Wp, Wp));
        if (r == 3) w = fx_mul(w, Wp);
        else if (r == 4) w = fx_norm(fx_mul(w, w));
    }
    return fx_to_double(fx_mul(w, cdx));
}

}  // namespace qmc
