// qmc_fixed.cuh -- the symmetric Korobov map (Sec. 2.3, Eq. (korobov)) on the integer pipe.
//
// For Korobov<r,r> the map is phi(v) = v^(r+1) P(v) on v = min(x, 1 - x) in [0, 1/2]
// (phi(x) = 1 - phi(1 - x) above 1/2), with P(v) = sum_k A_k v^k,
// A_k = C (-1)^k binom(r,k) / (r+1+k), and the weight is C (v (1 - v))^r.  For r <= 4 every
// A_k is an integer (3 -2 | 10 -15 6 | 35 -84 70 -20 | 126 -420 540 -315 70), so the map is
// evaluated with 64-bit integer multiplies, the order r being a compile-time constant:
//
//   * v enters in 0.64 fixed point, V = v 2^64, straight from the top word X of the shifted
//     lattice fraction x: V = X (x < 1/2) or 2^64 - 1 - X, within 2^-64 of min(x, 1 - x).
//   * P(v) by Horner in signed fixed point with F fractional bits, F the largest value that
//     keeps every Horner intermediate (bounded on [0, 1/2] by
//     M = max_k sum_{j>=k} |A_j| 2^(k-j)) below 2^62 / (M + 1); each step truncates by at
//     most 2^-F.  P decreases on [0, 1/2] from A_0 to 2^r, so P 2^(F+G) < 2^63 after a
//     further shift by G.
//   * phi = v^(r+1) P in 0.64 fixed point; the absolute error is below 2^-54 (the power's
//     truncations times P <= 126, and one truncation of the last product).  The integrands
//     that accept a fixed-point coordinate take it as is; otherwise it is rounded to double.
//   * t = v (1 - v) = V - V^2 2^-64 in 0.64 fixed point, normalized into the format Fx (a
//     64-bit mantissa and an exponent) for the running product over the dimensions, whose
//     r-th power times C^d is rounded once to double: the product keeps relative precision
//     however small it becomes, and each t is exact to 2^-64 absolutely, which moves the
//     weight by less than 2^-60 of its largest value C^d 4^(-rd).
//
// GB300 runs ~2 FP64 fused multiply-adds per clock per SM but ~32x as many 32-bit integer
// multiply-adds, so the ~8 FP64 instructions per dimension of the FP64 form cost more than
// the ~60 integer instructions that replace them.
#pragma once
#include <cstdint>

#include "qmc_params.cuh"

namespace qmc {

// ---------------------------------------------------------------------------------------
// Compile-time coefficients of Korobov<r,r>.
__host__ __device__ constexpr long long korobov_C(int r) {   // (2r+1) binom(2r, r)
    long long c = 2 * r + 1;
    for (int i = 1; i <= r; ++i) c = c * (r + i) / i;
    return c;
}
__host__ __device__ constexpr long long korobov_A(int r, int k) {   // C (-1)^k binom(r,k) / (r+1+k), exact for r <= 4
    long long b = 1;
    for (int i = 1; i <= k; ++i) b = b * (r - k + i) / i;
    const long long v = korobov_C(r) * b / (r + 1 + k);
    return (k & 1) ? -v : v;
}
__host__ __device__ constexpr bool korobov_exact(int r) {
    bool ok = true;
    for (int k = 0; k <= r; ++k) {
        long long b = 1;
        for (int i = 1; i <= k; ++i) b = b * (r - k + i) / i;
        ok = ok && (korobov_C(r) * b) % (r + 1 + k) == 0;
    }
    return ok;
}
__host__ __device__ constexpr double pow2_c(int e) {
    double x = 1.0;
    for (int i = 0; i < e; ++i) x *= 2.0;
    return x;
}
__host__ __device__ constexpr int korobov_F(int r) {   // Horner fractional bits
    double M = 0.0;
    for (int k = 0; k <= r; ++k) {
        double s = 0.0;
        for (int j = r; j >= k; --j) {
            const long long a = korobov_A(r, j);
            s = s * 0.5 + (double)(a < 0 ? -a : a);
        }
        if (s > M) M = s;
    }
    int F = 0;
    while ((M + 1.0) * pow2_c(F + 1) <= pow2_c(62)) ++F;
    return F;
}
__host__ __device__ constexpr int korobov_G(int r) {   // extra shift of P before the last product: A_0 2^(F+G) <= 2^62
    int G = 0;
    while ((double)korobov_A(r, 0) * pow2_c(korobov_F(r) + G + 1) <= pow2_c(62)) ++G;
    return G;
}

// ---------------------------------------------------------------------------------------
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

// Normalize any mantissa (zero stays zero).
__device__ __forceinline__ Fx fx_norm_any(uint64_t m, int e) {
    const int lz = __clzll(m);   // 64 for zero
    return {m ? (m << (lz & 63)) : 0ull, e - lz};
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

// x 2^-64 for a 0.64 fixed-point x, rounded to nearest.
__device__ __forceinline__ double fixed_to_double64(uint64_t x) {
    const long long b = __double_as_longlong(__ull2double_rn(x));
    return __longlong_as_double(b ? b - (64ll << 52) : 0ll);
}

// ---------------------------------------------------------------------------------------
// Horner steps k = K, K-1, ..., 0 of P for Korobov<R,R>: p <- floor(p V / 2^64) + A_k 2^F.
// For signed p, hi(p_unsigned V) = floor(p V / 2^64) + V [p < 0].
template <int R, int K>
__device__ __forceinline__ long long korobov_horner(long long p, uint64_t V) {
    constexpr long long a = korobov_A(R, K) * (1ll << korobov_F(R));
    const uint64_t hi = __umul64hi((uint64_t)p, V) - (p < 0 ? V : 0ull);
    p = (long long)hi + a;
    if constexpr (K > 0) return korobov_horner<R, K - 1>(p, V);
    else return p;
}

// phi(v) 2^64 for V = v 2^64 (v <= 1/2), and t = v (1 - v) folded into the normalized
// running product Wp.
template <int R>
__device__ __forceinline__ uint64_t korobov_phi_fixed(uint64_t V, Fx &Wp) {
    static_assert(R >= 1 && R <= kMaxKorobovInt && korobov_exact(R), "integer Korobov order");
    constexpr int F = korobov_F(R);
    constexpr int G = korobov_G(R);
    constexpr long long top = korobov_A(R, R) * (1ll << F);
    const long long p = korobov_horner<R, R - 1>(top, V);
    // v^(r+1) 2^64
    const uint64_t V2 = __umul64hi(V, V);
    uint64_t pw;
    if constexpr (R == 1) pw = V2;
    else if constexpr (R == 2) pw = __umul64hi(V2, V);
    else if constexpr (R == 3) pw = __umul64hi(V2, V2);
    else pw = __umul64hi(__umul64hi(V2, V2), V);
    // t = v - v^2 in 0.64 fixed point (<= 2^62), into the weight product
    Wp = fx_norm(fx_mul(Wp, fx_norm_any(V - V2, 0)));
    return __umul64hi(pw, (uint64_t)p << G) << (64 - F - G);
}

// C^d (prod_j t_j)^r rounded to double; cdx = C^d as Fx.
template <int R>
__device__ __forceinline__ double korobov_weight_fixed(Fx Wp, Fx cdx) {
    Fx w = Wp;
    if constexpr (R >= 2) {
        w = fx_norm(fx_mul(Wp, Wp));
        if constexpr (R == 3) w = fx_mul(w, Wp);
        else if constexpr (R == 4) w = fx_norm(fx_mul(w, w));
    }
    return fx_to_double(fx_mul(w, cdx));
}

}  // namespace qmc
