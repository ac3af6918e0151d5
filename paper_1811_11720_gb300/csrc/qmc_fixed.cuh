// qmc_fixed.cuh -- the symmetric Korobov map (Sec. 2.3, Eq. (korobov)) on the integer pipe.
//
// For Korobov<r,r> the map is phi(v) = v^(r+1) P(v) on v = min(x, 1 - x) in [0, 1/2]
// (phi(x) = 1 - phi(1 - x) above 1/2), with P(v) = sum_k A_k v^k,
// A_k = C (-1)^k binom(r,k) / (r+1+k), and the weight is C (v (1 - v))^r.  In w = 1 - v the
// polynomial has positive integer coefficients, so for r = 1..6 (compiled orders) the map
// is evaluated with unsigned 64-bit integer multiplies, r being a compile-time constant:
//
//   * v enters in 0.64 fixed point, V = v 2^64, straight from the top word X of the shifted
//     lattice fraction x: V = X (x < 1/2) or 2^64 - 1 - X, within 2^-64 of min(x, 1 - x).
//   * P is evaluated in w = 1 - v, where its coefficients are positive:
//       P(v) = C int_0^1 s^r (1 - v s)^r ds = sum_k binom(r+k, k) (1 - v)^k
//     (expand (1 - v s)^r = ((1 - s) + w s)^r and integrate the Beta integrals), e.g.
//     1 + 2w | 1 + 3w + 6w^2 | 1 + 4w + 10w^2 + 20w^3 | 1 + 5w + 15w^2 + 35w^3 + 70w^4.
//     Unsigned Estrin form in fixed point with F fractional bits, F the largest value with
//     P(1) 2^F = sum_k binom(r+k, k) 2^F < 2^64 (every partial sum is at most that for
//     w <= 1): coefficient pairs (c_2j + c_2j+1 w) by shifts and adds, times w^2j from
//     squarings; each product truncates by at most 3 units of 2^-F (F = 62, 60, 58, 57,
//     55, 53 for r = 1..6; the products drop their low partial products, see mulhi_trunc).
//     w^2 comes from v^2 by additions.  Exact-arithmetic checks of these integer steps give
//     the same worst phi error as Horner's scheme (2^-56.2 for r = 3) with one or two fewer
//     64-bit products per dimension (and no multiplies for the coefficients).
//   * phi = v^(r+1) P in 0.64 fixed point; the absolute error is below 2^-(61 - 1.7 r)
//     (2^-54.9 for r = 4, 2^-50.9 for r = 6: the power's truncations times
//     P <= binom(2r+1, r), and the truncations of the last product scaled by 2^(64 - F)).  The integrands
//     that accept a fixed-point coordinate take it as is; otherwise it is rounded to double.
//   * t = v (1 - v) = V - V^2 2^-64 in 0.64 fixed point enters the running product over
//     the dimensions, kept in the format Fx (a 64-bit mantissa, renormalized after each
//     factor, and an exponent), whose r-th power times C^d is rounded once to double: the
//     product keeps relative precision however small it becomes.  Each t is exact to
//     3 2^-64 absolutely, which moves the weight by less than 2^-58 of its largest value
//     C^d 4^(-rd); t itself is not normalized (its low bits are all it has), so a factor
//     t >= 2^-k costs the product about 2^-(62-k) relatively.
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
__host__ __device__ constexpr double pow2_c(int e) {
    double x = 1.0;
    for (int i = 0; i < e; ++i) x *= 2.0;
    return x;
}
__host__ __device__ constexpr long long korobov_Pw(int r, int k) {   // binom(r+k, k)
    long long b = 1;
    for (int i = 1; i <= k; ++i) b = b * (r + i) / i;
    return b;
}
__host__ __device__ constexpr int korobov_F(int r) {   // fractional bits of P in w = 1 - v
    double S = 0.0;
    for (int k = 0; k <= r; ++k) S += (double)korobov_Pw(r, k);
    int F = 0;
    while (S * pow2_c(F + 1) < pow2_c(64)) ++F;
    return F;
}

// ---------------------------------------------------------------------------------------
// High word of a 64 x 64-bit product without the low x low partial product and the low
// halves of the cross products: a 32 x 32 -> 64-bit multiply, two 32-bit high multiplies
// and a 64-bit add.  The result is at most 2 below floor(a b / 2^64) (never above), which
// the fixed-point error bounds below include.
__device__ __forceinline__ uint64_t mulhi_trunc(uint64_t a, uint64_t b) {
    const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32);
    const uint32_t bl = (uint32_t)b, bh = (uint32_t)(b >> 32);
    return (uint64_t)ah * bh + __umulhi(ah, bl) + __umulhi(al, bh);
}

// The same for a square: the two cross products are equal, so one 32-bit high multiply
// doubled (bit-identical to mulhi_trunc(a, a), which the compiler does not fold).
__device__ __forceinline__ uint64_t sqhi_trunc(uint64_t a) {
    const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32);
    return (uint64_t)ah * ah + ((uint64_t)__umulhi(ah, al) << 1);
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

// Truncated product (relative error below 2^-61 for normalized inputs); exponents add.
__device__ __forceinline__ Fx fx_mul(Fx a, Fx b) { return {mulhi_trunc(a.m, b.m), a.e + b.e}; }
__device__ __forceinline__ Fx fx_sq(Fx a) { return {sqhi_trunc(a.m), 2 * a.e}; }

// Normalize a mantissa that is zero or >= 2^32 (shift 0..32; zero stays zero).
__device__ __forceinline__ Fx fx_norm(Fx a) {
    const int lz = __clz((unsigned)(a.m >> 32));
    return {a.m << lz, a.e - lz};
}

// Normalize any mantissa (zero stays zero).  Mantissas below 2^32 (a lattice coordinate
// within 2^-32 of 0 or 1) take the slower branch.
__device__ __forceinline__ Fx fx_norm_any(uint64_t m, int e) {
    const uint32_t hi = (uint32_t)(m >> 32);
    if (hi) {
        const int lz = __clz(hi);
        return {m << lz, e - lz};
    }
    const int lz = __clzll(m);   // 64 for zero
    return {m ? (m << (lz & 63)) : 0ull, e - lz};
}

// Round to the nearest double (ties to even on the truncated mantissa).  Zero, and values
// below the normal range, give 0.
__device__ __forceinline__ double fx_to_double(Fx a) {
    a = fx_norm_any(a.m, a.e);
    const int be = a.e + 1021;   // biased exponent minus one
    if (!a.m || be < 0) return 0.0;
    uint64_t mant = a.m >> 11;
    const uint64_t rb = (a.m >> 10) & 1u;
    const uint64_t sticky = a.m & 0x3FFull;
    mant += rb & ((sticky != 0) | (mant & 1u));
    // adding the mantissa with its leading one to (exponent - 1) << 52 carries correctly
    return __longlong_as_double((long long)(((uint64_t)be << 52) + mant));
}

// The same for a normalized (or zero) mantissa, with overflow to +infinity.
__device__ __forceinline__ double fx_to_double_sat(Fx a) {
    const int be = a.e + 1021;
    if (!a.m || be < 0) return 0.0;
    if (be > 2045) return __longlong_as_double(0x7FF0000000000000ll);
    uint64_t mant = a.m >> 11;
    const uint64_t rb = (a.m >> 10) & 1u;
    const uint64_t sticky = a.m & 0x3FFull;
    mant += rb & ((sticky != 0) | (mant & 1u));
    return __longlong_as_double((long long)(((uint64_t)be << 52) + mant));
}

// a^p for a normalized a and a runtime p >= 1 (binary powering from the top bit; the loop
// is uniform when p is).  Each product truncates by at most 2^-61 relatively.
__device__ __forceinline__ Fx fx_powi(Fx a, int p) {
    Fx r = a;
#pragma unroll 1
    for (int i = 30 - __clz(p); i >= 0; --i) {
        r = fx_norm(fx_sq(r));
        if ((p >> i) & 1) r = fx_norm(fx_mul(r, a));
    }
    return r;
}

// 1/a for a normalized a = m 2^(e - 64): R = 2^127 / m (R < 2^64 for m > 2^63) by Newton's
// iteration R <- R + R (2^127 - m R) 2^-127 from a single-precision seed (rcp.approx of
// the top 32 bits, relative error ~2^-22), two steps (2^-44, then below 2^-61: at most 4
// units low).  m within 2^32 of 2^63 takes the first-order value 2^64 - 2 (m - 2^63)
// (exact to 4 units there), m = 2^63 the exact power of two.  The result may fall a few
// units below 2^63; fx_to_double renormalizes.
__device__ __forceinline__ Fx fx_recip(Fx a) {
    const uint64_t m = a.m;
    const uint32_t mh = (uint32_t)(m >> 32);
    if (mh == 0x80000000u) {
        const uint64_t dl = m - 0x8000000000000000ull;
        if (!dl) return Fx{0x8000000000000000ull, 2 - a.e};
        return Fx{0 - 2 * dl, 1 - a.e};
    }
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint2float_rn(mh)));
    const uint32_t rb = __float_as_uint(r);                 // r = 2^E (1 + f), E = -32 or -31
    const int E = (int)(rb >> 23) - 127;
    const uint64_t mant = (uint64_t)((rb & 0x7FFFFFu) | 0x800000u);
    uint64_t R = E >= -31 ? 0xFFFFFFFFFFFFFFFFull : mant << (72 + E);   // r 2^95
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t plo = m * R, phi = __umul64hi(m, R);
        // high word of 2^127 - m R (two's complement; |2^127 - m R| < 2^107)
        const uint64_t ehi = 0x8000000000000000ull - phi - (plo != 0 ? 1ull : 0ull);
        const bool neg = (long long)ehi < 0;
        const uint64_t c = __umul64hi(R, neg ? 0 - ehi : ehi) << 1;
        R = neg ? R - c : R + c;
    }
    return Fx{R, 1 - a.e};
}

// x 2^-64 for a 0.64 fixed-point x, rounded to nearest.
__device__ __forceinline__ double fixed_to_double64(uint64_t x) {
    const long long b = __double_as_longlong(__ull2double_rn(x));
    return __longlong_as_double(b ? b - (64ll << 52) : 0ll);
}

// ---------------------------------------------------------------------------------------
// v^E 2^64 for V = v 2^64 and V2 = v^2 2^64 (E >= 2): products of squares, E - 1 roundings
// at most (each truncating by at most 3 units of 2^-64).
template <int E>
__device__ __forceinline__ uint64_t fixed_pow(uint64_t V, uint64_t V2) {
    static_assert(E >= 2, "power");
    if constexpr (E == 2) {
        return V2;
    } else if constexpr (E == 3) {
        return mulhi_trunc(V2, V);
    } else {
        const uint64_t h = fixed_pow<E / 2>(V, V2);
        const uint64_t sq = sqhi_trunc(h);
        if constexpr (E % 2) return mulhi_trunc(sq, V);
        else return sq;
    }
}

// x C for a compile-time constant C as shifts and adds (the integer-multiply pipe is the
// busier one in this kernel; the product must fit in 64 bits).
__host__ __device__ constexpr int ctz_c(uint64_t c) {
    int b = 0;
    while (!(c & 1)) {
        c >>= 1;
        ++b;
    }
    return b;
}
template <uint64_t C>
__device__ __forceinline__ uint64_t mul_const(uint64_t x) {
    if constexpr (C == 0) return 0;
    else return (x << ctz_c(C)) + mul_const<(C & (C - 1))>(x);
}

// The pair J of P's coefficients as (binom(R+2J, 2J) + binom(R+2J+1, 2J+1) w) 2^F, with
// ws = w 2^F (the second coefficient is 0 past k = R).
template <int R, int J>
__device__ __forceinline__ uint64_t korobov_pair(uint64_t ws) {
    constexpr int F = korobov_F(R);
    constexpr uint64_t c0 = (uint64_t)korobov_Pw(R, 2 * J) << F;
    constexpr uint64_t c1 = 2 * J + 1 <= R ? (uint64_t)korobov_Pw(R, 2 * J + 1) : 0ull;
    return c0 + mul_const<c1>(ws);
}

// P(w) 2^F = sum_k binom(R+k, k) w^k 2^F for Korobov<R,R>, W = w 2^64 (w = 1 - v), in
// Estrin's form: sum_J (c_2J + c_2J+1 w) w^2J.  The pairs need only shifts and adds, and
// w^2 = 1 - 2v + v^2 comes from V2 = v^2 2^64 by additions (2^64 - 2 - 2V + V2, within 3
// units of floor(W^2 2^-64); V < 2^63), so P costs 0 (R = 1), 1 (R = 2, 3), 3 (R = 4, 5)
// or 5 (R = 6) 64-bit high products against R in Horner's scheme, with the same error
// bound (every term is positive, every partial sum at most P(1) 2^F < 2^64).
template <int R>
__device__ __forceinline__ uint64_t korobov_P(uint64_t V, uint64_t V2) {
    constexpr int F = korobov_F(R);
    const uint64_t W = ~V;
    const uint64_t ws = W >> (64 - F);
    uint64_t P = korobov_pair<R, 0>(ws);
    if constexpr (R >= 2) {
        const uint64_t W2 = V2 - 2 * V - 2;
        P += mulhi_trunc(korobov_pair<R, 1>(ws), W2);
        if constexpr (R >= 4) {
            const uint64_t W4 = sqhi_trunc(W2);
            P += mulhi_trunc(korobov_pair<R, 2>(ws), W4);
            if constexpr (R >= 6) P += mulhi_trunc(korobov_pair<R, 3>(ws), mulhi_trunc(W4, W2));
        }
    }
    return P;
}

// phi(v) 2^64 for V = v 2^64 (v <= 1/2), and t = v (1 - v) folded into the normalized
// running product Wp.
template <int R>
__device__ __forceinline__ uint64_t korobov_phi_fixed(uint64_t V, Fx &Wp) {
    static_assert(R >= 1 && R <= kMaxKorobovInt, "integer Korobov order");
    constexpr int F = korobov_F(R);
    const uint64_t V2 = sqhi_trunc(V);
    // P in w = 1 - v (2^64 - 1 - V, within 2^-64 of (1 - v) 2^64)
    const uint64_t p = korobov_P<R>(V, V2);
    // v^(r+1) 2^64
    const uint64_t pw = fixed_pow<R + 1>(V, V2);
    // t = v - v^2 in 0.64 fixed point (<= 2^62), into the weight product as it is: its
    // leading zeros carry no information (t is exact to 3 2^-64 absolutely), and the
    // product, at least 2^31 for t >= 2^-32, is renormalized afterwards
    Wp = fx_norm(fx_mul(Wp, Fx{V - V2, 0}));
    return mulhi_trunc(pw, p) << (64 - F);
}

// Wp^E for a normalized Wp, normalized (binary powering).
template <int E>
__device__ __forceinline__ Fx fx_pow(Fx Wp) {
    if constexpr (E == 1) {
        return Wp;
    } else {
        const Fx h = fx_pow<E / 2>(Wp);
        const Fx sq = fx_norm(fx_sq(h));
        if constexpr (E % 2) return fx_norm(fx_mul(sq, Wp));
        else return sq;
    }
}

// C^d (prod_j t_j)^r rounded to double; cdx = C^d as Fx.
template <int R>
__device__ __forceinline__ double korobov_weight_fixed(Fx Wp, Fx cdx) {
    return fx_to_double(fx_mul(fx_pow<R>(Wp), cdx));
}

}  // namespace qmc
