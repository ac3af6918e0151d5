// qmc_lattice.cuh -- exact rank-1 lattice points on the integer pipe.
//
// A point coordinate of the shifted rank-1 lattice (Sec. 2.1, Eq. (lattice); Fig. 1) is
//     v = frac(r/n + Delta),  r = i z_j mod n,  Delta = D 2^-53  (D a 53-bit integer),
// and the library's contract is u = RN(v): the exact rational rounded once to the nearest
// double.  On GB300 the FP64 pipe is the scarce resource (~2 DFMA/clk/SM), while the
// integer pipe is ~30x wider, so the point itself never touches FP64:
//
//   * r/n is carried as a 128-bit fixed-point fraction F = floor(r 2^128 / n) plus the
//     exact remainder rem = r 2^128 mod n.  Stepping i -> i+1 adds the constants
//     Fz = floor(z 2^128 / n), remz = z 2^128 mod n with a carry from the remainder; the
//     wrap of r past n is the natural overflow of the 128-bit add (mod 2^128 is frac).
//   * The shift enters as D 2^75, i.e. D << 11 added to the high word (mod 2^64).
//   * v = (V + rem/n) 2^-128 with V = F + D 2^75 mod 2^128; rounding to 53 bits needs the
//     leading-zero count, a funnel shift, the round bit and a sticky bit (lower bits of V
//     or rem != 0).  When V's high word is zero (v < 2^-64, which needs r/n + Delta within
//     2^-64 of an integer) more quotient bits are produced from rem by long division.
//
// Everything here is exact integer arithmetic; the only floating-point objects are the
// final bit pattern and, at the start of a stream, FP64 estimates of a quotient that is
// then corrected exactly (divmod_128_64_fast).
#pragma once
#include <cstdint>

namespace qmc {

struct DimConst {
    uint64_t fz_hi, fz_lo;  // floor(z 2^128 / n)
    uint64_t remz;          // z 2^128 mod n
};

// Restoring division of (hi:lo) by n, requiring hi < n: quotient < 2^64.
__host__ __device__ inline void divmod_128_64(uint64_t hi, uint64_t lo, uint64_t n, uint64_t *q,
                                              uint64_t *r) {
    uint64_t quo = 0;
#pragma unroll 1
    for (int b = 0; b < 64; ++b) {
        uint64_t top = hi >> 63;
        hi = (hi << 1) | (lo >> 63);
        lo <<= 1;
        quo <<= 1;
        if (top || hi >= n) {
            hi -= n;
            quo |= 1;
        }
    }
    *q = quo;
    *r = hi;
}

// The same quotient and remainder for n < 2^62 in a few dozen instructions: a quotient
// estimate q0 from FP64 (within 2^13 + 2 of the exact one: the operands and 1/n carry
// relative errors of a few 2^-53), the exact remainder r = p - q0 n in two's-complement
// 128-bit arithmetic (|r| < 2^14 n), a second FP64 estimate of r / n (within 1), and at
// most two exact corrections.  The result is exact; only the work differs from the loop.
__device__ __forceinline__ void divmod_128_64_fast(uint64_t hi, uint64_t lo, uint64_t n,
                                                   uint64_t *q, uint64_t *r) {
    if (n >= (1ull << 62)) {
        divmod_128_64(hi, lo, n, q, r);
        return;
    }
    const double inv = 1.0 / (double)n;
    const double pd = fma((double)hi, 0x1p64, (double)lo);
    const double qd = fmin(fmax(pd * inv, 0.0), 0x1.fffffffffffffp63);
    const uint64_t q0 = (uint64_t)qd;
    const uint64_t ml = q0 * n, mh = __umul64hi(q0, n);
    const uint64_t rl = lo - ml;
    const uint64_t rh = hi - mh - (lo < ml ? 1ull : 0ull);   // r = (int64)rh 2^64 + rl
    const double rd = fma((double)(long long)rh, 0x1p64, (double)rl);
    const long long q1 = (long long)floor(rd * inv);
    // r - q1 n lies in (-2n, 2n), inside the int64 range for n < 2^62: its low word is it
    long long r2 = (long long)(rl - (uint64_t)q1 * n);
    uint64_t qq = q0 + (uint64_t)q1;
#pragma unroll 1
    for (int it = 0; it < 3 && r2 < 0; ++it) {
        r2 += (long long)n;
        --qq;
    }
#pragma unroll 1
    for (int it = 0; it < 3 && r2 >= (long long)n; ++it) {
        r2 -= (long long)n;
        ++qq;
    }
    *q = qq;
    *r = (uint64_t)r2;
}

// Lattice state of one coordinate at index i: F(i) and rem(i) for r = i z mod n.
// F(i) = (i Fz + floor(i remz / n)) mod 2^128, rem(i) = i remz mod n.
__device__ __forceinline__ void lattice_state_at(uint64_t i, const DimConst &c, uint64_t n,
                                                 uint64_t &f_hi, uint64_t &f_lo,
                                                 uint64_t &rem) {
    uint64_t p_lo = i * c.remz;
    uint64_t p_hi = __umul64hi(i, c.remz);  // i < n and remz < n: p < n^2, p_hi < n
    uint64_t q;
    divmod_128_64_fast(p_hi, p_lo, n, &q, &rem);
    uint64_t lo = i * c.fz_lo;
    uint64_t hi = __umul64hi(i, c.fz_lo) + i * c.fz_hi;
    f_lo = lo + q;
    f_hi = hi + (f_lo < lo);
}

// One lattice step i -> i+1.
__device__ __forceinline__ void lattice_step(const DimConst &c, uint64_t n, uint64_t &f_hi,
                                             uint64_t &f_lo, uint64_t &rem) {
    uint64_t r2 = rem + c.remz;             // < 2n < 2^64 for n < 2^63
    uint64_t carry = (r2 >= n) ? 1u : 0u;
    rem = carry ? r2 - n : r2;
    uint64_t lo = f_lo + c.fz_lo;
    uint64_t c1 = (lo < f_lo) ? 1u : 0u;
    uint64_t lo2 = lo + carry;
    uint64_t c2 = (lo2 < lo) ? 1u : 0u;
    f_lo = lo2;
    f_hi = f_hi + c.fz_hi + c1 + c2;
}

// Round (vhi:vlo + rem/n) 2^-128 to the nearest double; general path for vhi == 0.
static __device__ __noinline__ double fixed_to_double_small(uint64_t vlo, uint64_t rem, uint64_t n) {
    if (vlo == 0 && rem == 0) return 0.0;
    // more bits: rem 2^64 = e n + rem2, so the value is (vlo 2^64 + e + rem2/n) 2^-192
    uint64_t e, rem2;
    divmod_128_64(rem, 0, n, &e, &rem2);
    uint64_t whi, wlo;
    int bexp;  // biased exponent minus one, see the fast path
    if (vlo != 0) {
        int lz = __clzll(vlo);
        whi = lz ? ((vlo << lz) | (e >> (64 - lz))) : vlo;
        wlo = lz ? (e << lz) : e;
        bexp = 957 - lz;   // value in [2^(-65-lz), 2^(-64-lz))
    } else {
        // v < 2^-128 cannot happen for n < 2^64 and a 53-bit shift (v >= 2^-53 / n);
        // kept total for any input
        if (e == 0) return 0.0;
        int lz = __clzll(e);
        whi = e << lz;
        wlo = 0;
        bexp = 893 - lz;   // value in [2^(-129-lz), 2^(-128-lz))
    }
    uint64_t mant = whi >> 11;
    uint64_t rb = (whi >> 10) & 1u;
    uint64_t sticky = (whi & 0x3FFull) | wlo | rem2;
    mant += rb & ((sticky != 0) | (mant & 1u));
    return __longlong_as_double((long long)(((uint64_t)bexp << 52) + mant));
}

// u = RN((V + rem/n) 2^-128) for V = (vhi:vlo).  Fast path for vhi != 0.
__device__ __forceinline__ double fixed_to_double(uint64_t vhi, uint64_t vlo, uint64_t rem,
                                                  uint64_t n) {
    if (vhi == 0) return fixed_to_double_small(vlo, rem, n);
    int lz = __clzll(vhi);
    uint64_t whi = lz ? ((vhi << lz) | (vlo >> (64 - lz))) : vhi;
    uint64_t wlo = lz ? (vlo << lz) : vlo;
    uint64_t mant = whi >> 11;                 // 53 bits, leading one at bit 52
    uint64_t rb = (whi >> 10) & 1u;
    uint64_t sticky = (whi & 0x3FFull) | wlo | rem;
    mant += rb & ((sticky != 0) | (mant & 1u));
    // value = mant 2^(-53-lz), biased exponent 1022 - lz; adding mant (implicit bit
    // included) to (exponent - 1) << 52 also handles the carry mant == 2^53.
    return __longlong_as_double((long long)(((uint64_t)(1021 - lz) << 52) + mant));
}

}  // namespace qmc
