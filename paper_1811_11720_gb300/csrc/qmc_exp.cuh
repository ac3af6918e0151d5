// qmc_exp.cuh -- e^x by the table-driven method of P. T. P. Tang ("Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic", ACM TOMS
// 15 (1989) 144-157), written for the separable Genz integrands, whose per-evaluation
// FP64 budget after the fixed-point forms is dominated by the exponential.
//
// x = (32 m + j) ln2/32 + r with |r| <= ln2/64, so e^x = 2^m 2^(j/32) e^r:
//   * k = 32 m + j = round(x 32/ln2) by adding 1.5 2^52 (the rounded k lands in the low
//     mantissa bits); r = x - k ln2/32 by two fused multiply-adds with ln2/32 split into
//     L1 = RN(ln2/32) and L2 = RN(ln2/32 - L1);
//   * e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24 + r^3/120 + r^4/720) (Taylor; the omitted
//     r^7/5040 is below 2^-58 relative for |r| <= ln2/64);
//   * 2^(j/32) from a 32-entry table of correctly rounded values (staged in shared memory),
//     the product t (1 + p) as one fused multiply-add, and 2^m added to the exponent field
//     on the integer pipe.
// Ten FP64 instructions; the result is within about 1 ulp.  Arguments outside
// [-708.3, 709] (where 2^m would leave the normal range) take the library exp.
#pragma once
#include <cstdint>

namespace qmc {

// 2^(j/32), j = 0..31, rounded to nearest (computed in 300-bit arithmetic).
static __constant__ double kExp2Table[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0,
};

// tab: kExp2Table staged in shared memory.
__device__ __forceinline__ double exp_table(double x, const double *tab) {
    if (!(x >= -708.3 && x <= 709.0)) return exp(x);   // also NaN
    const double kInvL = 0x1.71547652b82fep+5;        // 32 / ln2
    const double kL1 = 0x1.62e42fefa39efp-6;          // ln2 / 32, rounded
    const double kL2 = 0x1.abc9e3b39803fp-61;         // ln2 / 32 - kL1, rounded
    const double kShift = 0x1.8p52;
    const double t = fma(x, kInvL, kShift);
    const int k = (int)(uint32_t)__double_as_longlong(t);   // low word: round(x 32/ln2)
    const double kd = t - kShift;
    double r = fma(kd, -kL1, x);
    r = fma(kd, -kL2, r);
    double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(r * r, q, r);
    const double tj = tab[k & 31];
    const double v = fma(tj, p, tj);
    return __longlong_as_double(__double_as_longlong(v) + ((long long)(k >> 5) << 52));
}

}  // namespace qmc
