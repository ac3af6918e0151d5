// qmc_exp.cuh -- e^x for the separable Genz integrands by the table-driven method of
// P. T. P. Tang ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15 (1989) 144-157), in two forms.
//
// exp_fixed: e^(+-a) for a fixed-point argument a = A 2^-E (the Gaussian, C0 and
// discontinuous forms), carried out in 64-bit integer arithmetic:
//   * u = a log2(e) = A L 2^-(E + 63) with L = log2(e) 2^63 rounded: the 128-bit product
//     holds u exactly up to L's rounding (relative 2^-64); its integer part k and its
//     fraction F = frac(u) 2^64 are two shifts of the product's words by E - 1 bits.
//   * e^-a = 2^(-k - [F > 0]) 2^(F' 2^-64) with F' = 2^64 - F (mod 2^64); e^a = 2^k 2^(F 2^-64).
//   * 2^(F 2^-64) = 2^(j/64) e^y: j is F's top 6 bits, y = rho ln2 2^-6 with rho the
//     other 58 bits as a 0.64 fraction (0 <= y < ln2/64); 2^(j/64) 2^63 from a 64-entry
//     table (rounded to nearest, in shared memory), e^y - 1 = y + y^2 (1/2 + y/6 + y^2/24 +
//     y^3/120 + y^4/720) (Taylor; the omitted y^7/5040 is below 2^-61 relative), evaluated
//     on Y = y 2^70 with coefficients 2^(-6 (k - 1))/k! 2^64, and the product
//     2^(j/64) (1 + (e^y - 1)) lands in [2^63, 2^64): a normalized mantissa.
//   Every product is a truncated high word (mulhi_trunc); the result is within 2^-55
//   relative of e^(+-a) before its single rounding to double (random checks in exact
//   arithmetic give at most 0.15 units of 2^-53).
//
// exp_table: the same method in FP64 for a double argument x = (32 m + j) ln2/32 + r,
// |r| <= ln2/64, so e^x = 2^m 2^(j/32) e^r:
//   * k = 32 m + j = round(x 32/ln2) by adding 1.5 2^52 (the rounded k lands in the low
//     mantissa bits); r = x - k ln2/32 by two fused multiply-adds with ln2/32 split into
//     L1 = RN(ln2/32) and L2 = RN(ln2/32 - L1);
//   * e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24 + r^3/120 + r^4/720) (Taylor; the omitted
//     r^7/5040 is below 2^-58 relative for |r| <= ln2/64);
//   * 2^(j/32) from a 32-entry table (the even entries of the fixed-point table rounded to
//     double, which are the correctly rounded values), the product t (1 + p) as one fused
//     multiply-add, and 2^m added to the exponent field on the integer pipe.
//   Ten FP64 instructions, within about 1 ulp; arguments outside [-708.3, 709] (where 2^m
//   would leave the normal range) take the library exp.
//
// GB300 issues ~2 FP64 fused multiply-adds per clock per SM against ~32x as many integer
// multiply-adds.  The integer form (~60 integer instructions for ~13 FP64 ones) pays when
// the rest of the evaluation leaves the integer multiply pipe room (baker, none, Korobov up
// to r = 3 for the exp families); under the higher Korobov orders that pipe is the
// bottleneck and the FP64 form, on the otherwise idle FP64 pipe, is faster (the crossover
// is FamilyAcc::kIntFinishMaxR).
#pragma once
#include <cstdint>

#include "qmc_fixed.cuh"

namespace qmc {

// 2^(j/64) 2^63, j = 0..63, rounded to nearest (computed in 300-bit arithmetic).
static __constant__ uint64_t kExp2Fixed[64] = {
    0x8000000000000000ull, 0x8164d1f3bc030773ull, 0x82cd8698ac2ba1d7ull, 0x843a28c3acde4046ull,
    0x85aac367cc487b15ull, 0x871f61969e8d1010ull, 0x88980e8092da8527ull, 0x8a14d575496efd9aull,
    0x8b95c1e3ea8bd6e7ull, 0x8d1adf5b7e5ba9e6ull, 0x8ea4398b45cd53c0ull, 0x9031dc431466b1dcull,
    0x91c3d373ab11c336ull, 0x935a2b2f13e6e92cull, 0x94f4efa8fef70961ull, 0x96942d3720185a00ull,
    0x9837f0518db8a96full, 0x99e0459320b7fa65ull, 0x9b8d39b9d54e5539ull, 0x9d3ed9a72cffb751ull,
    0x9ef5326091a111aeull, 0xa0b0510fb9714fc2ull, 0xa27043030c496819ull, 0xa43515ae09e6809eull,
    0xa5fed6a9b15138eaull, 0xa7cd93b4e965356aull, 0xa9a15ab4ea7c0ef8ull, 0xab7a39b5a93ed337ull,
    0xad583eea42a14ac6ull, 0xaf3b78ad690a4375ull, 0xb123f581d2ac2590ull, 0xb311c412a9112489ull,
    0xb504f333f9de6484ull, 0xb6fd91e328d17791ull, 0xb8fbaf4762fb9ee9ull, 0xbaff5ab2133e45fbull,
    0xbd08a39f580c36bfull, 0xbf1799b67a731083ull, 0xc12c4cca66709456ull, 0xc346ccda24976407ull,
    0xc5672a115506daddull, 0xc78d74c8abb9b15dull, 0xc9b9bd866e2f27a3ull, 0xcbec14fef2727c5dull,
    0xce248c151f8480e4ull, 0xd06333daef2b2595ull, 0xd2a81d91f12ae45aull, 0xd4f35aabcfedfa1full,
    0xd744fccad69d6af4ull, 0xd99d15c278afd7b6ull, 0xdbfbb797daf23755ull, 0xde60f4825e0e9124ull,
    0xe0ccdeec2a94e111ull, 0xe33f8972be8a5a51ull, 0xe5b906e77c8348a8ull, 0xe8396a503c4bdc68ull,
    0xeac0c6e7dd24392full, 0xed4f301ed9942b84ull, 0xefe4b99bdcdaf5cbull, 0xf281773c59ffb13aull,
    0xf5257d152486cc2cull, 0xf7d0df730ad13bb9ull, 0xfa83b2db722a033aull, 0xfd3e0c0cf486c175ull,
};

// e^(-a) (negate) or e^(+a) for a = A 2^-E, 2 <= E <= 64, as an Fx (value m 2^(e - 64));
// tab: kExp2Fixed staged in shared memory.  |u| beyond 4096 saturates (e^-a to zero, e^a
// to an exponent that fx_to_double_sat turns into infinity).
__device__ __forceinline__ Fx exp_fixed(uint64_t A, int E, bool negate, const uint64_t *tab) {
    constexpr uint64_t kLog2e = 0xb8aa3b295c17f0bcull;   // log2(e) 2^63
    constexpr uint64_t kLn2 = 0xb17217f7d1cf79acull;     // ln2 2^64
    constexpr uint64_t kD3 = 0x0002aaaaaaaaaaabull;      // 2^-12 / 6
    constexpr uint64_t kD4 = 0x000002aaaaaaaaabull;      // 2^-18 / 24
    constexpr uint64_t kD5 = 0x0000000222222222ull;      // 2^-24 / 120
    constexpr uint64_t kD6 = 0x00000000016c16c1ull;      // 2^-30 / 720
    constexpr uint64_t kD2 = 0x0200000000000000ull;      // 2^-6 / 2
    const uint64_t lo = A * kLog2e, hi = __umul64hi(A, kLog2e);   // u 2^(E + 63)
    const int sh = E - 1;                                          // 1..63
    uint64_t k = hi >> sh;
    uint64_t F = (hi << (64 - sh)) | (lo >> sh);
    if (k > 4096) k = 4096;
    int ke = (int)k;
    if (negate) {
        ke = -ke - (F != 0);
        F = 0 - F;
    }
    const uint64_t rho = F << 6;
    const uint64_t Y = mulhi_trunc(rho, kLn2);                     // y 2^70
    uint64_t G = kD6;
    G = kD5 + mulhi_trunc(G, Y);
    G = kD4 + mulhi_trunc(G, Y);
    G = kD3 + mulhi_trunc(G, Y);
    G = kD2 + mulhi_trunc(G, Y);
    const uint64_t em1 = Y + mulhi_trunc(Y, mulhi_trunc(Y, G));     // (e^y - 1) 2^70
    const uint64_t t = tab[F >> 58];
    return Fx{t + (mulhi_trunc(t, em1) >> 6), ke + 1};
}

// tab: 2^(j/32), j = 0..31, staged in shared memory (exp2_table_entry).
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

// 2^(j/32) as the correctly rounded double: entry 2j of kExp2Fixed rounded to 53 bits.
__device__ __forceinline__ double exp2_table_entry(int j) {
    return __ull2double_rn(kExp2Fixed[2 * j]) * 0x1p-63;
}

}  // namespace qmc
