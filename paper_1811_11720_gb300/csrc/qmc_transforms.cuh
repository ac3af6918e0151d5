// qmc_transforms.cuh -- periodizing transforms (Sec. 2.3) and the PolySingular
// variance-reduction map (Sec. 2.4, Eq. (ISfit)) as device functions.
//
// FP64 is the scarce unit on GB300, so every step that is exact in integer arithmetic is
// done on the integer pipe: comparisons of non-negative doubles are integer comparisons
// of their bit patterns, 1 - u for u >= 1/2 (exact by Sterbenz' lemma) and multiplication
// by 2 are bit manipulations.  The symmetric Korobov maps r <= 6, baker and the identity
// also have a fixed-point form (transform_fixed; Korobov in qmc_fixed.cuh) that hands the
// integrand x in 0.64 fixed point; the FP64 forms here serve the other transforms, the
// fitted rules and the integrands without a fixed-point form.
//
// A transform returns the mapped coordinate in reflected form: x = y (refl == false) or
// x = 1 - y (refl == true), with y <= 1/2 for the symmetric maps.  Evaluating the Korobov
// polynomial on v = min(u, 1 - u) keeps relative accuracy at both ends of [0, 1], and the
// integrands fold the reflection into their own per-dimension fused multiply-add instead
// of spending an FP64 subtraction on 1 - y.
#pragma once
#include <cstdint>

#include "qmc_fixed.cuh"
#include "qmc_fp.cuh"
#include "qmc_params.cuh"

namespace qmc {

// Per-evaluation weight accumulator.
//  * Korobov<r,r>: w = C^d prod_j (v_j (1 - v_j))^r, kept as prod_j t_j with
//    t_j = v_j (1 - v_j) (one fused multiply-add) and raised to r once per evaluation.
//  * Korobov<r0,r1>: prod u_j and prod (1 - u_j), raised to r0 and r1 once.
//  * w: other factors (fit Jacobian, Sidi weights).
//  * wp: integer-pipe Korobov<r,r>, prod_j t_j as a normalized Fx.
struct Weight {
    double wu, w1, w;
    Fx wp;
};

struct Mapped {
    double y;
    bool refl;
};

__device__ __forceinline__ double reflected(const Mapped &m) { return m.refl ? 1.0 - m.y : m.y; }

template <int TK>
__device__ __forceinline__ Mapped apply_transform(double u, const TransformParams &t, Weight &W) {
    if constexpr (TK == QMC_T_NONE) {
        return {u, false};
    } else if constexpr (TK == QMC_T_BAKER) {
        // phi(u) = 2u for u <= 1/2, 2 - 2u = 2 (1 - u) otherwise (Eq. (baker)); weight 1.
        return {twice(le_half(u) ? u : one_minus_upper(u)), false};
    } else if constexpr (TK == QMC_T_KOROBOV) {
        // phi(u) = v^(e) P(v) with v = u (u <= 1/2, e = r0+1, P = A) or v = 1 - u (reflected,
        // e = r1+1, P = B); Eq. (korobov) integrated term by term (coefficients on the host).
        const bool lo = le_half(u);
        const double v = lo ? u : one_minus_upper(u);
        double P = lo ? t.A[t.deg] : t.B[t.deg];
#pragma unroll 1
        for (int q = t.deg - 1; q >= 0; --q) P = fma(P, v, lo ? t.A[q] : t.B[q]);
        const double y = ipow_u(v, lo ? t.r0 + 1 : t.r1 + 1) * P;
        if (t.r0 == t.r1) {
            W.wu *= fma(-v, v, v);            // v (1 - v) = u (1 - u)
        } else {
            const double w1v = 1.0 - v;       // rounded for v < 1/2
            W.wu *= lo ? v : w1v;             // u
            W.w1 *= lo ? w1v : v;             // 1 - u
        }
        return {y, !lo};
    } else {
        static_assert(TK == QMC_T_SIDI, "kTKorobovInt is evaluated by korobov_int_x");
        // phi = cr I_r(u), I_r = base I_(r mod 2) - (cos(pi u)/pi) sum_q a_q sin^(r-1-2q)
        double s, c;
        sincospi(u, &s, &c);
        const int r = t.r0;
        const double s2 = s * s;
        // sum_{q < nq} a_q s^(r-1-2q), nq = floor(r/2): Horner in s^2 on a_0..a_(nq-1)
        // (sidi_c[q] = a_q, zero when nq = 0), then one factor s (r even: powers
        // r-1, ..., 1) or s^2 (r odd: powers r-1, ..., 2).
        double poly = t.sidi_c[0];
        const int nq = r / 2;
#pragma unroll 1
        for (int q = 1; q < nq; ++q) poly = fma(poly, s2, t.sidi_c[q]);
        poly *= (r & 1) ? s2 : s;
        double base = (r & 1) ? (1.0 - c) * 0.31830988618379067154 : u;
        double I = t.sidi_c[kMaxSidi] * base - c * 0.31830988618379067154 * poly;
        double sr = ipow_u(s, r);
        W.w *= t.C * sr;
        return {t.C * I, false};
    }
}

// The integer-pipe Korobov<R,R> (kTKorobovInt) takes the lattice state's top word
// X = x 2^64 instead of the rounded u: v = min(x, 1 - x) in 0.64 fixed point.
template <int R>
__device__ __forceinline__ Mapped korobov_int_x(uint64_t X, Weight &W) {
    const bool lo = !(X >> 63);
    return {fixed_to_double64(korobov_phi_fixed<R>(lo ? X : ~X, W.wp)), !lo};
}

// Transforms that are exact or fixed-point on the integer pipe can hand the integrand the
// coordinate itself in 0.64 fixed point, x 2^64 (truncated), when the integrand takes it
// (FamilyAcc::add_fixed): none (x is the shifted lattice fraction), baker (2 min(x, 1 - x))
// and the integer Korobov (phi, or 1 - phi when reflected).
template <int TK>
constexpr bool kFixedTransform = TK == QMC_T_NONE || TK == QMC_T_BAKER || TK == kTKorobovInt;

template <int TK, int R>
__device__ __forceinline__ uint64_t transform_fixed(uint64_t X, Weight &W) {
    if constexpr (TK == QMC_T_NONE) {
        return X;
    } else if constexpr (TK == QMC_T_BAKER) {
        return ((X >> 63) ? ~X : X) << 1;   // min(X, 2^64 - 1 - X) < 2^63
    } else {
        static_assert(TK == kTKorobovInt, "no fixed-point form");
        const bool lo = !(X >> 63);
        const uint64_t F = korobov_phi_fixed<R>(lo ? X : ~X, W.wp);
        return lo ? F : ~F;
    }
}

// cd = C^d for Korobov (folded once per launch).
template <int TK, int R = 0>
__device__ __forceinline__ double weight_finish(const Weight &W, const TransformParams &t,
                                                double cd) {
    if constexpr (TK == QMC_T_KOROBOV) {
        if (t.r0 == t.r1) return cd * ipow_u(W.wu, t.r0) * W.w;
        return cd * ipow_u(W.wu, t.r0) * ipow_u(W.w1, t.r1) * W.w;
    } else if constexpr (TK == kTKorobovInt) {
        return korobov_weight_fixed<R>(W.wp, fx_of_double(cd)) * W.w;
    } else {
        return W.w;
    }
}

// PolySingular map p(x) and p'(x) (Eq. (ISfit) with |a2|, |a3| as in App. A.5).  fp holds
// per-dimension constants prepared in shared memory:
//   [0] a0, [1] a1, [2] |a2| (a0 - 1), [3] |a3| (a1 - 1), [4] a4, [5] a5,
//   [6] a6 = 1 - |a2| - |a3| - a4 - a5, [7] |a2| (a0 - 1) a0, [8] |a3| (a1 - 1) a1,
//   [9] 2 a5, [10] 3 a6 (the derivative's coefficients).
constexpr int kFitStride = 11;

__device__ __forceinline__ double apply_fit(double x, const double *fp, double &jac) {
    const double d0 = fp[0] - x;
    const double d1 = fp[1] - x;
    const double inv = 1.0 / (d0 * d1);
    const double r0 = d1 * inv;   // 1 / (a0 - x)
    const double r1 = d0 * inv;   // 1 / (a1 - x)
    const double poly = fma(fma(fp[6], x, fp[5]), x, fp[4]);
    const double p = x * fma(fp[2], r0, fma(fp[3], r1, poly));
    const double dpoly = fma(fma(fp[10], x, fp[9]), x, fp[4]);
    const double dp = fma(fp[7] * r0, r0, fma(fp[8] * r1, r1, dpoly));
    jac *= dp;
    return p;
}

}  // namespace qmc
