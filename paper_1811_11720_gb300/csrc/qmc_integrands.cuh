// qmc_integrands.cuh -- integrand families as device code.
//
// Genz families (Sec. 5.2, table of test functions), the minimal example of Sec. 3.2, a
// trigonometric product used by the lattice-exactness tests, and the polynomial
// (sector-like) families.  Separable families are evaluated while the coordinates are
// produced (FamilyAcc::add per dimension), so no coordinate array is kept; the polynomial
// families store x and evaluate U and F in finish().
//
// add() receives the coordinate in reflected form (x = y or x = 1 - y, see
// qmc_transforms.cuh).  The Genz families fold the reflection into their own fused
// multiply-add with per-dimension constants staged in shared memory:
//   c (x - w) = (+-c) y + (-c w  or  c (1 - w)),
// and for the linear forms sum c_j x_j the constant part, the sum of c_j over reflected
// dimensions, is read from two 256-entry subset-sum tables (dimensions 0-7 and 8-15)
// indexed by the reflection bit mask.
#pragma once
#include <cstdint>

#include "qmc_cos.cuh"
#include "qmc_exp.cuh"
#include "qmc_fp.cuh"
#include "qmc_params.cuh"
#include "qmc_poly.cuh"
#include "qmc_transforms.cuh"

namespace qmc {

// Fixed-point constants of the separable Genz families 1-6, whose linear and quadratic
// forms run on the integer pipe when the coordinate arrives in 0.64 fixed point:
//   linear (1, 3, 5, 6): cl_j = c_j 2^S with S = 62 - floor(log2 sum_j c_j), so every
//     partial sum of c_j x_j (or c_j |x_j - w_j|) stays below 2^63;
//   Gaussian (4) and product peak (2): cq_j = c_j 2^S with S = 61 - floor(log2 max_j c_j),
//     so |c_j (x_j - w_j)| 2^S < 2^62 and each square (2^(2S - 64) scale) is below 2^60.
//     A square keeps only 2S - 64 fractional bits, so these forms need S >= 57 (max c < 32,
//     at least 50 fractional bits); the product peak also caps S at 62, so that 1 at the
//     square's scale, one = 2^(2S - 64), is at most 2^60 and 1 + q_j^2 fits below 2^61.
// S is capped at 64 otherwise (small c keep 2^-64 absolute precision), so that the
// exponential's argument scale, S or 2S - 64, lies in [2, 64] (exp_fixed).
// Each term truncates by at most three units (2^-S, or 2^(64 - 2S) for squares); the forms
// are therefore exact to ~2^-48 absolutely or better.  ok is false (double path) unless
// every c_j >= 0 and 0 <= w_j <= 1.
//   oscillatory (1), integer finish: the phase in turns, (w_1 + sum_j c_j x_j / (2 pi)) mod 1
//     as a 64-bit fraction: c_j / (2 pi) = tk_j + tg_j 2^-64 (integer and fraction parts,
//     from a double-double product), so each term is tk_j X_j + floor(tg_j X_j 2^-64) mod
//     2^64 and the wrap of the 64-bit sum is the reduction mod 1.
struct FixedForms {
    uint64_t cl[kMaxDim];
    uint64_t cq[kMaxDim];
    uint64_t w64[kMaxDim];   // w_j 2^64, at most 2^64 - 1
    uint64_t tk[kMaxDim];    // oscillatory: integer part of c_j / (2 pi)
    uint64_t tg[kMaxDim];    // oscillatory: fraction of c_j / (2 pi), 2^64 scale
    uint64_t t0;             // oscillatory: w_1 2^64 mod 2^64
    bool tk_any;             // oscillatory: some c_j >= 2 pi (a nonzero integer part)
    uint64_t one;            // 2^(2S - 64) (product peak)
    double num;              // prod_j c_j^2 (product peak)
    Fx numx;                 // the same as Fx (zero or normal)
    int S;
    bool ok;
};

struct FamilyShared {
    double c[kMaxDim], w[kMaxDim], aux[kMaxDim];
    double mcw[kMaxDim];    // -c w
    double c1w[kMaxDim];    // c (1 - w)
    double w1[kMaxDim];     // 1 - w
    double sub_lo[256];     // sum of c_j over the set bits j of the index, j < 8
    double sub_hi[256];     // the same for j = 8 + bit
    double s0;
    int64_t h[kMaxDim];
    union {
        uint64_t exp2q[64];     // 2^(j/64) 2^63 for exp_fixed (families with an exponential)
        uint64_t cos256[65];    // cos(2 pi i/256) 2^62 for cos_turns_fixed (oscillatory)
    };
    double exp2t[32];       // 2^(j/32) for exp_table
    FixedForms fx;
    PolyShared poly;
};

template <int FAM>
constexpr bool kHasFixedForm = FAM == QMC_GENZ_OSCILLATORY || FAM == QMC_GENZ_PRODUCT_PEAK ||
                               FAM == QMC_GENZ_CORNER_PEAK || FAM == QMC_GENZ_GAUSSIAN ||
                               FAM == QMC_GENZ_C0 || FAM == QMC_GENZ_DISCONTINUOUS;

// v 2^-S for an integer v < 2^64, rounded once (the power of two is exact; v 2^-S is normal).
__device__ __forceinline__ double scaled_fixed(uint64_t v, int S) {
    const long long b = __double_as_longlong(__ull2double_rn(v));
    return __longlong_as_double(b ? b - ((long long)S << 52) : 0ll);
}

// Per-thread staging of the fixed-point constants (threads tid < d; thread 0 writes S, ok).
template <int FAM, class P>
__device__ __forceinline__ void stage_fixed_forms(const P &p, FixedForms &fx) {
    const int tid = threadIdx.x;
    if (tid >= p.d) return;
    double csum = 0.0, cmax = 0.0;
    bool ok = p.c != nullptr && (p.w != nullptr || FAM == QMC_GENZ_OSCILLATORY ||
                                 FAM == QMC_GENZ_CORNER_PEAK);
    for (int i = 0; ok && i < p.d; ++i) {
        const double c = p.c[i];
        const double w = p.w ? p.w[i] : 0.0;
        ok = c >= 0.0 && w >= 0.0 && w <= 1.0 && (FAM != QMC_GENZ_OSCILLATORY || c < 0x1p40);
        csum += c;
        cmax = fmax(cmax, c);
    }
    int S;
    if constexpr (FAM == QMC_GENZ_GAUSSIAN) {
        S = cmax > 0.0 ? min(61 - ilogb(cmax), 64) : 64;
        ok = ok && S >= 57;
    } else if constexpr (FAM == QMC_GENZ_PRODUCT_PEAK) {
        S = cmax > 0.0 ? min(61 - ilogb(cmax), 62) : 62;
        ok = ok && S >= 57;
    } else {
        S = csum > 0.0 ? min(62 - ilogb(csum), 64) : 64;
    }
    ok = ok && S >= 2;
    if (ok) {
        const double c = p.c[tid];
        const double w = p.w ? p.w[tid] : 0.0;
        fx.cl[tid] = __double2ull_rz(ldexp(c, S));
        fx.cq[tid] = __double2ull_rz(ldexp(c, S));
        fx.w64[tid] = w >= 1.0 ? 0xFFFFFFFFFFFFFFFFull : __double2ull_rz(ldexp(w, 64));
        if constexpr (FAM == QMC_GENZ_OSCILLATORY) {
            // c / (2 pi) = hi + lo (double-double), then integer part and 64-bit fraction
            constexpr double kInv2PiHi = 0x1.45f306dc9c883p-3;
            constexpr double kInv2PiLo = -0x1.6b01ec5417056p-57;
            const double hi = c * kInv2PiHi;
            const double lo = fma(c, kInv2PiHi, -hi) + c * kInv2PiLo;
            double k = floor(hi);
            const double f = hi - k;                                  // exact, in [0, 1)
            long long g_lo = llrint(ldexp(lo, 64));                   // |lo| 2^64 < 2^12 hi
            uint64_t g = __double2ull_rz(ldexp(f, 64)) + (uint64_t)g_lo;
            // a carry out of (or borrow into) the fraction moves the integer part
            if (g_lo < 0 && g > __double2ull_rz(ldexp(f, 64))) k -= 1.0;
            if (g_lo > 0 && g < __double2ull_rz(ldexp(f, 64))) k += 1.0;
            fx.tg[tid] = g;
            fx.tk[tid] = (uint64_t)(long long)k;
        }
    }
    if (tid == 0) {
        if constexpr (FAM == QMC_GENZ_OSCILLATORY) {
            const double w1 = p.w ? p.w[0] : 0.0;
            fx.t0 = ok ? (w1 >= 1.0 ? 0ull : __double2ull_rz(ldexp(w1, 64))) : 0ull;
            fx.tk_any = cmax >= 6.283185307179586;
        }
        if constexpr (FAM == QMC_GENZ_PRODUCT_PEAK) {
            double num = 1.0;
            for (int i = 0; ok && i < p.d; ++i) num *= p.c[i] * p.c[i];
            ok = ok && (num == 0.0 || num >= 0x1p-1022);   // Fx takes zero or normal values
            fx.num = num;
            fx.numx = fx_of_double(ok ? num : 0.0);
            fx.one = ok ? 1ull << (2 * S - 64) : 0ull;
        }
        fx.S = S;
        fx.ok = ok;
    }
}

// Subset sums of c over the reflected dimensions, for the FP64 forms of families 1, 3
// and 6 (reflected_c_sum); the fixed-point forms do not read them.
template <int FAM, class P>
__device__ __forceinline__ void stage_subset_sums(const P &p, FamilyShared &fs) {
    if constexpr (FAM == QMC_GENZ_OSCILLATORY || FAM == QMC_GENZ_CORNER_PEAK ||
                  FAM == QMC_GENZ_DISCONTINUOUS) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) {
            double lo = 0.0, hi = 0.0;
            for (int j = 0; j < 8; ++j) {
                if ((b >> j) & 1) {
                    if (j < p.d) lo += p.c[j];
                    if (j + 8 < p.d) hi += p.c[j + 8];
                }
            }
            fs.sub_lo[b] = lo;
            fs.sub_hi[b] = hi;
        }
    }
}

// P: SumsParams or BatchItem (fields d, c, w, h, nu, nf, ucoef, fcoef, uexp, fexp, pa, pb, lam).
// kSubsets = false leaves the subset-sum tables to the caller (stage_subset_sums), which
// builds them only when an FP64 form may run.
template <int FAM, bool kSubsets = true, class P>
__device__ __forceinline__ void stage_family(const P &p, FamilyShared &fs) {
    const int tid = threadIdx.x;
    if constexpr (FAM == QMC_SECTOR || FAM == QMC_FEYNMAN) {
        stage_poly(p, fs.poly, FAM == QMC_SECTOR);
    } else {
        if (tid < p.d) {
            double c = p.c ? p.c[tid] : 0.0;
            double w = p.w ? p.w[tid] : 0.0;
            fs.c[tid] = c;
            fs.w[tid] = w;
            fs.mcw[tid] = -(c * w);
            fs.c1w[tid] = c * (1.0 - w);
            fs.w1[tid] = 1.0 - w;
            if constexpr (FAM == QMC_GENZ_PRODUCT_PEAK) fs.aux[tid] = 1.0 / (c * c);
            fs.h[tid] = p.h ? p.h[tid] : 0;
        }
        if (tid == 0) fs.s0 = (FAM == QMC_GENZ_OSCILLATORY && p.w) ? 6.283185307179586476925 * p.w[0] : 0.0;
        if constexpr (kSubsets) stage_subset_sums<FAM>(p, fs);
        if constexpr (kHasFixedForm<FAM>) stage_fixed_forms<FAM>(p, fs.fx);
        if constexpr (FAM == QMC_GENZ_OSCILLATORY) {
            for (int i = tid; i < 65; i += blockDim.x) fs.cos256[i] = kCos256[i];
        }
        if constexpr (FAM == QMC_GENZ_GAUSSIAN || FAM == QMC_GENZ_C0 ||
                      FAM == QMC_GENZ_DISCONTINUOUS) {
            for (int i = tid; i < 64; i += blockDim.x) fs.exp2q[i] = kExp2Fixed[i];
            for (int i = tid; i < 32; i += blockDim.x) fs.exp2t[i] = exp2_table_entry(i);
        }
    }
}

template <int FAM>
struct FamilyAcc;

// sum of c_j over reflected dimensions
__device__ __forceinline__ double reflected_c_sum(uint32_t mask, int d, const FamilyShared &fs) {
    double r = fs.sub_lo[mask & 255u];
    if (d > 8) r += fs.sub_hi[(mask >> 8) & 255u];
    return r;
}

// 1: cos(2 pi w_1 + sum c_i x_i)
template <>
struct FamilyAcc<QMC_GENZ_OSCILLATORY> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 4;   // integer finish up to this Korobov order
    double s;
    uint32_t mask;
    __device__ __forceinline__ void init(const FamilyShared &fs) { s = fs.s0; mask = 0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        s = fma(m.refl ? -fs.c[j] : fs.c[j], m.y, s);
        mask |= (uint32_t)m.refl << j;
    }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &) {
        re = cos(mask ? s + reflected_c_sum(mask, d, fs) : s);
        im = 0.0;
    }
    // fixed point: sum c_j x_j on the integer pipe, either scaled by 2^S (then cos in FP64)
    // or, for the integer finish, as the phase in turns mod 1 (FixedForms)
    uint64_t sl;
    __device__ __forceinline__ void init_fixed() { sl = 0; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        if constexpr (kInt) {
            // the integer turns per unit x only when some c_j >= 2 pi (a uniform branch;
            // the Genz ranges have ||c||_1 = 6)
            if (fs.fx.tk_any) sl += x * fs.fx.tk[j];
            sl += mulhi_trunc(x, fs.fx.tg[j]);
        } else {
            sl += mulhi_trunc(x, fs.fx.cl[j]);
        }
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        if constexpr (kInt) re = cos_turns_fixed(sl + fs.fx.t0, fs.cos256);
        else re = cos(fs.s0 + scaled_fixed(sl, fs.fx.S));
        im = 0.0;
    }
};

// 2: prod (c_i^-2 + (x_i - w_i)^2)^-1, one reciprocal per evaluation
template <>
struct FamilyAcc<QMC_GENZ_PRODUCT_PEAK> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 6;   // integer finish up to this Korobov order
    double prod;
    __device__ __forceinline__ void init(const FamilyShared &) { prod = 1.0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        // x - w = y - w, or (1 - w) - y when reflected
        double t = m.refl ? fs.w1[j] - m.y : m.y - fs.w[j];
        prod *= fma(t, t, fs.aux[j]);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = 1.0 / prod;
        im = 0.0;
    }
    // fixed point: f = prod c_j^2 / prod (1 + q_j^2), q_j = c_j |x_j - w_j|; each factor
    // 1 + q_j^2 at scale 2^(2S - 64) (below 2^61, at least 2^50), the product in Fx
    Fx pf;
    __device__ __forceinline__ void init_fixed() { pf = {0x8000000000000000ull, 1}; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        const uint64_t w = fs.fx.w64[j];
        const uint64_t a = x >= w ? x - w : w - x;                       // |x - w| 2^64
        const uint64_t q = mulhi_trunc(a, fs.fx.cq[j]);                 // c |x - w| 2^S
        const uint64_t s = fs.fx.one + sqhi_trunc(q);               // (1 + q^2) 2^(2S-64)
        pf = fx_norm(fx_mul(pf, fx_norm({s, 128 - 2 * fs.fx.S})));
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        // prod c_j^2 times the reciprocal of the product (Newton on the integer pipe), or
        // one FP64 division
        if constexpr (kInt) re = fx_to_double(fx_mul(fs.fx.numx, fx_recip(pf)));
        else re = fs.fx.num / fx_to_double(pf);
        im = 0.0;
    }
};

// 3: (1 + sum c_i x_i)^-(d+1)
template <>
struct FamilyAcc<QMC_GENZ_CORNER_PEAK> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 1;   // integer finish up to this Korobov order
    double s;
    uint32_t mask;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 1.0; mask = 0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        s = fma(m.refl ? -fs.c[j] : fs.c[j], m.y, s);
        mask |= (uint32_t)m.refl << j;
    }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &) {
        const double t = mask ? s + reflected_c_sum(mask, d, fs) : s;
        re = 1.0 / ipow_u(t, d + 1);
        im = 0.0;
    }
    uint64_t sl;
    __device__ __forceinline__ void init_fixed() { sl = 0; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        sl += mulhi_trunc(x, fs.fx.cl[j]);
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int d, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        if constexpr (kInt) {
            // 1 + s as Fx (s = sl 2^-S, sl < 2^63; S = 64 drops sl's lowest bit), its
            // (d+1)-th power and the reciprocal, all on the integer pipe
            const int S = fs.fx.S;
            const Fx b = S <= 63 ? fx_norm_any((1ull << S) + sl, 64 - S)
                                 : Fx{0x8000000000000000ull + (sl >> 1), 1};
            re = fx_to_double(fx_recip(fx_powi(b, d + 1)));
        } else {
            re = 1.0 / ipow_u(1.0 + scaled_fixed(sl, fs.fx.S), d + 1);
        }
        im = 0.0;
    }
};

// 4: exp(-sum c_i^2 (x_i - w_i)^2)
template <>
struct FamilyAcc<QMC_GENZ_GAUSSIAN> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 3;   // integer finish up to this Korobov order
    double s;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        // c (x - w) = c y - c w, or -c y + c (1 - w) when reflected: one fused multiply-add
        const double q = fma(m.refl ? -fs.c[j] : fs.c[j], m.y, m.refl ? fs.c1w[j] : fs.mcw[j]);
        s = fma(q, q, s);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = exp(-s);
        im = 0.0;
    }
    // fixed point: q = c |x - w| 2^S < 2^62, q^2 2^(2S - 64) < 2^60, summed in 64 bits
    uint64_t sq;
    __device__ __forceinline__ void init_fixed() { sq = 0; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        const uint64_t w = fs.fx.w64[j];
        const uint64_t a = x >= w ? x - w : w - x;                       // |x - w| 2^64
        const uint64_t q = mulhi_trunc(a, fs.fx.cq[j]);                 // c |x - w| 2^S
        sq += sqhi_trunc(q);
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        if constexpr (kInt) re = fx_to_double_sat(exp_fixed(sq, 2 * fs.fx.S - 64, true, fs.exp2q));
        else re = exp_table(-scaled_fixed(sq, 2 * fs.fx.S - 64), fs.exp2t);
        im = 0.0;
    }
};

// 5: exp(-sum c_i |x_i - w_i|)
template <>
struct FamilyAcc<QMC_GENZ_C0> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 3;   // integer finish up to this Korobov order
    double s;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        double t = m.refl ? fs.w1[j] - m.y : m.y - fs.w[j];
        s = fma(fs.c[j], fabs(t), s);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = exp(-s);
        im = 0.0;
    }
    uint64_t sl;
    __device__ __forceinline__ void init_fixed() { sl = 0; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        const uint64_t w = fs.fx.w64[j];
        const uint64_t a = x >= w ? x - w : w - x;                       // |x - w| 2^64
        sl += mulhi_trunc(a, fs.fx.cl[j]);
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        if constexpr (kInt) re = fx_to_double_sat(exp_fixed(sl, fs.fx.S, true, fs.exp2q));
        else re = exp_table(-scaled_fixed(sl, fs.fx.S), fs.exp2t);
        im = 0.0;
    }
};

// 6: 0 if x_1 > w_1 or x_2 > w_2, else exp(sum c_i x_i)
template <>
struct FamilyAcc<QMC_GENZ_DISCONTINUOUS> {
    static constexpr bool kComplex = false;
    static constexpr int kIntFinishMaxR = 3;   // integer finish up to this Korobov order
    double s;
    uint32_t mask;
    bool zero;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; mask = 0; zero = false; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        // x > w is y > w, or (1 - y > w, i.e. y < 1 - w) when reflected; w may lie outside
        // [0, 1] here (the fixed-point form covers 0 <= w <= 1), so compare as doubles
        if (j < 2) zero |= m.refl ? (fs.w1[j] > m.y) : (m.y > fs.w[j]);
        s = fma(m.refl ? -fs.c[j] : fs.c[j], m.y, s);
        mask |= (uint32_t)m.refl << j;
    }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &) {
        re = zero ? 0.0 : exp(mask ? s + reflected_c_sum(mask, d, fs) : s);
        im = 0.0;
    }
    uint64_t sl;
    __device__ __forceinline__ void init_fixed() { sl = 0; zero = false; }
    template <bool kInt>
    __device__ __forceinline__ void add_fixed(int j, uint64_t x, const FamilyShared &fs) {
        if (j < 2) zero |= x > fs.fx.w64[j];
        sl += mulhi_trunc(x, fs.fx.cl[j]);
    }
    template <bool kInt>
    __device__ __forceinline__ void finish_fixed(int, const FamilyShared &fs, double &re,
                                                 double &im, unsigned long long &) {
        if constexpr (kInt) re = zero ? 0.0 : fx_to_double_sat(exp_fixed(sl, fs.fx.S, false, fs.exp2q));
        else re = zero ? 0.0 : exp_table(scaled_fixed(sl, fs.fx.S), fs.exp2t);
        im = 0.0;
    }
};

// 10: prod x_i
template <>
struct FamilyAcc<QMC_MONOMIAL> {
    static constexpr bool kComplex = false;
    double prod;
    __device__ __forceinline__ void init(const FamilyShared &) { prod = 1.0; }
    __device__ __forceinline__ void add(int, const Mapped &m, const FamilyShared &) { prod *= reflected(m); }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = prod;
        im = 0.0;
    }
};

// 11: prod (1 + c_i cos(2 pi (h_i x_i + w_i)))
template <>
struct FamilyAcc<QMC_TRIG> {
    static constexpr bool kComplex = false;
    double prod;
    __device__ __forceinline__ void init(const FamilyShared &) { prod = 1.0; }
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &fs) {
        double a = fma((double)fs.h[j], reflected(m), fs.w[j]);
        prod *= fma(fs.c[j], cospi(2.0 * a), 1.0);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = prod;
        im = 0.0;
    }
};

// 21: U(x)^a F(x)^-b, real
template <>
struct FamilyAcc<QMC_SECTOR> {
    static constexpr bool kComplex = false;
    double x[kMaxDim];
    __device__ __forceinline__ void init(const FamilyShared &) {}
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &) { x[j] = reflected(m); }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &) {
        re = sector_value(x, d, fs.poly);
        im = 0.0;
    }
};

// 20: U(z)^a F(z)^-b det(dz/dx) on the deformed contour, complex
template <>
struct FamilyAcc<QMC_FEYNMAN> {
    static constexpr bool kComplex = true;
    double x[kMaxDim];
    __device__ __forceinline__ void init(const FamilyShared &) {}
    __device__ __forceinline__ void add(int j, const Mapped &m, const FamilyShared &) { x[j] = reflected(m); }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &signfail) {
        feynman_value(x, d, fs.poly, re, im, signfail);
    }
};

}  // namespace qmc
