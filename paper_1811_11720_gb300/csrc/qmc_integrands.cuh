// qmc_integrands.cuh -- integrand families as device code.
//
// Genz families (Sec. 5.2, table of test functions), the minimal example of Sec. 3.2, a
// trigonometric product used by the lattice-exactness tests, and the polynomial
// (sector-like) families.  Separable families are evaluated while the coordinates are
// produced (FamilyAcc::add per dimension), so no coordinate array is kept; the polynomial
// families store x in registers and evaluate U and F in finish().
#pragma once
#include <cstdint>

#include "qmc_fp.cuh"
#include "qmc_params.cuh"
#include "qmc_poly.cuh"

namespace qmc {

struct FamilyShared {
    double c[kMaxDim], w[kMaxDim], aux[kMaxDim];
    double s0;
    int64_t h[kMaxDim];
    PolyShared poly;
};

template <int FAM>
__device__ __forceinline__ void stage_family(const SumsParams &p, FamilyShared &fs) {
    const int tid = threadIdx.x;
    if constexpr (FAM == QMC_SECTOR || FAM == QMC_FEYNMAN) {
        stage_poly(p, fs.poly);
    } else {
        if (tid < p.d) {
            double c = p.c ? p.c[tid] : 0.0;
            double w = p.w ? p.w[tid] : 0.0;
            fs.c[tid] = c;
            fs.w[tid] = w;
            if constexpr (FAM == QMC_GENZ_PRODUCT_PEAK) fs.aux[tid] = 1.0 / (c * c);
            fs.h[tid] = p.h ? p.h[tid] : 0;
        }
        if (tid == 0) fs.s0 = (FAM == QMC_GENZ_OSCILLATORY && p.w) ? 6.283185307179586476925 * p.w[0] : 0.0;
    }
}

template <int FAM>
struct FamilyAcc;

// 1: cos(2 pi w_1 + sum c_i x_i)
template <>
struct FamilyAcc<QMC_GENZ_OSCILLATORY> {
    static constexpr bool kComplex = false;
    double s;
    __device__ __forceinline__ void init(const FamilyShared &fs) { s = fs.s0; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) { s = fma(fs.c[j], x, s); }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = cos(s);
        im = 0.0;
    }
};

// 2: prod (c_i^-2 + (x_i - w_i)^2)^-1, one reciprocal per evaluation
template <>
struct FamilyAcc<QMC_GENZ_PRODUCT_PEAK> {
    static constexpr bool kComplex = false;
    double prod;
    __device__ __forceinline__ void init(const FamilyShared &) { prod = 1.0; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) {
        double t = x - fs.w[j];
        prod *= fma(t, t, fs.aux[j]);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = 1.0 / prod;
        im = 0.0;
    }
};

// 3: (1 + sum c_i x_i)^-(d+1)
template <>
struct FamilyAcc<QMC_GENZ_CORNER_PEAK> {
    static constexpr bool kComplex = false;
    double s;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 1.0; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) { s = fma(fs.c[j], x, s); }
    __device__ __forceinline__ void finish(int d, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = 1.0 / ipow_u(s, d + 1);
        im = 0.0;
    }
};

// 4: exp(-sum c_i^2 (x_i - w_i)^2)
template <>
struct FamilyAcc<QMC_GENZ_GAUSSIAN> {
    static constexpr bool kComplex = false;
    double s;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) {
        double q = fs.c[j] * (x - fs.w[j]);
        s = fma(q, q, s);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = exp(-s);
        im = 0.0;
    }
};

// 5: exp(-sum c_i |x_i - w_i|)
template <>
struct FamilyAcc<QMC_GENZ_C0> {
    static constexpr bool kComplex = false;
    double s;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) {
        s = fma(fs.c[j], fabs(x - fs.w[j]), s);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = exp(-s);
        im = 0.0;
    }
};

// 6: 0 if x_1 > w_1 or x_2 > w_2, else exp(sum c_i x_i)
template <>
struct FamilyAcc<QMC_GENZ_DISCONTINUOUS> {
    static constexpr bool kComplex = false;
    double s;
    bool zero;
    __device__ __forceinline__ void init(const FamilyShared &) { s = 0.0; zero = false; }
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) {
        if (j < 2) zero |= gt_nonneg(x, fs.w[j]);
        s = fma(fs.c[j], x, s);
    }
    __device__ __forceinline__ void finish(int, const FamilyShared &, double &re, double &im,
                                           unsigned long long &) {
        re = zero ? 0.0 : exp(s);
        im = 0.0;
    }
};

// 10: prod x_i
template <>
struct FamilyAcc<QMC_MONOMIAL> {
    static constexpr bool kComplex = false;
    double prod;
    __device__ __forceinline__ void init(const FamilyShared &) { prod = 1.0; }
    __device__ __forceinline__ void add(int, double x, const FamilyShared &) { prod *= x; }
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
    __device__ __forceinline__ void add(int j, double x, const FamilyShared &fs) {
        double a = fma((double)fs.h[j], x, fs.w[j]);
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
    __device__ __forceinline__ void add(int j, double xv, const FamilyShared &) { x[j] = xv; }
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
    __device__ __forceinline__ void add(int j, double xv, const FamilyShared &) { x[j] = xv; }
    __device__ __forceinline__ void finish(int d, const FamilyShared &fs, double &re, double &im,
                                           unsigned long long &signfail) {
        feynman_value(x, d, fs.poly, re, im, signfail);
    }
};

}  // namespace qmc
