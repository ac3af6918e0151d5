// qmc_poly.cuh -- polynomial (Feynman-parameter-like) integrands.
//
// U and F are sums of monomials c prod_k x_k^e_k.  Each monomial is stored as a packed
// factor list (low nibble: degree, then one nibble per factor: the variable index), so a
// monomial of degree q costs q - 1 multiplies plus one fused multiply-add.
//
// QMC_FEYNMAN evaluates, at the real point x (after transform and fit),
//   z_k = x_k - i lam x_k (1 - x_k) dF/dx_k(x),
//   J_kl = dz_k/dx_l = delta_kl - i lam [delta_kl (1 - 2 x_k) dF_k + x_k (1 - x_k) d2F_kl],
//   f = U(z)^a F(z)^-b det J   (principal branch),
// the contour deformation used for Feynman-parameter integrals with an F that changes sign
// (the "F - i delta" prescription realised by the deformation).  J = I - i lam (D H + E)
// with D = diag(x (1 - x)), E = diag((1 - 2x) dF) and H the (symmetric) Hessian of F.  The
// diagonal similarity D^(1/2) (.) D^(-1/2) maps J to I - i lam (D^(1/2) H D^(1/2) + E),
// whose Hermitian part is I; leading principal minors, hence the pivots of Gaussian
// elimination, are unchanged by the similarity, so elimination on J without pivoting
// cannot break down (every pivot has real part >= 1 in the symmetrised form) and
// det J is the product of the pivots.
#pragma once
#include <cstdint>

#include "qmc_params.cuh"

namespace qmc {

constexpr int kMaxTerms = QMC_MAX_TERMS;

struct PolyShared {
    int nu, nf, d;
    double pa, pb, lam;
    double ucoef[kMaxTerms], fcoef[kMaxTerms];
    uint64_t umono[kMaxTerms], fmono[kMaxTerms];
};

__device__ __forceinline__ uint64_t pack_monomial(const int32_t *e, int d) {
    uint64_t code = 0;
    int deg = 0;
    for (int k = 0; k < d; ++k)
        for (int q = 0; q < e[k] && deg < 15; ++q) {
            code |= (uint64_t)k << (4 * (deg + 1));
            ++deg;
        }
    return code | (uint64_t)deg;
}

template <class P>
__device__ __forceinline__ void stage_poly(const P &p, PolyShared &ps) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        ps.nu = p.nu;
        ps.nf = p.nf;
        ps.d = p.d;
        ps.pa = p.pa;
        ps.pb = p.pb;
        ps.lam = p.lam;
    }
    for (int q = tid; q < p.nu; q += blockDim.x) {
        ps.ucoef[q] = p.ucoef[q];
        ps.umono[q] = pack_monomial(p.uexp + (size_t)q * p.d, p.d);
    }
    for (int q = tid; q < p.nf; q += blockDim.x) {
        ps.fcoef[q] = p.fcoef[q];
        ps.fmono[q] = pack_monomial(p.fexp + (size_t)q * p.d, p.d);
    }
}

// Real polynomial value at x (x indexed at run time: x lives in local memory).
__device__ __forceinline__ double poly_real(const double *x, int nterm, const double *coef,
                                            const uint64_t *mono) {
    double s = 0.0;
#pragma unroll 1
    for (int q = 0; q < nterm; ++q) {
        uint64_t code = mono[q];
        int deg = (int)(code & 15u);
        double t = 1.0;
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t *= x[(code >> (4 * f)) & 15u];
        s = fma(coef[q], t, s);
    }
    return s;
}

// x^y for x > 0 (library pow for non-integer exponents).
__device__ __forceinline__ double pow_pos(double x, double y) {
    if (y == 1.0) return x;
    if (y == -1.0) return 1.0 / x;
    return pow(x, y);
}

__device__ __forceinline__ double sector_value(const double *xin, int d, const PolyShared &ps) {
    double x[kMaxDim];
#pragma unroll
    for (int k = 0; k < kMaxDim; ++k) x[k] = xin[k];
    double U = poly_real(x, ps.nu, ps.ucoef, ps.umono);
    double F = poly_real(x, ps.nf, ps.fcoef, ps.fmono);
    return pow_pos(U, ps.pa) * pow_pos(F, -ps.pb);
}

// ---- complex helpers --------------------------------------------------------------------
struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cplx crecip(cplx a) {
    // scaled to avoid overflow of |a|^2 for the magnitudes met here (|a| in 1e-150..1e150)
    double s = 1.0 / fma(a.re, a.re, a.im * a.im);
    return {a.re * s, -a.im * s};
}

// principal a^p for real p: exp(p Log a)
__device__ __forceinline__ cplx cpow_real(cplx a, double p) {
    if (p == 1.0) return a;
    double r = hypot(a.re, a.im);
    double th = atan2(a.im, a.re);
    double lr = log(r);
    double mag = exp(p * lr);
    double s, c;
    sincos(p * th, &s, &c);
    return {mag * c, mag * s};
}

static __device__ __noinline__ void feynman_value(const double *xin, int d, const PolyShared &ps,
                                           double &re, double &im,
                                           unsigned long long &signfail) {
    double x[kMaxDim];
    double grad[kMaxDim];
    double H[kMaxDim * kMaxDim];
#pragma unroll 1
    for (int k = 0; k < d; ++k) {
        x[k] = xin[k];
        grad[k] = 0.0;
    }
#pragma unroll 1
    for (int q = 0; q < d * d; ++q) H[q] = 0.0;
    // value is not needed; gradient and Hessian of F at the real point
#pragma unroll 1
    for (int q = 0; q < ps.nf; ++q) {
        uint64_t code = ps.fmono[q];
        int deg = (int)(code & 15u);
        double c = ps.fcoef[q];
        // factor list v_1..v_deg; derivative w.r.t. factor a: product of the others
#pragma unroll 1
        for (int a = 1; a <= deg; ++a) {
            int ka = (int)((code >> (4 * a)) & 15u);
            double pa = c;
#pragma unroll 1
            for (int f = 1; f <= deg; ++f)
                if (f != a) pa *= x[(code >> (4 * f)) & 15u];
            grad[ka] += pa;
#pragma unroll 1
            for (int b = a + 1; b <= deg; ++b) {
                int kb = (int)((code >> (4 * b)) & 15u);
                double pab = c;
#pragma unroll 1
                for (int f = 1; f <= deg; ++f)
                    if (f != a && f != b) pab *= x[(code >> (4 * f)) & 15u];
                H[ka * d + kb] += pab;
                H[kb * d + ka] += pab;
            }
        }
    }
    const double lam = ps.lam;
    cplx z[kMaxDim];
    double xo[kMaxDim];   // x (1 - x)
#pragma unroll 1
    for (int k = 0; k < d; ++k) {
        xo[k] = x[k] * (1.0 - x[k]);
        z[k] = {x[k], -lam * xo[k] * grad[k]};
    }
    // U(z), F(z)
    cplx U = {0.0, 0.0}, F = {0.0, 0.0};
#pragma unroll 1
    for (int q = 0; q < ps.nu; ++q) {
        uint64_t code = ps.umono[q];
        int deg = (int)(code & 15u);
        cplx t = {1.0, 0.0};
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t = cmul(t, z[(code >> (4 * f)) & 15u]);
        U.re = fma(ps.ucoef[q], t.re, U.re);
        U.im = fma(ps.ucoef[q], t.im, U.im);
    }
#pragma unroll 1
    for (int q = 0; q < ps.nf; ++q) {
        uint64_t code = ps.fmono[q];
        int deg = (int)(code & 15u);
        cplx t = {1.0, 0.0};
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t = cmul(t, z[(code >> (4 * f)) & 15u]);
        F.re = fma(ps.fcoef[q], t.re, F.re);
        F.im = fma(ps.fcoef[q], t.im, F.im);
    }
    if (F.im > 0.0) ++signfail;
    // J_kl = delta_kl - i lam [delta_kl (1 - 2 x_k) dF_k + x_k (1 - x_k) d2F_kl]; Gaussian
    // elimination without pivoting, det = product of the pivots.
    cplx A[kMaxDim * kMaxDim];
#pragma unroll 1
    for (int k = 0; k < d; ++k)
#pragma unroll 1
        for (int l = 0; l < d; ++l) {
            double mkl = xo[k] * H[k * d + l];
            if (k == l) mkl = fma(1.0 - 2.0 * x[k], grad[k], mkl);
            A[k * d + l] = {(k == l) ? 1.0 : 0.0, -lam * mkl};
        }
    cplx det = {1.0, 0.0};
#pragma unroll 1
    for (int c = 0; c < d; ++c) {
        cplx piv = A[c * d + c];
        det = cmul(det, piv);
        if (c + 1 == d) break;
        cplx inv = crecip(piv);
#pragma unroll 1
        for (int r = c + 1; r < d; ++r) {
            cplx l = cmul(A[r * d + c], inv);
#pragma unroll 1
            for (int q = c + 1; q < d; ++q) {
                cplx a = A[c * d + q];
                cplx &t = A[r * d + q];
                t.re -= fma(l.re, a.re, -l.im * a.im);
                t.im -= fma(l.re, a.im, l.im * a.re);
            }
        }
    }
    cplx Ua = cpow_real(U, ps.pa);
    cplx Fb = cpow_real(F, -ps.pb);
    cplx v = cmul(cmul(Ua, Fb), det);
    re = v.re;
    im = v.im;
}

}  // namespace qmc
