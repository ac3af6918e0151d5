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
constexpr int kDenseCap = 1024;   // >= C(16 + 3, 3) = 969 coefficients of a dense cubic in d+1 <= 17 variables

// Polynomial coefficients in shared memory, in one of two forms per polynomial:
//  * sparse: the monomial list (coefficient, packed factor list);
//  * dense: all monomials of degree exactly D (2 or 3) in the d+1 variables
//    x_0..x_(d-1), x_d = 1 (so lower degrees are included), stored in the loop order of a
//    multivariate Horner scheme, duplicates of the input list merged in input order.
// Dense costs C(d+D, D) + ... fused multiply-adds independent of the number of input
// monomials; it is chosen when that is cheaper than the sparse loop.
struct PolyShared {
    int nu, nf, d;
    int dense_u, dense_f;   // 0: sparse; 2 or 3: dense degree
    double pa, pb, lam;
    union {                          // U owns [0, 1024), F owns [1024, 2048), either form:
        double v[4 * kMaxTerms];     // sparse U: coef [0, 512), mono [512, 1024)
        uint64_t u[4 * kMaxTerms];   // sparse F: coef [1024, 1536), mono [1536, 2048)
    } buf;                           // dense U: [0, 1024), dense F: [1024, 2048)
    uint16_t ukey[kMaxTerms], fkey[kMaxTerms];     // dense keys as a cubic
    uint16_t ukey2[kMaxTerms], fkey2[kMaxTerms];   // dense keys as a quadratic (0xFFFF: degree 3)
    int maxdeg_u, maxdeg_f;
};

__device__ __forceinline__ double ps_ucoef(const PolyShared &ps, int q) { return ps.buf.v[q]; }
__device__ __forceinline__ double ps_fcoef(const PolyShared &ps, int q) { return ps.buf.v[2 * kMaxTerms + q]; }
__device__ __forceinline__ uint64_t ps_umono(const PolyShared &ps, int q) { return ps.buf.u[kMaxTerms + q]; }
__device__ __forceinline__ uint64_t ps_fmono(const PolyShared &ps, int q) { return ps.buf.u[3 * kMaxTerms + q]; }

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

// Number of monomials of degree exactly D in v variables: C(v + D - 1, D).
__host__ __device__ constexpr int dense_size(int v, int D) {
    return D == 2 ? v * (v + 1) / 2 : v * (v + 1) * (v + 2) / 6;
}

// Position of the monomial with sorted factors f[0] <= ... <= f[D-1] (variables 0..V-1,
// V = d+1, padding with V-1) in the Horner loop order: a over 0..V-1, b over a..V-1,
// c over b..V-1.
__device__ __forceinline__ int dense_index(const int *f, int D, int V) {
    int idx = 0;
    if (D == 3) {
        for (int a = 0; a < f[0]; ++a) idx += (V - a) * (V - a + 1) / 2;
        for (int b = f[0]; b < f[1]; ++b) idx += V - b;
        return idx + (f[2] - f[1]);
    }
    for (int a = 0; a < f[0]; ++a) idx += V - a;
    return idx + (f[1] - f[0]);
}

// Dense key of monomial e (degree <= D) or -1 when its degree exceeds D; sets *deg.
__device__ __forceinline__ int monomial_key(const int32_t *e, int d, int D, int *deg) {
    int f[3] = {d, d, d};
    int n = 0;
    for (int k = 0; k < d; ++k)
        for (int q = 0; q < e[k]; ++q) {
            if (n < 3) f[n] = k;
            ++n;
        }
    *deg = n;
    if (n > D) return -1;
    return dense_index(f, D, d + 1);
}

// allow_dense: the real sector family evaluates through the dense form when cheaper; the
// complex deformed family keeps the sparse list (its derivatives use the factor lists).
template <class P>
__device__ __forceinline__ void stage_poly(const P &p, PolyShared &ps, bool allow_dense) {
    const int tid = threadIdx.x;
    const int d = p.d;
    if (tid == 0) {
        ps.nu = p.nu;
        ps.nf = p.nf;
        ps.d = d;
        ps.pa = p.pa;
        ps.pb = p.pb;
        ps.lam = p.lam;
        ps.maxdeg_u = 0;
        ps.maxdeg_f = 0;
    }
    __syncthreads();
    // keys as a cubic in d+1 variables (degree of each monomial recorded)
    for (int q = tid; q < p.nu; q += blockDim.x) {
        int deg;
        int key = monomial_key(p.uexp + (size_t)q * d, d, 3, &deg);
        ps.ukey[q] = (uint16_t)(key < 0 ? 0xFFFF : key);
        key = monomial_key(p.uexp + (size_t)q * d, d, 2, &deg);
        ps.ukey2[q] = (uint16_t)(key < 0 ? 0xFFFF : key);
        atomicMax(&ps.maxdeg_u, deg);
    }
    for (int q = tid; q < p.nf; q += blockDim.x) {
        int deg;
        int key = monomial_key(p.fexp + (size_t)q * d, d, 3, &deg);
        ps.fkey[q] = (uint16_t)(key < 0 ? 0xFFFF : key);
        key = monomial_key(p.fexp + (size_t)q * d, d, 2, &deg);
        ps.fkey2[q] = (uint16_t)(key < 0 ? 0xFFFF : key);
        atomicMax(&ps.maxdeg_f, deg);
    }
    __syncthreads();
    // choose the form per polynomial from the FP64 operation counts
    const int V = d + 1;
    const int cost3 = dense_size(V, 3) + dense_size(V, 2) + V;
    const int cost2 = dense_size(V, 2) + V;
    const int du = !allow_dense || ps.maxdeg_u > 3 ? 0 : (ps.maxdeg_u <= 2 ? 2 : 3);
    const int df = !allow_dense || ps.maxdeg_f > 3 ? 0 : (ps.maxdeg_f <= 2 ? 2 : 3);
    const int sparse_u = p.nu * (ps.maxdeg_u + 1), sparse_f = p.nf * (ps.maxdeg_f + 1);
    const int use_u = (du && (du == 2 ? cost2 : cost3) < sparse_u) ? du : 0;
    const int use_f = (df && (df == 2 ? cost2 : cost3) < sparse_f) ? df : 0;
    __syncthreads();   // every thread has read maxdeg before the buffers are rewritten
    if (tid == 0) {
        ps.dense_u = use_u;
        ps.dense_f = use_f;
    }
    if (use_u) {
        // re-key as a quadratic when the dense form is quadratic
        const int n2 = dense_size(V, use_u);
        for (int e = tid; e < n2; e += blockDim.x) {
            double acc = 0.0;
            const uint16_t *keys = use_u == 2 ? ps.ukey2 : ps.ukey;
            for (int q = 0; q < p.nu; ++q)
                if (keys[q] == e) acc += p.ucoef[q];
            ps.buf.v[e] = acc;
        }
    } else {
        for (int q = tid; q < p.nu; q += blockDim.x) {
            ps.buf.v[q] = p.ucoef[q];
            ps.buf.u[kMaxTerms + q] = pack_monomial(p.uexp + (size_t)q * d, d);
        }
    }
    if (use_f) {
        const int n3 = dense_size(V, use_f);
        for (int e = tid; e < n3; e += blockDim.x) {
            double acc = 0.0;
            const uint16_t *keys = use_f == 2 ? ps.fkey2 : ps.fkey;
            for (int q = 0; q < p.nf; ++q)
                if (keys[q] == e) acc += p.fcoef[q];
            ps.buf.v[2 * kMaxTerms + e] = acc;
        }
    } else {
        for (int q = tid; q < p.nf; q += blockDim.x) {
            ps.buf.v[2 * kMaxTerms + q] = p.fcoef[q];
            ps.buf.u[3 * kMaxTerms + q] = pack_monomial(p.fexp + (size_t)q * d, d);
        }
    }
}

// Dense Horner evaluation at x[0..d] with x[d] = 1 (x in local memory).
__device__ __forceinline__ double dense_eval(const double *x, int V, int D, const double *C) {
    double F = 0.0;
    int idx = 0;
    if (D == 3) {
#pragma unroll 1
        for (int a = 0; a < V; ++a) {
            double sa = 0.0;
#pragma unroll 1
            for (int b = a; b < V; ++b) {
                double t = 0.0;
#pragma unroll 1
                for (int c = b; c < V; ++c) t = fma(C[idx++], x[c], t);
                sa = fma(x[b], t, sa);
            }
            F = fma(x[a], sa, F);
        }
    } else {
#pragma unroll 1
        for (int a = 0; a < V; ++a) {
            double t = 0.0;
#pragma unroll 1
            for (int b = a; b < V; ++b) t = fma(C[idx++], x[b], t);
            F = fma(x[a], t, F);
        }
    }
    return F;
}

// Real polynomial value at x (x indexed at run time: x lives in local memory).
__device__ __forceinline__ double poly_real(const double *x, int nterm, const double *coef,
                                            const uint64_t *mono) {
    double s = 0.0;
#pragma unroll 1
    for (int q = 0; q < nterm; ++q) {
        uint64_t code = mono[q];
        int deg = (int)(code & 15u);
        double t = coef[q];
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t *= x[(code >> (4 * f)) & 15u];
        s += t;
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
    double x[kMaxDim + 1];
#pragma unroll 1
    for (int k = 0; k < d; ++k) x[k] = xin[k];
    x[d] = 1.0;
    const double U = ps.dense_u ? dense_eval(x, d + 1, ps.dense_u, ps.buf.v)
                                : poly_real(x, ps.nu, ps.buf.v, ps.buf.u + kMaxTerms);
    const double F = ps.dense_f ? dense_eval(x, d + 1, ps.dense_f, ps.buf.v + 2 * kMaxTerms)
                                : poly_real(x, ps.nf, ps.buf.v + 2 * kMaxTerms, ps.buf.u + 3 * kMaxTerms);
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
        uint64_t code = ps_fmono(ps, q);
        int deg = (int)(code & 15u);
        double c = ps_fcoef(ps, q);
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
        uint64_t code = ps_umono(ps, q);
        int deg = (int)(code & 15u);
        cplx t = {1.0, 0.0};
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t = cmul(t, z[(code >> (4 * f)) & 15u]);
        U.re = fma(ps_ucoef(ps, q), t.re, U.re);
        U.im = fma(ps_ucoef(ps, q), t.im, U.im);
    }
#pragma unroll 1
    for (int q = 0; q < ps.nf; ++q) {
        uint64_t code = ps_fmono(ps, q);
        int deg = (int)(code & 15u);
        cplx t = {1.0, 0.0};
#pragma unroll 1
        for (int f = 1; f <= deg; ++f) t = cmul(t, z[(code >> (4 * f)) & 15u]);
        F.re = fma(ps_fcoef(ps, q), t.re, F.re);
        F.im = fma(ps_fcoef(ps, q), t.im, F.im);
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
