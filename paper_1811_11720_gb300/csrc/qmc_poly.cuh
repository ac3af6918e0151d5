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
#include <type_traits>

#include "qmc_fixed.cuh"
#include "qmc_fp.cuh"
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
    int feyn_dense;   // complex family: symmetric-tensor form (see stage_feynman_tensors)
    // complex family, d <= kFeynFixedMaxDim: the tensors also in signed fixed point, F's
    // as round(c 2^sf) at u[3 kMaxTerms + e], U's as round(c 2^su) at u[kMaxTerms + e];
    // the nested-form coefficients of F and U after their FP64 tensors (feyn_add_horner)
    int feyn_fixed, sf, su;
    // real family, dense F with non-negative coefficients and a positive constant term
    // whose error bound passes (stage_poly): the dense coefficients in place as
    // round(c 2^sfix) (unsigned), evaluated by dense_eval_fixed
    int fixed_f, sfix;
    // a = 1 and b = n + 1/2 (0 <= n <= 15): n, so that U^a F^-b = U / (F^n sqrt F) needs no
    // per-evaluation tests of the exponents; -1 otherwise
    int pow_half;
};

// Symmetric-tensor form of the complex family (deg U <= 2, deg F <= 3, d <= kFeynDenseMaxDim):
//   U = u0 + sum_i u1_i x_i + sum_ij U2_ij x_i x_j,
//   F = f0 + sum_i f1_i x_i + sum_ij F2_ij x_i x_j + sum_ijk F3_ijk x_i x_j x_k
// with U2, F2, F3 fully symmetric (a monomial's coefficient shared equally by the
// permutations of its factors).  Layout in buf: U at [0]: u0, u1[d], U2[d][d];
// F at [2 kMaxTerms]: f0, f1[d], F2[d][d], 6 F3[pair(i <= j)][k] (row-major upper triangle).
constexpr int kFeynDenseMaxDim = 11;   // 1 + d + d^2 + d^2 (d+1)/2 <= 2 kMaxTerms
// The fixed-point copies sit in the halves of the U and F blocks the tensors leave free
// (1 + d + d^2 + d^2 (d+1)/2 <= kMaxTerms for d <= 6), the nested-form coefficients of
// the values after the FP64 tensors (1 + d + d^2 + d^2 (d+1)/2 + C(d+3, 3) <= kMaxTerms).
constexpr int kFeynFixedMaxDim = 6;
__device__ __forceinline__ int feyn_pair(int i, int j, int d) {   // i <= j
    return i * d - i * (i - 1) / 2 + (j - i);
}

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

// Adds coefficient c of monomial e (degree <= 3) to the symmetric tensors at base
// (constant, linear, square matrix, then for deg 3 the F3[pair][k] block when t3 != null).
// The cubic block is stored times 6 (6 F3), the factor of the Hessian 2 F2 + 6 F3 x, so
// that the Hessian costs one fused multiply-add per entry; F3[y, y, y] divides it out.
__device__ __forceinline__ void feyn_add_term(double *base, double *t3, const int32_t *e, int d,
                                              double c) {
    int f[3];
    int n = 0;
    for (int k = 0; k < d; ++k)
        for (int q = 0; q < e[k] && n < 3; ++q) f[n++] = k;
    double *lin = base + 1, *sq = base + 1 + d;
    if (n == 0) {
        base[0] += c;
    } else if (n == 1) {
        lin[f[0]] += c;
    } else if (n == 2) {
        if (f[0] == f[1]) {
            sq[f[0] * d + f[0]] += c;
        } else {
            sq[f[0] * d + f[1]] += 0.5 * c;
            sq[f[1] * d + f[0]] += 0.5 * c;
        }
    } else {
        const int a = f[0], b = f[1], e3 = f[2];   // a <= b <= e3
        if (a == b && b == e3) {
            t3[feyn_pair(a, a, d) * d + a] += 6.0 * c;
        } else if (a == b) {          // a a e3: (aa, e3), (a e3, a)
            t3[feyn_pair(a, a, d) * d + e3] += 2.0 * c;
            t3[feyn_pair(a, e3, d) * d + a] += 2.0 * c;
        } else if (b == e3) {         // a b b: (ab, b), (bb, a)
            t3[feyn_pair(a, b, d) * d + b] += 2.0 * c;
            t3[feyn_pair(b, b, d) * d + a] += 2.0 * c;
        } else {                      // distinct: (ab, e3), (a e3, b), (b e3, a)
            t3[feyn_pair(a, b, d) * d + e3] += c;
            t3[feyn_pair(a, e3, d) * d + b] += c;
            t3[feyn_pair(b, e3, d) * d + a] += c;
        }
    }
}

// Adds coefficient c of monomial e (degree <= 3) to the coefficient list of the nested
// (Horner) form P = c0 + sum_i x_i (c1_i + sum_{j >= i} x_j (c2_ij + sum_{k >= j} c3_ijk x_k)),
// laid out as c0, c1[d], c2 over i <= j, c3 over i <= j <= k (lexicographic).
__device__ __forceinline__ void feyn_add_horner(double *h, const int32_t *e, int d, double c) {
    int f[3];
    int n = 0;
    for (int k = 0; k < d; ++k)
        for (int q = 0; q < e[k] && n < 3; ++q) f[n++] = k;
    int slot = 0;
    if (n >= 1) slot = 1 + f[0];
    if (n >= 2) slot = 1 + d + feyn_pair(f[0], f[1], d);
    if (n == 3) {
        int off = 0;   // triples with first index below f[0], then pairs (j, k) from f[0]
        for (int i = 0; i < f[0]; ++i) off += (d - i) * (d - i + 1) / 2;
        for (int j = f[0]; j < f[1]; ++j) off += d - j;
        slot = 1 + d + d * (d + 1) / 2 + off + (f[2] - f[1]);
    }
    h[slot] += c;
}

// FP64 operations per evaluation of the two forms of the complex family (derivatives,
// values at the complex point; the Jacobian and powers are common).
__device__ __forceinline__ bool feyn_tensor_cheaper(const PolyShared &ps, const int32_t *uexp,
                                                    const int32_t *fexp, int d) {
    if (d > kFeynDenseMaxDim || ps.maxdeg_u > 2 || ps.maxdeg_f > 3) return false;
    int sparse = 0;
    for (int q = 0; q < ps.nf; ++q) {
        int deg = 0;
        for (int k = 0; k < d; ++k) deg += fexp[(size_t)q * d + k];
        sparse += 2 * deg * deg + 8 * deg + 2;
    }
    for (int q = 0; q < ps.nu; ++q) {
        int deg = 0;
        for (int k = 0; k < d; ++k) deg += uexp[(size_t)q * d + k];
        sparse += 8 * deg + 2;
    }
    const int dense = d * d * (d + 1) + 7 * d * d + 10 * d;
    return dense < sparse;
}

// allow_dense: the real sector family evaluates through the dense Horner form when
// cheaper; the complex deformed family uses the symmetric-tensor form when cheaper.
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
        ps.feyn_fixed = 0;
        ps.fixed_f = 0;
        const double tb = 2.0 * p.pb;
        ps.pow_half = (p.pa == 1.0 && tb >= 1.0 && tb <= 31.0 && tb == floor(tb) &&
                       ((int)tb & 1)) ? (int)tb / 2 : -1;
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
    const bool tensors = !allow_dense && feyn_tensor_cheaper(ps, p.uexp, p.fexp, d);
    __syncthreads();   // every thread has read maxdeg before the buffers are rewritten
    if (tid == 0) {
        ps.dense_u = use_u;
        ps.dense_f = use_f;
        ps.feyn_dense = tensors;
    }
    if (tensors) {
        // one thread, input order: duplicates and symmetric slots summed deterministically
        const int nU = 1 + d + d * d;
        const int nF = nU + d * d * (d + 1) / 2;
        for (int e = tid; e < nU; e += blockDim.x) ps.buf.v[e] = 0.0;
        for (int e = tid; e < nF; e += blockDim.x) ps.buf.v[2 * kMaxTerms + e] = 0.0;
        __syncthreads();
        if (tid == 0) {
            for (int q = 0; q < p.nu; ++q)
                feyn_add_term(ps.buf.v, nullptr, p.uexp + (size_t)q * d, d, p.ucoef[q]);
            double *fb = ps.buf.v + 2 * kMaxTerms;
            for (int q = 0; q < p.nf; ++q)
                feyn_add_term(fb, fb + nU, p.fexp + (size_t)q * d, d, p.fcoef[q]);
            // Scales of the fixed-point form: with B the sum of |entries| of a polynomial's
            // tensors, every quantity feyn_fixed_parts forms at x in [0, 1]^d (Hessian
            // entries, contractions, gradients and their partial sums) is below 3 B, so
            // with 16 B 2^s < 2^62 nothing can overflow.
            double bf = 0.0, bu = 0.0;
            for (int e = 0; e < nF; ++e) bf += fabs(fb[e]);
            for (int e = 0; e < nU; ++e) bu += fabs(ps.buf.v[e]);
            int ok = d <= kFeynFixedMaxDim && bf > 0.0 && bf < 1e300 && bu > 0.0 && bu < 1e300;
            const int sf = ok ? 61 - ilogb(16.0 * bf) : 0;
            const int su = ok ? 61 - ilogb(16.0 * bu) : 0;
            ok = ok && sf >= 32 && su >= 32 && sf <= 120 && su <= 120;
            ps.feyn_fixed = ok;
            ps.sf = sf;
            ps.su = su;
        }
        __syncthreads();
        if (ps.feyn_fixed) {
            for (int e = tid; e < nF; e += blockDim.x)
                ps.buf.u[3 * kMaxTerms + e] = (uint64_t)llrint(ldexp(ps.buf.v[2 * kMaxTerms + e], ps.sf));
            for (int e = tid; e < nU; e += blockDim.x)
                ps.buf.u[kMaxTerms + e] = (uint64_t)llrint(ldexp(ps.buf.v[e], ps.su));
            // the values F(x), U(x) in FP64 through the nested form (see feyn_fixed_parts)
            double *hu = ps.buf.v + nU, *hf = ps.buf.v + 2 * kMaxTerms + nF;
            const int nHu = 1 + d + d * (d + 1) / 2, nHf = nHu + d * (d + 1) * (d + 2) / 6;
            for (int e = tid; e < nHu; e += blockDim.x) hu[e] = 0.0;
            for (int e = tid; e < nHf; e += blockDim.x) hf[e] = 0.0;
            __syncthreads();
            if (tid == 0) {
                for (int q = 0; q < p.nu; ++q) feyn_add_horner(hu, p.uexp + (size_t)q * d, d, p.ucoef[q]);
                for (int q = 0; q < p.nf; ++q) feyn_add_horner(hf, p.fexp + (size_t)q * d, d, p.fcoef[q]);
            }
        }
        return;
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
        // Fixed point for F when its relative error provably stays below 2^-42: with
        // non-negative coefficients of sum B and constant term c0 > 0, F >= c0 on the
        // cube; s = 62 - ilogb(B) keeps every partial sum below 2^63 with 2^-s <= 2^-62 B,
        // and N products at under 4.5 units of 2^-s each (dense_eval_fixed) give a
        // relative error below 4.5 N (B / c0) 2^-62, required <= 2^-42.
        __syncthreads();
        if (tid == 0) {
            const double *c = ps.buf.v + 2 * kMaxTerms;
            double B = 0.0;
            int ok = 1;
            for (int e = 0; e < n3; ++e) {
                ok = ok && c[e] >= 0.0;
                B += c[e];
            }
            const double c0 = c[n3 - 1];   // x_d^D: the constant term
            const int N = n3 + (use_f == 3 ? dense_size(V, 2) : 0) + V;
            ok = ok && c0 > 0.0 && B < 1e300 && 4.5 * N * B <= 0x1p20 * c0;
            ps.fixed_f = ok;
            ps.sfix = ok ? 62 - ilogb(B) : 0;
        }
        __syncthreads();
        if (ps.fixed_f)
            for (int e = tid; e < n3; e += blockDim.x)
                ps.buf.u[2 * kMaxTerms + e] =
                    (uint64_t)llrint(ldexp(ps.buf.v[2 * kMaxTerms + e], ps.sfix));
    } else {
        for (int q = tid; q < p.nf; q += blockDim.x) {
            ps.buf.v[2 * kMaxTerms + q] = p.fcoef[q];
            ps.buf.u[3 * kMaxTerms + q] = pack_monomial(p.fexp + (size_t)q * d, d);
        }
    }
}

// Fixed point for polynomial work on the integer multiply pipe: a value v is held as the
// integer round(v 2^s) with one scale s per polynomial (signed for the complex family's
// tensors, unsigned for the real family's non-negative dense forms), a coordinate x in
// [0, 1] as the uint64 X = x 2^64.
//   c X / 2^64 for signed c: the unsigned high word of (c mod 2^64) X, minus X when c < 0.
__device__ __forceinline__ int64_t smulhi_x(int64_t c, uint64_t X) {
    const uint64_t h = mulhi_trunc((uint64_t)c, X);
    return (int64_t)(c < 0 ? h - X : h);
}
// x in [0, 1] to x 2^64, truncated (x = 1 saturates to 2^64 - 1).  For 0 < x < 1 with
// biased exponent E <= 1022, x 2^64 is the 64-bit mantissa shifted right by 1022 - E.
// The range tests compare the bit pattern as a signed integer (non-negative doubles order
// like their bits; negative ones have the sign bit set), which keeps them off the FP64 pipe.
__device__ __forceinline__ uint64_t unit_to_fixed64(double x) {
    const long long b = __double_as_longlong(x);
    if (b >= 0x3FF0000000000000ll) return ~0ull;   // x >= 1
    if (b <= 0) return 0ull;                       // x <= 0
    const int r = 1022 - (int)(b >> 52);
    const uint64_t m = ((uint64_t)b << 11) | 0x8000000000000000ull;
    return r >= 64 ? 0ull : (m >> r);
}
// v 2^-s to double, truncated toward zero, by integer operations.
__device__ __forceinline__ double fixed_s64_to_double(int64_t v, int s) {
    const uint64_t sign = (uint64_t)v & 0x8000000000000000ull;
    const uint64_t a = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    if (!a) return 0.0;
    const int lz = __clzll(a);
    const uint64_t m = a << lz;   // a 2^lz in [2^63, 2^64): v = m 2^(63 - lz - s) / 2^63
    const uint64_t be1 = (uint64_t)(1085 - lz - s);   // biased exponent minus one
    return __longlong_as_double((long long)(sign | ((be1 << 52) + (m >> 11))));
}

// Unsigned u 2^-s to double, truncated, by integer operations (u = 0 gives 0).
__device__ __forceinline__ double fixed_u64_to_double(uint64_t u, int s) {
    if (!u) return 0.0;
    const int lz = __clzll(u);
    const uint64_t m = u << lz;
    const uint64_t be1 = (uint64_t)(1085 - lz - s);
    return __longlong_as_double((long long)((be1 << 52) + (m >> 11)));
}

// The dense Horner form below in unsigned fixed point, for non-negative coefficients
// C = round(c 2^s) and X[k] = x_k 2^64, k < V - 1.  The padding variable x_(V-1) = 1 is
// not multiplied: the loop iterations that meet it are peeled into plain additions.
// Every partial sum is at most the sum of the coefficients, below 2^63.  Each truncated
// product is off by under 3 units of 2^-s (mulhi_trunc's bound and the dropped
// fraction), each coefficient by half a unit.  VT > 0: V compiled in (unrolled loops,
// X in registers); VT = 0: V at run time.  Same operations in the same order.
template <int VT>
__device__ __forceinline__ uint64_t dense_eval_fixed(const uint64_t *X, int V_rt, int D,
                                                     const uint64_t *C) {
    const int V = VT > 0 ? VT : V_rt;
    uint64_t F = 0;
    int idx = 0;
    if (D == 3) {
#pragma unroll
        for (int a = 0; a < V - 1; ++a) {
            uint64_t sa = 0;
#pragma unroll
            for (int b = a; b < V - 1; ++b) {
                uint64_t t = 0;
#pragma unroll
                for (int c = b; c < V - 1; ++c) t += mulhi_trunc(C[idx++], X[c]);
                t += C[idx++];                 // c = V - 1
                sa += mulhi_trunc(X[b], t);
            }
            sa += C[idx++];                    // b = c = V - 1
            F += mulhi_trunc(X[a], sa);
        }
    } else {
#pragma unroll
        for (int a = 0; a < V - 1; ++a) {
            uint64_t t = 0;
#pragma unroll
            for (int b = a; b < V - 1; ++b) t += mulhi_trunc(C[idx++], X[b]);
            t += C[idx++];                     // b = V - 1
            F += mulhi_trunc(X[a], t);
        }
    }
    return F + C[idx];                         // the constant term
}

// The FP64 dense Horner form with V compiled in, the x_(V-1) = 1 iterations peeled:
// fma(c, 1, t) and fma(1, t, s) round like the additions that replace them, so the
// result equals dense_eval's bit for bit.
template <int V, int D>
__device__ __forceinline__ double dense_eval_t(const double *x, const double *C) {
    double F = 0.0;
    int idx = 0;
    if constexpr (D == 3) {
#pragma unroll
        for (int a = 0; a < V; ++a) {
            double sa = 0.0;
#pragma unroll
            for (int b = a; b < V; ++b) {
                double t = 0.0;
#pragma unroll
                for (int c = b; c < V - 1; ++c) t = fma(C[idx++], x[c], t);
                t = t + C[idx++];
                sa = b < V - 1 ? fma(x[b], t, sa) : sa + t;
            }
            F = a < V - 1 ? fma(x[a], sa, F) : F + sa;
        }
    } else {
#pragma unroll
        for (int a = 0; a < V; ++a) {
            double t = 0.0;
#pragma unroll
            for (int b = a; b < V - 1; ++b) t = fma(C[idx++], x[b], t);
            t = t + C[idx++];
            F = a < V - 1 ? fma(x[a], t, F) : F + t;
        }
    }
    return F;
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

// x^y for x > 0: integer and half-integer |y| <= 16 by repeated squaring and one square
// root (x^(n + 1/2) = x^n sqrt(x), negative y through one reciprocal), otherwise the
// library pow.
__device__ __forceinline__ double pow_pos(double x, double y) {
    if (y == 1.0) return x;
    if (y == -1.0) return 1.0 / x;
    const double ay = fabs(y), twoy = 2.0 * ay;
    if (ay <= 16.0 && twoy == floor(twoy) && x > 0.0) {
        const int n = (int)ay;   // integer part
        double v = ipow_u(x, n);
        if (twoy != 2.0 * n) v = n ? v * sqrt(x) : sqrt(x);
        return y < 0.0 ? 1.0 / v : v;
    }
    return pow(x, y);
}

// U^a F^-b of the real family: U (F^-1/2)^(2n+1) when a = 1, b = n + 1/2 and F > 0 (one
// reciprocal square root and its powers instead of a square root and a division; the
// exponent tests made once at staging), else pow_pos.
__device__ __forceinline__ double sector_power(double U, double F, const PolyShared &ps) {
    if (ps.pow_half >= 0 && F > 0.0) return U * ipow_u(rsqrt(F), 2 * ps.pow_half + 1);
    return pow_pos(U, ps.pa) * pow_pos(F, -ps.pb);
}

// The real family with F in fixed point, both forms dense and d compiled in (d = 3..8):
// the coordinates and the unrolled loops stay in registers.  x (doubles, for U) and X
// (x 2^64, for F) hold the same point.
template <int D>
__device__ __forceinline__ double sector_fixed_core(const double *x, const uint64_t *X,
                                                    const PolyShared &ps) {
    constexpr int V = D + 1;
    const double U = ps.dense_u == 3 ? dense_eval_t<V, 3>(x, ps.buf.v) : dense_eval_t<V, 2>(x, ps.buf.v);
    const uint64_t *C = ps.buf.u + 2 * kMaxTerms;
    const uint64_t Fq = ps.dense_f == 3 ? dense_eval_fixed<V>(X, V, 3, C) : dense_eval_fixed<V>(X, V, 2, C);
    return sector_power(U, fixed_u64_to_double(Fq, ps.sfix), ps);   // F >= c0 > 0
}
template <int D>
static __device__ __noinline__ double sector_value_fixed(const double *xin, const PolyShared &ps) {
    double x[D];
    uint64_t X[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        x[k] = xin[k];
        X[k] = unit_to_fixed64(x[k]);
    }
    return sector_fixed_core<D>(x, X, ps);
}
// The same from the coordinates in 0.64 fixed point (the integer-pipe transforms), x
// from X by integer operations (truncated).
template <int D>
static __device__ __noinline__ double sector_value_fixed_x(const uint64_t *Xin, const PolyShared &ps) {
    double x[D];
    uint64_t X[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        X[k] = Xin[k];
        x[k] = fixed_u64_to_double(X[k], 64);
    }
    return sector_fixed_core<D>(x, X, ps);
}

// Whether sector_value_fixed(_x) serves this integrand (uniform over the block).
__device__ __forceinline__ bool sector_fixed_ok(const PolyShared &ps, int d) {
    return ps.fixed_f && ps.dense_u && d >= 3 && d <= 8;
}

__device__ __forceinline__ double sector_value_x(const uint64_t *X, int d, const PolyShared &ps) {
    switch (d) {
    case 3: return sector_value_fixed_x<3>(X, ps);
    case 4: return sector_value_fixed_x<4>(X, ps);
    case 5: return sector_value_fixed_x<5>(X, ps);
    case 6: return sector_value_fixed_x<6>(X, ps);
    case 7: return sector_value_fixed_x<7>(X, ps);
    default: return sector_value_fixed_x<8>(X, ps);
    }
}

__device__ __forceinline__ double sector_value(const double *xin, int d, const PolyShared &ps) {
    if (sector_fixed_ok(ps, d)) {
        switch (d) {
        case 3: return sector_value_fixed<3>(xin, ps);
        case 4: return sector_value_fixed<4>(xin, ps);
        case 5: return sector_value_fixed<5>(xin, ps);
        case 6: return sector_value_fixed<6>(xin, ps);
        case 7: return sector_value_fixed<7>(xin, ps);
        case 8: return sector_value_fixed<8>(xin, ps);
        default: break;
        }
    }
    double x[kMaxDim + 1];
#pragma unroll 1
    for (int k = 0; k < d; ++k) x[k] = xin[k];
    x[d] = 1.0;
    const double U = ps.dense_u ? dense_eval(x, d + 1, ps.dense_u, ps.buf.v)
                                : poly_real(x, ps.nu, ps.buf.v, ps.buf.u + kMaxTerms);
    double F;
    if (ps.fixed_f) {
        uint64_t X[kMaxDim];
#pragma unroll 1
        for (int k = 0; k < d; ++k) X[k] = unit_to_fixed64(x[k]);
        F = fixed_u64_to_double(dense_eval_fixed<0>(X, d + 1, ps.dense_f, ps.buf.u + 2 * kMaxTerms),
                                ps.sfix);
    } else {
        F = ps.dense_f ? dense_eval(x, d + 1, ps.dense_f, ps.buf.v + 2 * kMaxTerms)
                       : poly_real(x, ps.nf, ps.buf.v + 2 * kMaxTerms, ps.buf.u + 3 * kMaxTerms);
    }
    return sector_power(U, F, ps);
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


// log a = (log |a|, arg a), principal branch.
__device__ __forceinline__ cplx clog_principal(cplx a) {
    const double n2 = fma(a.re, a.re, a.im * a.im);
    // |a|^2 stays normal for the magnitudes met here; otherwise take log(hypot)
    const double lr = (n2 > 1e-300 && n2 < 1e300) ? 0.5 * log(n2) : log(hypot(a.re, a.im));
    return {lr, atan2(a.im, a.re)};
}

// det J = det(I - i lam (D H + E)), D = diag(x (1 - x)), E = diag((1 - 2x) g), by
// elimination without pivoting (see the header comment).  lx[k] = -lam x_k (1 - x_k): the
// imaginary part of J is lx_k H_kl, plus -lam (1 - 2 x_k) g_k on the diagonal.  DT > 0 is
// the dimension as a compile-time constant (the loops unroll and the d x d work array can
// live in registers); DT = 0 takes d at run time (the array in local memory).  Both run
// the same operations in the same order.
template <int DT>
__device__ __forceinline__ cplx feynman_jacobian_det(const double *x, const double *lx,
                                                     const double *g, const double *H, int d_rt,
                                                     double lam) {
    constexpr int DA = DT > 0 ? DT : kMaxDim;
    const int d = DT > 0 ? DT : d_rt;
    cplx A[DA * DA];
#pragma unroll
    for (int k = 0; k < d; ++k)
#pragma unroll
        for (int l = 0; l < d; ++l) {
            double im = lx[k] * H[k * d + l];
            if (k == l) im = fma(-lam * fma(-2.0, x[k], 1.0), g[k], im);
            A[k * d + l] = {(k == l) ? 1.0 : 0.0, im};
        }
    // Column 0 by hand: before any elimination the off-diagonal entries are purely
    // imaginary (A = I - i lam M), so the multipliers and the updates need two real
    // products each instead of a full complex product (about a quarter of the
    // determinant's FP64 work for d = 5).
    cplx det = A[0];
    if (d == 1) return det;
    {
        const cplx inv = crecip(A[0]);
#pragma unroll
        for (int r = 1; r < d; ++r) {
            const double a = A[r * d].im;                      // A[r][0] = i a
            const cplx l = {-a * inv.im, a * inv.re};          // i a / A[0][0]
#pragma unroll
            for (int q = 1; q < d; ++q) {
                const double b = A[q].im;                      // A[0][q] = i b
                cplx &t = A[r * d + q];                        // t -= l (i b)
                t.re = fma(l.im, b, t.re);
                t.im = fma(-l.re, b, t.im);
            }
        }
    }
#pragma unroll
    for (int c = 1; c < d; ++c) {
        cplx piv = A[c * d + c];
        det = cmul(det, piv);
        if (c + 1 == d) break;
        cplx inv = crecip(piv);
#pragma unroll
        for (int r = c + 1; r < d; ++r) {
            cplx l = cmul(A[r * d + c], inv);
#pragma unroll
            for (int q = c + 1; q < d; ++q) {
                const cplx a = A[c * d + q];
                cplx &t = A[r * d + q];                        // t -= l a, four fused steps
                t.re = fma(-l.re, a.re, fma(l.im, a.im, t.re));
                t.im = fma(-l.re, a.im, fma(-l.im, a.re, t.im));
            }
        }
    }
    return det;
}

// The same determinant by symmetric elimination.  J = D + P K with D = diag(1 + i Λ),
// Λ_k = -lam (1 - 2 x_k) g_k, P = diag(lx) real and K = i H complex symmetric.
// Eliminating column c (pivot A_cc = D_c + p_c K_cc) leaves the trailing block in the same
// shape, D + P K' with K'_rq = K_rq - (p_c / A_cc) K_rc K_cq, still symmetric, so only the
// upper triangle of K is updated: about two thirds of the general elimination's complex
// updates, and J's entries p_k H_kl are never formed.  The pivots, and so det J, equal
// those of the elimination above up to rounding.  In the first step K is purely
// imaginary and K_rc K_cq = -H_rc H_cq is real.
template <int D>
__device__ __forceinline__ cplx feynman_jacobian_det_sym(const double *x, const double *lx,
                                                         const double *g, const double *H,
                                                         double lam) {
    double Kr[D * D], Ki[D * D];   // upper triangle, K_rq at r * D + q for q >= r
    double lamb[D];
#pragma unroll
    for (int k = 0; k < D; ++k) lamb[k] = -lam * fma(-2.0, x[k], 1.0) * g[k];
    cplx det = {1.0, fma(lx[0], H[0], lamb[0])};   // A_00 = 1 + i (Λ_0 + p_0 H_00)
    if constexpr (D == 1) return det;
    {
        const cplx inv = crecip(det);
        const cplx c0 = {lx[0] * inv.re, lx[0] * inv.im};
#pragma unroll
        for (int r = 1; r < D; ++r) {
            const cplx u = {c0.re * H[r], c0.im * H[r]};   // (p_0 / A_00) H_r0
#pragma unroll
            for (int q = r; q < D; ++q) {                   // K'_rq = i H_rq + u H_0q
                Kr[r * D + q] = u.re * H[q];
                Ki[r * D + q] = fma(u.im, H[q], H[r * D + q]);
            }
        }
    }
#pragma unroll
    for (int c = 1; c < D; ++c) {
        const cplx piv = {fma(lx[c], Kr[c * D + c], 1.0), fma(lx[c], Ki[c * D + c], lamb[c])};
        det = cmul(det, piv);
        if (c + 1 == D) break;
        const cplx inv = crecip(piv);
        const cplx cc = {lx[c] * inv.re, lx[c] * inv.im};
#pragma unroll
        for (int r = c + 1; r < D; ++r) {
            const cplx w = cmul(cc, {Kr[c * D + r], Ki[c * D + r]});   // (p_c / A_cc) K_rc
#pragma unroll
            for (int q = r; q < D; ++q) {                              // K_rq -= w K_cq
                const double ar = Kr[c * D + q], ai = Ki[c * D + q];
                Kr[r * D + q] = fma(-w.re, ar, fma(w.im, ai, Kr[r * D + q]));
                Ki[r * D + q] = fma(-w.re, ai, fma(-w.im, ar, Ki[r * D + q]));
            }
        }
    }
    return det;
}

// Principal square root: Re >= 0, the sign of Im from Im a (so a = -x - 0i maps to the
// lower side of the cut, as exp(Log(a) / 2) with the arg in (-pi, pi] and signed zeros).
// The branch that avoids cancellation: t = sqrt((|a| + |Re a|) / 2), the other part
// Im a / (2 t).
__device__ __forceinline__ cplx csqrt_principal(cplx a) {
    // |a| without the library's rescaling where the squares can neither overflow nor
    // underflow (both exponents within (2^-500, 2^500): a test on the bit patterns, off the
    // FP64 pipe; relative error within 1.5 ulp)
    const uint64_t br = (uint64_t)__double_as_longlong(a.re), bi = (uint64_t)__double_as_longlong(a.im);
    const uint32_t er = (uint32_t)(br >> 52) & 0x7FFu, ei = (uint32_t)(bi >> 52) & 0x7FFu;
    const double r = (er - 524u < 998u && ei - 524u < 998u)   // 524 <= E <= 1521
                         ? sqrt(fma(a.re, a.re, a.im * a.im))
                         : hypot(a.re, a.im);
    if (((br | bi) << 1) == 0) return {0.0, a.im};            // a = 0
    // t = sqrt(s) and a.im / (2 t) from one reciprocal square root
    const double s = 0.5 * (r + fabs(a.re));
    const double q = rsqrt(s);
    const double t = s * q;
    const double o = a.im * (0.5 * q);
    if (!(br >> 63) || !(br << 1)) return {t, o};             // a.re >= 0 (and -0)
    return {fabs(o), copysign(t, a.im)};
}

// U^a F^-b det for principal branches: exp(a Log U - b Log F) det (a = 1: U exp(-b Log F)).
// For a = 1 and a half-integer b = n + 1/2 (pow_half = n, 0 <= n <= 15, decided once at
// staging), F^-b = 1 / (F^n sqrt(F)) with the principal root, the same branch as
// exp(-b Log F): two square roots and a reciprocal instead of a logarithm, an arctangent,
// an exponential and a sine/cosine pair.
__device__ __forceinline__ void feynman_combine(cplx U, cplx F, cplx det, double pa, double pb,
                                                int pow_half, double &re, double &im) {
    if (pow_half >= 0) {
        cplx den = csqrt_principal(F);
        const int nint = pow_half;
#pragma unroll 1
        for (int q = 0; q < nint; ++q) den = cmul(den, F);
        cplx v = cmul(cmul(U, crecip(den)), det);
        re = v.re;
        im = v.im;
        return;
    }
    const cplx lf = clog_principal(F);
    double er = -pb * lf.re, ei = -pb * lf.im;
    if (pa != 1.0) {
        const cplx lu = clog_principal(U);
        er = fma(pa, lu.re, er);
        ei = fma(pa, lu.im, ei);
    }
    const double mag = exp(er);
    double sn, cs;
    sincos(ei, &sn, &cs);
    cplx v = {mag * cs, mag * sn};
    if (pa == 1.0) v = cmul(U, v);
    v = cmul(v, det);
    re = v.re;
    im = v.im;
}

// Hessian and gradient of F and grad U of the symmetric-tensor form at x, as
// feynman_value_dense forms them in FP64, here in the fixed point above (same formulas:
// H_ij = 2 F2_ij + sum_k (6 F3)_ijk x_k, g_i = f1_i + (F2 x)_i + (H x)_i / 2,
// grad U_i = u1_i + 2 (U2 x)_i).  A product is off by under 4.5 units of 2^-s
// (mulhi_trunc's bound, the dropped fraction, the rounded entry and the truncated X), so
// for d <= 6 each result is within 2^8 units, i.e. 2^-49 of the sum B of the polynomial's
// |entries| (2^-s <= 2^-57 B by the choice of s); every partial sum stays below
// 3 B < 2^62 2^-s.  These enter the integrand only through the deformation
// y = -lam x (1 - x) g and the Jacobian, where an error small against B is small against
// the terms it joins.  The values F(x) and U(x) need relative accuracy instead: near the
// zero set of F, F(x) is many orders below B, and its error there is raised to the power
// -b.  They stay in FP64, by the nested form of the monomial list
// (c0 + sum_i x_i (c1_i + sum_{j >= i} x_j (c2_ij + sum_{k >= j} c3_ijk x_k))).
template <int D>
__device__ __forceinline__ void feyn_fixed_parts(const double *x, const uint64_t *X,
                                                 const PolyShared &ps, double *H, double *g,
                                                 double *gU, double &Fx, double &Ux) {
    constexpr int nU = 1 + D + D * D, nF = nU + D * D * (D + 1) / 2;
    const int64_t *ff = reinterpret_cast<const int64_t *>(ps.buf.u + 3 * kMaxTerms);
    const int64_t *uf = reinterpret_cast<const int64_t *>(ps.buf.u + kMaxTerms);
    const int64_t *f1 = ff + 1, *F2 = ff + 1 + D, *F3 = ff + 1 + D + D * D;
    const int64_t *u1 = uf + 1, *U2 = uf + 1 + D;
    const int sf = ps.sf, su = ps.su;
    int64_t Hq[D * D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
            const int64_t *t = F3 + feyn_pair(i, j, D) * D;
            int64_t s = 2 * F2[i * D + j];
#pragma unroll
            for (int k = 0; k < D; ++k) s += smulhi_x(t[k], X[k]);
            Hq[i * D + j] = s;
            Hq[j * D + i] = s;
        }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        int64_t hx = 0, qx = 0, px = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            hx += smulhi_x(Hq[i * D + j], X[j]);
            qx += smulhi_x(F2[i * D + j], X[j]);
            px += smulhi_x(U2[i * D + j], X[j]);
        }
        g[i] = fixed_s64_to_double(f1[i] + qx + (hx >> 1), sf);
        gU[i] = fixed_s64_to_double(u1[i] + 2 * px, su);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
            const double h = fixed_s64_to_double(Hq[i * D + j], sf);
            H[i * D + j] = h;
            H[j * D + i] = h;
        }
    // values: nested form, coefficients after the FP64 tensors
    const double *hu = ps.buf.v + nU, *hf = ps.buf.v + 2 * kMaxTerms + nF;
    const double *c2u = hu + 1 + D;
    const double *c2f = hf + 1 + D, *c3f = hf + 1 + D + D * (D + 1) / 2;
    double Fv = hf[0], Uv = hu[0];
    int p2 = 0, p3 = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double tf = hf[1 + i], tu = hu[1 + i];
#pragma unroll
        for (int j = i; j < D; ++j) {
            double tij = c2f[p2];
#pragma unroll
            for (int k = j; k < D; ++k) tij = fma(c3f[p3++], x[k], tij);
            tf = fma(tij, x[j], tf);
            tu = fma(c2u[p2], x[j], tu);
            ++p2;
        }
        Fv = fma(tf, x[i], Fv);
        Uv = fma(tu, x[i], Uv);
    }
    Fx = Fv;
    Ux = Uv;
}

// Symmetric-tensor form (deg U <= 2, deg F <= 3).  At the real point x:
//   H_ij = 2 F2_ij + 6 sum_k F3_ijk x_k,  g_i = f1_i + (F2 x)_i + (H x)_i / 2,
//   F(x) = f0 + sum_i x_i (f1_i + (H x)_i / 6 + 2 (F2 x)_i / 3),
// and at z = x + i y (y = -lam x (1 - x) g) the cubic's Taylor series is exact:
//   F(z) = F(x) - y.H y / 2 + i (g.y - sum_ijk F3_ijk y_i y_j y_k),
//   U(z) = U(x) - y.U2 y + i grad U.y,  grad U = u1 + 2 U2 x.
// DT > 0: the dimension as a compile-time constant (unrolled loops, per-thread arrays of
// d entries that can stay in registers); DT = 0: d at run time.  Same operations, same order.
// IN = uint64_t (with FX): the coordinates arrive as x 2^64 from the integer-pipe map and
// the doubles are formed from them by integer operations.
template <int DT, bool FX = false, class IN = double>
static __device__ __noinline__ void feynman_value_dense(const IN *xin, int d_rt,
                                                        const PolyShared &ps, double &re,
                                                        double &im,
                                                        unsigned long long &signfail) {
    constexpr int DA = DT > 0 ? DT : kMaxDim;
    const int d = DT > 0 ? DT : d_rt;
    const double *ub = ps.buf.v;
    const double *u1 = ub + 1, *U2 = ub + 1 + d;
    const double *fb = ps.buf.v + 2 * kMaxTerms;
    const double *f1 = fb + 1, *F2 = fb + 1 + d, *F3 = fb + 1 + d + d * d;   // F3: 6 F3
    double x[DA], g[DA], y[DA], xo[DA];
    double H[DA * DA];
    double Fx = 0.0, Ux = 0.0;
    double gU[DA];
    uint64_t X[DA];   // x 2^64 (fixed-point form only)
    if constexpr (FX) {
        static_assert(DT > 0 && DT <= kFeynFixedMaxDim, "fixed point needs a compiled dimension");
#pragma unroll
        for (int k = 0; k < d; ++k) {
            if constexpr (std::is_same<IN, uint64_t>::value) {
                X[k] = xin[k];
                x[k] = fixed_u64_to_double(X[k], 64);
            } else {
                x[k] = xin[k];
                X[k] = unit_to_fixed64(x[k]);
            }
        }
        feyn_fixed_parts<DT>(x, X, ps, H, g, gU, Fx, Ux);
    } else {
#pragma unroll
        for (int k = 0; k < d; ++k) x[k] = xin[k];
        // Hessian of F (symmetric)
#pragma unroll
        for (int i = 0; i < d; ++i)
#pragma unroll
            for (int j = i; j < d; ++j) {
                const double *t = F3 + feyn_pair(i, j, d) * d;
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < d; ++k) s = fma(t[k], x[k], s);
                const double h = fma(2.0, F2[i * d + j], s);   // s = (6 F3 x)_ij
                H[i * d + j] = h;
                H[j * d + i] = h;
            }
        // gradient, F(x), U(x), grad U
#pragma unroll
        for (int i = 0; i < d; ++i) {
            double hx = 0.0, qx = 0.0, px = 0.0;
#pragma unroll
            for (int j = 0; j < d; ++j) {
                hx = fma(H[i * d + j], x[j], hx);
                qx = fma(F2[i * d + j], x[j], qx);
                px = fma(U2[i * d + j], x[j], px);
            }
            g[i] = fma(0.5, hx, f1[i] + qx);
            Fx = fma(x[i], fma(hx, 1.0 / 6.0, fma(qx, 2.0 / 3.0, f1[i])), Fx);
            gU[i] = fma(2.0, px, u1[i]);
            Ux = fma(x[i], u1[i] + px, Ux);
        }
        Fx += fb[0];
        Ux += ub[0];
    }
    // deformation: xo holds -lam x (1 - x)
    const double lam = ps.lam;
#pragma unroll
    for (int k = 0; k < d; ++k) {
        if constexpr (FX)   // x (1 - x) 2^64 as the truncated high product X (2^64 - 1 - X)
            xo[k] = -lam * fixed_u64_to_double(mulhi_trunc(X[k], ~X[k]), 64);
        else
            xo[k] = -lam * (x[k] * (1.0 - x[k]));
        y[k] = xo[k] * g[k];
    }
    // F(z), U(z)
    cplx Fz, Uz;
    if constexpr (FX) {
        // y.H y over the upper triangle; the quadratic part of U and the cubic part of F
        // at y by their nested forms (the same monomial coefficients as F(x), U(x))
        constexpr int nU = 1 + DA + DA * DA, nF = nU + DA * DA * (DA + 1) / 2;
        const double *c2u = ps.buf.v + nU + 1 + DA;
        const double *c3f = ps.buf.v + 2 * kMaxTerms + nF + 1 + DA + DA * (DA + 1) / 2;
        double yHy = 0.0, gy = 0.0, gUy = 0.0, qU = 0.0, cF = 0.0;
        int p2 = 0, p3 = 0;
#pragma unroll
        for (int i = 0; i < DA; ++i) {
            double t = 0.0;
#pragma unroll
            for (int j = i + 1; j < DA; ++j) t = fma(H[i * DA + j], y[j], t);
            yHy = fma(y[i], fma(2.0, t, H[i * DA + i] * y[i]), yHy);
            gy = fma(g[i], y[i], gy);
            gUy = fma(gU[i], y[i], gUy);
            double tf = 0.0, tu = 0.0;
#pragma unroll
            for (int j = i; j < DA; ++j) {
                double tij = 0.0;
#pragma unroll
                for (int k = j; k < DA; ++k) tij = fma(c3f[p3++], y[k], tij);
                tf = fma(tij, y[j], tf);
                tu = fma(c2u[p2++], y[j], tu);
            }
            cF = fma(tf, y[i], cF);
            qU = fma(tu, y[i], qU);
        }
        Fz = {fma(-0.5, yHy, Fx), gy - cF};
        Uz = {Ux - qU, gUy};
    } else {
        double yHy = 0.0, gy = 0.0, yU2y = 0.0, gUy = 0.0, t3 = 0.0;
#pragma unroll
        for (int i = 0; i < d; ++i) {
            double hy = 0.0, uy = 0.0;
#pragma unroll
            for (int j = 0; j < d; ++j) {
                hy = fma(H[i * d + j], y[j], hy);
                uy = fma(U2[i * d + j], y[j], uy);
            }
            yHy = fma(y[i], hy, yHy);
            yU2y = fma(y[i], uy, yU2y);
            gy = fma(g[i], y[i], gy);
            gUy = fma(gU[i], y[i], gUy);
#pragma unroll
            for (int j = i; j < d; ++j) {
                const double *t = F3 + feyn_pair(i, j, d) * d;
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < d; ++k) s = fma(t[k], y[k], s);
                t3 = fma((i == j ? 1.0 : 2.0) * y[i] * y[j], s, t3);
            }
        }
        Fz = {fma(-0.5, yHy, Fx), fma(t3, -1.0 / 6.0, gy)};   // t3 = 6 F3[y, y, y]
        Uz = {Ux - yU2y, gUy};
    }
    if (Fz.im > 0.0) ++signfail;
    cplx det;
    if constexpr (FX) det = feynman_jacobian_det_sym<DT>(x, xo, g, H, lam);
    else det = feynman_jacobian_det<DT>(x, xo, g, H, d, lam);
    feynman_combine(Uz, Fz, det, ps.pa, ps.pb, ps.pow_half, re, im);
}

// Whether the fixed-point form serves this integrand with coordinates given as x 2^64
// (uniform over the block).
__device__ __forceinline__ bool feyn_fixed_ok(const PolyShared &ps, int d) {
    return ps.feyn_dense && ps.feyn_fixed && d >= 3 && d <= kFeynFixedMaxDim;
}

__device__ __forceinline__ void feynman_value_x(const uint64_t *X, int d, const PolyShared &ps,
                                                double &re, double &im,
                                                unsigned long long &signfail) {
    switch (d) {
    case 3: feynman_value_dense<3, true>(X, d, ps, re, im, signfail); return;
    case 4: feynman_value_dense<4, true>(X, d, ps, re, im, signfail); return;
    case 5: feynman_value_dense<5, true>(X, d, ps, re, im, signfail); return;
    default: feynman_value_dense<6, true>(X, d, ps, re, im, signfail); return;
    }
}

static __device__ __noinline__ void feynman_value(const double *xin, int d, const PolyShared &ps,
                                           double &re, double &im,
                                           unsigned long long &signfail) {
    if (ps.feyn_dense) {
        // the symmetric-tensor form with the dimension compiled in for the common sizes
        if (ps.feyn_fixed) {
            switch (d) {
            case 3: feynman_value_dense<3, true>(xin, d, ps, re, im, signfail); return;
            case 4: feynman_value_dense<4, true>(xin, d, ps, re, im, signfail); return;
            case 5: feynman_value_dense<5, true>(xin, d, ps, re, im, signfail); return;
            case 6: feynman_value_dense<6, true>(xin, d, ps, re, im, signfail); return;
            default: break;
            }
        }
        switch (d) {
        case 3: feynman_value_dense<3>(xin, d, ps, re, im, signfail); return;
        case 4: feynman_value_dense<4>(xin, d, ps, re, im, signfail); return;
        case 5: feynman_value_dense<5>(xin, d, ps, re, im, signfail); return;
        case 6: feynman_value_dense<6>(xin, d, ps, re, im, signfail); return;
        default: feynman_value_dense<0>(xin, d, ps, re, im, signfail); return;
        }
    }
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
    double xo[kMaxDim];   // -lam x (1 - x)
#pragma unroll 1
    for (int k = 0; k < d; ++k) {
        xo[k] = -lam * (x[k] * (1.0 - x[k]));
        z[k] = {x[k], xo[k] * grad[k]};
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
    // J_kl = delta_kl - i lam [delta_kl (1 - 2 x_k) dF_k + x_k (1 - x_k) d2F_kl]
    const cplx det = feynman_jacobian_det<0>(x, xo, grad, H, d, lam);
    feynman_combine(U, F, det, ps.pa, ps.pb, ps.pow_half, re, im);
}

}  // namespace qmc
