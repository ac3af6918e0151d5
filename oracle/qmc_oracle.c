/*
 * qmc_oracle.c -- plain, slow, obviously-correct CPU oracle for the randomly shifted
 * rank-1 lattice rule of Borowka et al., "A GPU compatible quasi-Monte Carlo integrator
 * interfaced to pySecDec" (arXiv:1811.11720).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
 * and reference legs may load this library.  It shares no code, header, table or helper
 * with the CUDA path in paper_1811_11720_gb300/.
 *
 * What it computes (paper Sec. 2.1, Eq. (lattice) and Eq. (lattice-error)):
 *   Q^(k) = (1/n) sum_{i<n} g( {i z/n + Delta_k} ),   Qbar = (1/m) sum_k Q^(k),
 *   sigma^2 = 1/(m(m-1)) sum_k (Q^(k) - Qbar)^2,
 * where g is the integrand after the optional PolySingular variance-reduction map
 * (Sec. 2.4, Eq. (ISfit)) and the periodizing transform (Sec. 2.3: Korobov Eq. (korobov),
 * Sidi Eq. (sidi), baker Eq. (baker), or none).
 *
 * Readings taken where the paper leaves a choice:
 *  - Lattice point.  u = RN( frac(r/n + D 2^-53) ) with r = i z mod n computed exactly and
 *    Delta = D 2^-53 (D a 53-bit integer): the exact rational fractional part rounded
 *    once to the nearest double (ties to even).  u may equal 1.0 when the fraction lies
 *    within half an ulp of 1.
 *  - Shifts.  D_{k,j} = splitmix64 output number (k d + j) >> 11, the published SplitMix64
 *    generator (Steele, Lea, Flood 2014) seeded with `seed`: state += 0x9e3779b97f4a7c15
 *    before each output, then the published mixing function.
 *  - Composition.  g(u) = prod_j w(u_j) * prod_j p_j'(phi(u_j)) * f(p(phi(u))): the
 *    periodizing transform is applied to the fitted integrand (Sec. 3.3.1).
 *  - Baker weight is 1 (the tent map preserves Lebesgue measure).
 *  - Per-shift sums are accumulated in double-double (TwoSum), so the only rounding that
 *    matters is in the integrand itself.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------------------ */
/* Shifts: SplitMix64 (published generator), consumed in row-major [k][j] order.         */
/* ------------------------------------------------------------------------------------ */
static uint64_t splitmix64_mix(uint64_t x) {
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

/* Output number t (t = 0, 1, ...) of the sequential generator seeded with `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t t) {
    uint64_t state = seed;
    /* advance t+1 times; written as a multiply because the state update is a plain add */
    state += (t + 1) * 0x9e3779b97f4a7c15ULL;
    return splitmix64_mix(state);
}

/* D[k*d + j] = 53-bit integer numerator of Delta_{k,j} = D * 2^-53 in [0, 1). */
void oracle_shifts(uint64_t seed, int m, int d, uint64_t *D) {
    for (int k = 0; k < m; k++)
        for (int j = 0; j < d; j++)
            D[(size_t)k * d + j] = oracle_splitmix64(seed, (uint64_t)k * d + j) >> 11;
}

/* ------------------------------------------------------------------------------------ */
/* Lattice points (Eq. (lattice); Fig. 1): exact integer index, one final rounding.      */
/* ------------------------------------------------------------------------------------ */
uint64_t oracle_index(uint64_t i, uint64_t zj, uint64_t n) {
    return (uint64_t)(((u128)i * zj) % n);
}

/* Round the positive rational (N / den) * 2^e2 to the nearest double, ties to even.
 * Works from the binary expansion of N/den produced by long division, one bit at a time:
 * q holds the leading bits, rem the exact remainder. */
static double round_rational(u128 N, uint64_t den, int e2) {
    if (N == 0) return 0.0;
    u128 q = N / den;
    u128 rem = N % den;
    int e = e2;                      /* value = (q + rem/den) * 2^e */
    while (q < ((u128)1 << 54)) {   /* want >= 55 significant bits in q */
        rem <<= 1;
        q <<= 1;
        if (rem >= den) { rem -= den; q |= 1; }
        e -= 1;
    }
    int bits = 0;
    for (u128 t = q; t; t >>= 1) bits++;
    int drop = bits - 53;            /* >= 2 */
    u128 kept = q >> drop;
    int round_bit = (int)((q >> (drop - 1)) & 1);
    int sticky = ((q & (((u128)1 << (drop - 1)) - 1)) != 0) || rem != 0;
    if (round_bit && (sticky || (kept & 1))) kept += 1;
    if (kept == ((u128)1 << 53)) { kept >>= 1; drop += 1; }
    return ldexp((double)(uint64_t)kept, e + drop);
}

/* u = RN( frac(r/n + D 2^-53) ), computed as the exact rational
 * ((r 2^53 + D n) mod (n 2^53)) / (n 2^53). */
double oracle_point(uint64_t r, uint64_t n, uint64_t D) {
    u128 M = (u128)n << 53;
    u128 N = (((u128)r << 53) + (u128)D * n) % M;
    return round_rational(N, n, -53);
}

/* out[((i - i0) * m + k) * d + j] = u for lattice index i, shift k, coordinate j. */
void oracle_points(uint64_t n, const uint64_t *z, int d, const uint64_t *D, int m,
                   uint64_t i0, uint64_t count, double *out) {
    for (uint64_t t = 0; t < count; t++) {
        uint64_t i = i0 + t;
        for (int k = 0; k < m; k++)
            for (int j = 0; j < d; j++) {
                uint64_t r = oracle_index(i, z[j], n);
                out[(t * (uint64_t)m + k) * d + j] = oracle_point(r, n, D[(size_t)k * d + j]);
            }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Periodizing transforms (Sec. 2.3; table of integral transforms, App. A.4).           */
/* ------------------------------------------------------------------------------------ */
enum { OT_NONE = 0, OT_BAKER = 1, OT_KOROBOV = 2, OT_SIDI = 3 };

static double binom(int a, int b) {
    double r = 1.0;
    for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
    return r;
}

static double ipow(double x, int p) {
    double r = 1.0;
    for (int i = 0; i < p; i++) r *= x;
    return r;
}

/* Korobov<r0,r1>, Eq. (korobov): w(u) = (r0+r1+1) C(r0+r1,r0) u^r0 (1-u)^r1 and
 * phi(u) = int_0^u w.  Expanding (1-t)^r1 binomially and integrating term by term:
 * phi(u) = C sum_{k=0}^{r1} C(r1,k) (-1)^k u^(r0+k+1) / (r0+k+1).
 * For u > 1/2 the reflection phi_{r0,r1}(u) = 1 - phi_{r1,r0}(1-u) keeps the sum
 * away from its cancelling regime. */
static double korobov_phi_direct(double u, int r0, int r1) {
    double C = (r0 + r1 + 1) * binom(r0 + r1, r0);
    double s = 0.0;
    for (int k = 0; k <= r1; k++) {
        double term = binom(r1, k) * ipow(u, r0 + k + 1) / (r0 + k + 1);
        s += (k & 1) ? -term : term;
    }
    return C * s;
}

static void korobov(double u, int r0, int r1, double *phi, double *w) {
    double C = (r0 + r1 + 1) * binom(r0 + r1, r0);
    *w = C * ipow(u, r0) * ipow(1.0 - u, r1);
    if (u <= 0.5) *phi = korobov_phi_direct(u, r0, r1);
    else *phi = 1.0 - korobov_phi_direct(1.0 - u, r1, r0);
}

/* Sidi<r>, Eq. (sidi): w(u) = (pi/2^r) Gamma(r+1)/Gamma((r+1)/2)^2 sin^r(pi u) and
 * phi(u) = int_0^u w, using the textbook reduction
 * I_r(u) = int_0^u sin^r(pi t) dt = -sin^(r-1)(pi u) cos(pi u)/(r pi) + (r-1)/r I_(r-2)(u),
 * I_0(u) = u, I_1(u) = (1 - cos(pi u))/pi. */
static double sidi_I(double u, int r) {
    if (r == 0) return u;
    if (r == 1) return (1.0 - cos(M_PI * u)) / M_PI;
    double s = sin(M_PI * u), c = cos(M_PI * u);
    return -ipow(s, r - 1) * c / (r * M_PI) + (double)(r - 1) / r * sidi_I(u, r - 2);
}

static void sidi(double u, int r, double *phi, double *w) {
    double cr = M_PI / ldexp(1.0, r) * tgamma(r + 1.0) / (tgamma((r + 1.0) / 2.0) * tgamma((r + 1.0) / 2.0));
    *w = cr * ipow(sin(M_PI * u), r);
    *phi = cr * sidi_I(u, r);
}

/* Baker, Eq. (baker): phi(u) = 2u for u <= 1/2, 2 - 2u otherwise; weight 1. */
static void baker(double u, double *phi, double *w) {
    *phi = (u <= 0.5) ? 2.0 * u : 2.0 - 2.0 * u;
    *w = 1.0;
}

typedef struct { int kind, r0, r1; } oracle_transform;

static void apply_transform(const oracle_transform *t, double u, double *phi, double *w) {
    switch (t->kind) {
    case OT_BAKER: baker(u, phi, w); break;
    case OT_KOROBOV: korobov(u, t->r0, t->r1, phi, w); break;
    case OT_SIDI: sidi(u, t->r0, phi, w); break;
    default: *phi = u; *w = 1.0; break;
    }
}

void oracle_transform_eval(int kind, int r0, int r1, double u, double *phi, double *w) {
    oracle_transform t = {kind, r0, r1};
    apply_transform(&t, u, phi, w);
}

/* ------------------------------------------------------------------------------------ */
/* PolySingular fit function (Sec. 2.4, Eq. (ISfit); table of fit functions, App. A.5):  */
/* p(x) = |a2| x (a0-1)/(a0-x) + |a3| x (a1-1)/(a1-x) + x (a4 + x (a5 + x (1-|a2|-|a3|-a4-a5))) */
/* ------------------------------------------------------------------------------------ */
void oracle_polysingular(const double *a, double x, double *p, double *dp) {
    double a2 = fabs(a[2]), a3 = fabs(a[3]);
    double a6 = 1.0 - a2 - a3 - a[4] - a[5];
    *p = a2 * x * (a[0] - 1.0) / (a[0] - x) + a3 * x * (a[1] - 1.0) / (a[1] - x)
       + x * (a[4] + x * (a[5] + x * a6));
    *dp = a2 * (a[0] - 1.0) * a[0] / ((a[0] - x) * (a[0] - x))
        + a3 * (a[1] - 1.0) * a[1] / ((a[1] - x) * (a[1] - x))
        + a[4] + 2.0 * a[5] * x + 3.0 * a6 * x * x;
}

/* ------------------------------------------------------------------------------------ */
/* Integrands.                                                                           */
/* ------------------------------------------------------------------------------------ */
enum {
    OF_GENZ_OSC = 1, OF_GENZ_PRODUCT_PEAK = 2, OF_GENZ_CORNER_PEAK = 3, OF_GENZ_GAUSSIAN = 4,
    OF_GENZ_C0 = 5, OF_GENZ_DISCONTINUOUS = 6,
    OF_MONOMIAL = 10,     /* prod_j x_j  (the paper's minimal example, Sec. 3.2) */
    OF_TRIG = 11,         /* prod_j (1 + a_j cos(2 pi (h_j x_j + theta_j)))       */
    OF_FEYNMAN = 20,      /* complex U^a / F^b with contour deformation           */
    OF_SECTOR = 21        /* real U^a / F^b, positive coefficients, no deformation */
};

typedef struct {
    int family, d;
    const double *c, *w;          /* Genz c_j, w_j; trig amplitudes a_j (c) and phases (w) */
    const int64_t *h;             /* trig integer frequencies */
    int nu, nf;                   /* polynomial families: number of monomials in U and F */
    const double *ucoef, *fcoef;
    const int32_t *uexp, *fexp;   /* [nu][d], [nf][d] exponents */
    double pa, pb, lam;           /* U^pa / F^pb, deformation strength */
} oracle_integrand;

static double genz(const oracle_integrand *f, const double *x) {
    int d = f->d;
    const double *c = f->c, *w = f->w;
    double s, p;
    switch (f->family) {
    case OF_GENZ_OSC:            /* cos(2 pi w_1 + sum c_i x_i) */
        s = 2.0 * M_PI * w[0];
        for (int i = 0; i < d; i++) s += c[i] * x[i];
        return cos(s);
    case OF_GENZ_PRODUCT_PEAK:   /* prod (c_i^-2 + (x_i - w_i)^2)^-1 */
        p = 1.0;
        for (int i = 0; i < d; i++) p *= 1.0 / (1.0 / (c[i] * c[i]) + (x[i] - w[i]) * (x[i] - w[i]));
        return p;
    case OF_GENZ_CORNER_PEAK:    /* (1 + sum c_i x_i)^-(d+1) */
        s = 1.0;
        for (int i = 0; i < d; i++) s += c[i] * x[i];
        return pow(s, -(double)(d + 1));
    case OF_GENZ_GAUSSIAN:       /* exp(-sum c_i^2 (x_i - w_i)^2) */
        s = 0.0;
        for (int i = 0; i < d; i++) s += c[i] * c[i] * (x[i] - w[i]) * (x[i] - w[i]);
        return exp(-s);
    case OF_GENZ_C0:             /* exp(-sum c_i |x_i - w_i|) */
        s = 0.0;
        for (int i = 0; i < d; i++) s += c[i] * fabs(x[i] - w[i]);
        return exp(-s);
    case OF_GENZ_DISCONTINUOUS:  /* 0 if x_1 > w_1 or x_2 > w_2, else exp(sum c_i x_i) */
        if (x[0] > w[0] || (d > 1 && x[1] > w[1])) return 0.0;
        s = 0.0;
        for (int i = 0; i < d; i++) s += c[i] * x[i];
        return exp(s);
    case OF_MONOMIAL:
        p = 1.0;
        for (int i = 0; i < d; i++) p *= x[i];
        return p;
    case OF_TRIG:
        p = 1.0;
        for (int i = 0; i < d; i++) p *= 1.0 + c[i] * cos(2.0 * M_PI * ((double)f->h[i] * x[i] + w[i]));
        return p;
    }
    return NAN;
}

/* Polynomial sum_m coef[m] prod_k x_k^e[m][k] at a complex point, plain loops. */
static double complex cpoly(int nterm, int d, const double *coef, const int32_t *e, const double complex *z) {
    double complex s = 0.0;
    for (int m = 0; m < nterm; m++) {
        double complex t = coef[m];
        for (int k = 0; k < d; k++)
            for (int q = 0; q < e[m * d + k]; q++) t *= z[k];
        s += t;
    }
    return s;
}

/* Real polynomial value, gradient and Hessian at a real point (exact calculus on monomials). */
static void rpoly_derivs(int nterm, int d, const double *coef, const int32_t *e, const double *x,
                         double *val, double *grad, double *hess) {
    *val = 0.0;
    for (int k = 0; k < d; k++) grad[k] = 0.0;
    for (int k = 0; k < d * d; k++) hess[k] = 0.0;
    for (int m = 0; m < nterm; m++) {
        const int32_t *em = e + m * d;
        double t = coef[m];
        for (int k = 0; k < d; k++) t *= ipow(x[k], em[k]);
        *val += t;
        for (int k = 0; k < d; k++) {
            if (em[k] == 0) continue;
            double g = coef[m] * em[k];
            for (int l = 0; l < d; l++) g *= ipow(x[l], em[l] - (l == k ? 1 : 0));
            grad[k] += g;
            for (int l = 0; l < d; l++) {
                int el = em[l] - (l == k ? 1 : 0);
                if (el == 0) continue;
                double hterm = coef[m] * em[k] * el;
                for (int q = 0; q < d; q++) {
                    int eq = em[q] - (q == k ? 1 : 0) - (q == l ? 1 : 0);
                    hterm *= ipow(x[q], eq);
                }
                hess[k * d + l] += hterm;
            }
        }
    }
}

/* Determinant of a complex d x d matrix (row-major, destroyed) by Gaussian elimination
 * with partial pivoting on |a|^2. */
static double complex cdet(double complex *A, int d) {
    double complex det = 1.0;
    for (int c = 0; c < d; c++) {
        int piv = c;
        double best = creal(A[c * d + c]) * creal(A[c * d + c]) + cimag(A[c * d + c]) * cimag(A[c * d + c]);
        for (int r = c + 1; r < d; r++) {
            double v = creal(A[r * d + c]) * creal(A[r * d + c]) + cimag(A[r * d + c]) * cimag(A[r * d + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return 0.0;
        if (piv != c) {
            for (int q = 0; q < d; q++) {
                double complex t = A[c * d + q]; A[c * d + q] = A[piv * d + q]; A[piv * d + q] = t;
            }
            det = -det;
        }
        det *= A[c * d + c];
        for (int r = c + 1; r < d; r++) {
            double complex fac = A[r * d + c] / A[c * d + c];
            for (int q = c; q < d; q++) A[r * d + q] -= fac * A[c * d + q];
        }
    }
    return det;
}

#define OMAXD 16

/* U(z)^a F(z)^-b det(dz/dx) at the deformed point z_k = x_k - i lam x_k (1-x_k) dF/dx_k(x).
 * Jacobian: J_kl = delta_kl - i lam [delta_kl (1 - 2 x_k) dF_k + x_k (1 - x_k) d2F_kl].
 * Powers use the principal branch.  *signfail is set when Im F(z) > 0. */
static double complex feynman(const oracle_integrand *f, const double *x, int *signfail) {
    int d = f->d;
    double Fv, dF[OMAXD], H[OMAXD * OMAXD];
    rpoly_derivs(f->nf, d, f->fcoef, f->fexp, x, &Fv, dF, H);
    double complex z[OMAXD], J[OMAXD * OMAXD];
    for (int k = 0; k < d; k++) z[k] = x[k] - I * f->lam * x[k] * (1.0 - x[k]) * dF[k];
    for (int k = 0; k < d; k++)
        for (int l = 0; l < d; l++) {
            double re = (k == l) ? 1.0 : 0.0;
            double im = x[k] * (1.0 - x[k]) * H[k * d + l] + ((k == l) ? (1.0 - 2.0 * x[k]) * dF[k] : 0.0);
            J[k * d + l] = re - I * f->lam * im;
        }
    double complex U = cpoly(f->nu, d, f->ucoef, f->uexp, z);
    double complex F = cpoly(f->nf, d, f->fcoef, f->fexp, z);
    if (cimag(F) > 0.0) *signfail = 1;
    double complex detJ = cdet(J, d);
    double complex Ua = (f->pa == 1.0) ? U : cexp(f->pa * clog(U));
    double complex Fb = cexp(-f->pb * clog(F));
    return Ua * Fb * detJ;
}

/* Real sector-like integrand U(x)^a / F(x)^b (no deformation). */
static double sector(const oracle_integrand *f, const double *x) {
    double complex z[OMAXD];
    for (int k = 0; k < f->d; k++) z[k] = x[k];
    double U = creal(cpoly(f->nu, f->d, f->ucoef, f->uexp, z));
    double F = creal(cpoly(f->nf, f->d, f->fcoef, f->fexp, z));
    return pow(U, f->pa) * pow(F, -f->pb);
}

static int is_complex(const oracle_integrand *f) { return f->family == OF_FEYNMAN; }

/* Integrand value f(x) (real part in re, imaginary in im). */
static void eval_f(const oracle_integrand *f, const double *x, double *re, double *im, int *signfail) {
    if (f->family == OF_FEYNMAN) {
        double complex v = feynman(f, x, signfail);
        *re = creal(v); *im = cimag(v);
    } else if (f->family == OF_SECTOR) {
        *re = sector(f, x); *im = 0.0;
    } else {
        *re = genz(f, x); *im = 0.0;
    }
}

/* g(u) = prod_j w(u_j) * prod_j p_j'(phi(u_j)) * f(p(phi(u)))  (Sec. 3.3.1: the
 * periodizing transform is applied to the fitted function).  fitp: [d][6] or NULL. */
static void eval_g(const oracle_integrand *f, const oracle_transform *t, const double *fitp,
                   const double *u, double *re, double *im, int *signfail) {
    double x[OMAXD], wt = 1.0;
    for (int j = 0; j < f->d; j++) {
        double phi, w;
        apply_transform(t, u[j], &phi, &w);
        wt *= w;
        if (fitp) {
            double p, dp;
            oracle_polysingular(fitp + 6 * j, phi, &p, &dp);
            wt *= dp;
            phi = p;
        }
        x[j] = phi;
    }
    double fr, fi;
    eval_f(f, x, &fr, &fi, signfail);
    *re = wt * fr;
    *im = wt * fi;
}

void oracle_eval_g(const oracle_integrand *f, int tkind, int r0, int r1, const double *fitp,
                   const double *u, double *re, double *im) {
    oracle_transform t = {tkind, r0, r1};
    int sf = 0;
    eval_g(f, &t, fitp, u, re, im, &sf);
}

/* ------------------------------------------------------------------------------------ */
/* Per-shift sums S_k = sum_{i0 <= i < i1} g(x_{i,k}) in double-double (Eq. (lattice)).  */
/* ------------------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static void dd_add(dd *s, double v) {           /* TwoSum, error kept in lo */
    double t = s->hi + v;
    double bp = t - s->hi;
    double err = (s->hi - (t - bp)) + (v - bp);
    s->hi = t;
    s->lo += err;
}

static void dd_add_dd(dd *s, dd v) {
    dd_add(s, v.hi);
    dd_add(s, v.lo);
}

#define OBLOCK 16384

/* sums: [m][2] = (hi, lo) of the real part; sums_im likewise for complex integrands (may
 * be NULL for real); sums_abs (may be NULL): [m] sum of |g| (modulus), the scale against
 * which agreement with other implementations is judged.  The index range is split in fixed blocks of OBLOCK points whose
 * double-double partials are combined in block order, so the result does not depend on
 * nthreads.  Returns the number of sign-check failures (complex family) or 0. */
long oracle_shift_sums(const oracle_integrand *f, int tkind, int r0, int r1, const double *fitp,
                       uint64_t n, const uint64_t *z, const uint64_t *D, int m,
                       uint64_t i0, uint64_t i1, double *sums, double *sums_im, double *sums_abs,
                       int nthreads) {
    int d = f->d;
    oracle_transform t = {tkind, r0, r1};
    uint64_t nblk = (i1 > i0) ? (i1 - i0 + OBLOCK - 1) / OBLOCK : 0;
    dd *part = (dd *)calloc((size_t)(nblk ? nblk : 1) * m * 3, sizeof(dd));
    long fails = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : fails)
    for (uint64_t b = 0; b < nblk; b++) {
        uint64_t lo = i0 + b * OBLOCK, hi = lo + OBLOCK < i1 ? lo + OBLOCK : i1;
        dd *pr = part + b * m * 3, *pi = pr + m, *pa = pi + m;
        double u[OMAXD];
        for (uint64_t i = lo; i < hi; i++) {
            for (int k = 0; k < m; k++) {
                for (int j = 0; j < d; j++)
                    u[j] = oracle_point(oracle_index(i, z[j], n), n, D[(size_t)k * d + j]);
                double re, im;
                int sf = 0;
                eval_g(f, &t, fitp, u, &re, &im, &sf);
                fails += sf;
                dd_add(&pr[k], re);
                if (is_complex(f)) dd_add(&pi[k], im);
                dd_add(&pa[k], is_complex(f) ? hypot(re, im) : fabs(re));
            }
        }
    }
    for (int k = 0; k < m; k++) {
        dd sr = {0.0, 0.0}, si = {0.0, 0.0}, sa = {0.0, 0.0};
        for (uint64_t b = 0; b < nblk; b++) {
            dd_add_dd(&sr, part[b * m * 3 + k]);
            dd_add_dd(&si, part[b * m * 3 + m + k]);
            dd_add_dd(&sa, part[b * m * 3 + 2 * m + k]);
        }
        sums[2 * k] = sr.hi; sums[2 * k + 1] = sr.lo;
        if (sums_im) { sums_im[2 * k] = si.hi; sums_im[2 * k + 1] = si.lo; }
        if (sums_abs) sums_abs[k] = sa.hi + sa.lo;
    }
    free(part);
    return fails;
}

/* ------------------------------------------------------------------------------------ */
/* evaluate() and the per-dimension histogram of |f| used by the fit (Sec. 2.4; API      */
/* evaluate(), App. A.2).  One shift, no periodizing transform: the fit works on f(x).    */
/* ------------------------------------------------------------------------------------ */
void oracle_evaluate(const oracle_integrand *f, uint64_t n, const uint64_t *z, const uint64_t *D1,
                     uint64_t i0, uint64_t count, double *re, double *im) {
    int d = f->d;
    double x[OMAXD];
    for (uint64_t t = 0; t < count; t++) {
        for (int j = 0; j < d; j++) x[j] = oracle_point(oracle_index(i0 + t, z[j], n), n, D1[j]);
        int sf = 0;
        double a, b;
        eval_f(f, x, &a, &b, &sf);
        re[t] = a;
        if (im) im[t] = b;
    }
}

/* hist[j*B + b] = sum over lattice points with floor(x_j * B) == b (clamped to B-1) of |f(x)|,
 * |f| being the modulus for complex integrands.  Double-double per bin. */
void oracle_histogram(const oracle_integrand *f, uint64_t n, const uint64_t *z, const uint64_t *D1,
                      int B, double *hist) {
    int d = f->d;
    dd *h = (dd *)calloc((size_t)d * B, sizeof(dd));
    double x[OMAXD];
    for (uint64_t i = 0; i < n; i++) {
        for (int j = 0; j < d; j++) x[j] = oracle_point(oracle_index(i, z[j], n), n, D1[j]);
        int sf = 0;
        double a, b;
        eval_f(f, x, &a, &b, &sf);
        double v = is_complex(f) ? hypot(a, b) : fabs(a);
        for (int j = 0; j < d; j++) {
            int bin = (int)floor(x[j] * (double)B);
            if (bin >= B) bin = B - 1;
            dd_add(&h[(size_t)j * B + bin], v);
        }
    }
    for (size_t q = 0; q < (size_t)d * B; q++) hist[q] = h[q].hi + h[q].lo;
    free(h);
}

/* Pieces of the deformed Feynman-like integrand at one real point, for testing each step
 * separately: z[d] (re, im interleaved), J[d*d] (re, im interleaved), U(z), F(z), det J,
 * and the real F, grad F, Hessian F at x. */
void oracle_feynman_parts(const oracle_integrand *f, const double *x, double *z_out, double *J_out,
                          double *U_out, double *F_out, double *det_out,
                          double *Freal, double *grad, double *hess) {
    int d = f->d;
    double Fv, dF[OMAXD], H[OMAXD * OMAXD];
    rpoly_derivs(f->nf, d, f->fcoef, f->fexp, x, &Fv, dF, H);
    double complex z[OMAXD], J[OMAXD * OMAXD];
    for (int k = 0; k < d; k++) z[k] = x[k] - I * f->lam * x[k] * (1.0 - x[k]) * dF[k];
    for (int k = 0; k < d; k++)
        for (int l = 0; l < d; l++) {
            double re = (k == l) ? 1.0 : 0.0;
            double im = x[k] * (1.0 - x[k]) * H[k * d + l] + ((k == l) ? (1.0 - 2.0 * x[k]) * dF[k] : 0.0);
            J[k * d + l] = re - I * f->lam * im;
        }
    for (int k = 0; k < d; k++) { z_out[2 * k] = creal(z[k]); z_out[2 * k + 1] = cimag(z[k]); }
    for (int q = 0; q < d * d; q++) { J_out[2 * q] = creal(J[q]); J_out[2 * q + 1] = cimag(J[q]); }
    double complex U = cpoly(f->nu, d, f->ucoef, f->uexp, z);
    double complex F = cpoly(f->nf, d, f->fcoef, f->fexp, z);
    double complex det = cdet(J, d);
    U_out[0] = creal(U); U_out[1] = cimag(U);
    F_out[0] = creal(F); F_out[1] = cimag(F);
    det_out[0] = creal(det); det_out[1] = cimag(det);
    *Freal = Fv;
    for (int k = 0; k < d; k++) grad[k] = dF[k];
    for (int q = 0; q < d * d; q++) hess[q] = H[q];
}
