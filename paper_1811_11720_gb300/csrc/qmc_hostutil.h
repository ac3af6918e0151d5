// qmc_hostutil.h -- host-side helpers shared by the C-ABI translation units: argument
// checks, exact lattice constants, transform coefficient tables and the tile geometry.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "qmc_gb300.h"
#include "qmc_internal.h"

namespace qmc {
namespace host {

typedef unsigned __int128 u128_t;

constexpr uint64_t kNMax = (uint64_t)1 << 63;

inline uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// floor(z 2^128 / n) and z 2^128 mod n for z < n, by two 128/64 divisions.
inline DimConst dim_const(uint64_t z, uint64_t n) {
    u128_t a = (u128_t)z << 64;
    uint64_t q1 = (uint64_t)(a / n);
    uint64_t r1 = (uint64_t)(a % n);
    u128_t b = (u128_t)r1 << 64;
    uint64_t q0 = (uint64_t)(b / n);
    uint64_t r0 = (uint64_t)(b % n);
    return DimConst{q1, q0, r0};
}

inline double binom(int a, int b) {
    double r = 1.0;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

inline int check_transform(const qmc_transform &t) {
    switch (t.kind) {
    case QMC_T_NONE:
    case QMC_T_BAKER: return QMC_OK;
    case QMC_T_KOROBOV:
        return (t.r0 >= 0 && t.r1 >= 0 && t.r0 <= kMaxKorobov && t.r1 <= kMaxKorobov) ? QMC_OK : QMC_ERR_TRANSFORM;
    case QMC_T_SIDI: return (t.r0 >= 1 && t.r0 <= kMaxSidi) ? QMC_OK : QMC_ERR_TRANSFORM;
    default: return QMC_ERR_TRANSFORM;
    }
}

inline TransformParams make_transform(const qmc_transform &t) {
    TransformParams tp;
    std::memset(&tp, 0, sizeof(tp));
    tp.kind = t.kind;
    tp.r0 = t.r0;
    tp.r1 = t.r1;
    if (t.kind == QMC_T_KOROBOV) {
        const int r0 = t.r0, r1 = t.r1;
        tp.C = (r0 + r1 + 1) * binom(r0 + r1, r0);
        tp.deg = std::max(r0, r1);
        // phi(u) = u^(r0+1) sum_k A_k u^k with A_k = C (-1)^k C(r1,k)/(r0+k+1): the
        // binomial expansion of (1-t)^r1 integrated term by term (Eq. (korobov)).
        for (int k = 0; k <= r1; ++k) tp.A[k] = tp.C * ((k & 1) ? -1.0 : 1.0) * binom(r1, k) / (r0 + k + 1);
        for (int k = 0; k <= r0; ++k) tp.B[k] = tp.C * ((k & 1) ? -1.0 : 1.0) * binom(r0, k) / (r1 + k + 1);
        // Korobov<r,r> with r <= 6 has integer polynomial coefficients (in 1 - u) and runs on the
        // integer pipe (the coefficients are compile-time constants of the kernel)
        if (r0 == r1 && r0 >= 1 && r0 <= kMaxKorobovInt) tp.kind = kTKorobovInt;
    } else if (t.kind == QMC_T_SIDI) {
        const int r = t.r0;
        tp.r1 = r;
        // c_r = (pi / 2^r) Gamma(r+1) / Gamma((r+1)/2)^2 (Eq. (sidi))
        double g = std::tgamma((r + 1.0) / 2.0);
        tp.C = M_PI / std::ldexp(1.0, r) * std::tgamma(r + 1.0) / (g * g);
        // I_r = -s^(r-1) c/(r pi) + (r-1)/r I_(r-2): a_q and the trailing factor
        double carry = 1.0;
        int nq = r / 2;
        for (int q = 0; q < nq; ++q) {
            int rr = r - 2 * q;
            tp.sidi_c[q] = carry / rr;
            carry *= (double)(rr - 1) / rr;
        }
        if (nq == 0) tp.sidi_c[0] = 0.0;
        tp.sidi_c[kMaxSidi] = carry;
    }
    return tp;
}

// C^d of the Korobov weight (1 for the other transforms) by left-to-right binary powering:
// computed once per launch on the host, the same value for qmc_sums and batches.
inline double ipow_host(double x, int e) {
    if (e <= 0) return 1.0;
    int top = 31;
    while (!((e >> top) & 1)) --top;
    double r = x;
    for (int b = top - 1; b >= 0; --b) {
        r *= r;
        if ((e >> b) & 1) r *= x;
    }
    return r;
}
inline double korobov_cd(const qmc_transform &t, const TransformParams &tp, int d) {
    return t.kind == QMC_T_KOROBOV ? ipow_host(tp.C, d) : 1.0;
}

inline bool is_complex_family(int fam) { return fam == QMC_FEYNMAN; }

inline bool family_known(int fam) {
    switch (fam) {
    case QMC_GENZ_OSCILLATORY: case QMC_GENZ_PRODUCT_PEAK: case QMC_GENZ_CORNER_PEAK:
    case QMC_GENZ_GAUSSIAN: case QMC_GENZ_C0: case QMC_GENZ_DISCONTINUOUS: case QMC_MONOMIAL:
    case QMC_TRIG: case QMC_SECTOR: case QMC_FEYNMAN: return true;
    default: return false;
    }
}

inline int check_integrand_shape(const qmc_integrand *f) {
    if (!f) return QMC_ERR_ARG;
    if (!family_known(f->family)) return QMC_ERR_INTEGRAND;
    if (f->dim < 1 || f->dim > QMC_MAX_DIM) return QMC_ERR_DIM;
    switch (f->family) {
    case QMC_MONOMIAL: return QMC_OK;
    case QMC_TRIG: return (f->c && f->w && f->h) ? QMC_OK : QMC_ERR_INTEGRAND;
    case QMC_SECTOR:
    case QMC_FEYNMAN:
        if (f->nu < 1 || f->nf < 1 || f->nu > QMC_MAX_TERMS || f->nf > QMC_MAX_TERMS) return QMC_ERR_INTEGRAND;
        return (f->ucoef && f->fcoef && f->uexp && f->fexp) ? QMC_OK : QMC_ERR_INTEGRAND;
    case QMC_GENZ_OSCILLATORY:
        return (f->c && f->w) ? QMC_OK : QMC_ERR_INTEGRAND;
    default:
        return (f->c && f->w) ? QMC_OK : QMC_ERR_INTEGRAND;
    }
}

inline int check_rule(const qmc_rule *r) {
    if (!r) return QMC_ERR_ARG;
    if (r->dim < 1 || r->dim > QMC_MAX_DIM) return QMC_ERR_DIM;
    if (r->n < 2 || r->n >= kNMax) return QMC_ERR_N;
    if (r->m < 1 || r->m > QMC_MAX_SHIFTS) return QMC_ERR_M;
    if (!r->shifts) return QMC_ERR_ARG;
    for (int j = 0; j < r->dim; ++j) {
        uint64_t z = r->z[j] % r->n;
        if (z == 0 || gcd_u64(z, r->n) != 1) return QMC_ERR_GENVEC;
    }
    return check_transform(r->transform);
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA; }

inline int device_ok() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_NO_DEVICE;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return QMC_ERR_NO_DEVICE;
    return (major == 10 && minor == 3) ? QMC_OK : QMC_ERR_NO_DEVICE;
}

// Tile geometry, a function of (range, m) only.
struct Geometry {
    int spb;          // streams per block
    int threads;      // spb * mg
    uint32_t L;       // points per stream per tile
    uint64_t tiles;
};

constexpr int kMaxShiftGroup = kSumsThreads;   // shifts per launch (block holds spb * m threads)
// Tiles come in whole waves of kWaveTiles blocks (152 SMs x 5 resident blocks of the
// separable families on GB300): one wave for small ranges, up to kMaxWaves for large ones,
// so that the last wave is (nearly) full; streams of 8..8192 points.
constexpr uint64_t kWaveTiles = 152 * 5;
constexpr uint64_t kMaxWaves = 6;
constexpr uint64_t kWavePoints = 64;             // points per stream before a new wave
constexpr uint64_t kMinPointsPerStream = 8;
constexpr uint64_t kMaxPointsPerStream = 8192;

// Points per stream for a range split over spb streams per tile (a function of the range
// and spb only, so results do not depend on the device or the grid).
inline uint32_t points_per_stream(uint64_t range, uint64_t spb) {
    const uint64_t wave = spb * kWaveTiles * kWavePoints;
    const uint64_t waves = std::max<uint64_t>(1, std::min<uint64_t>(kMaxWaves, (range + wave - 1) / wave));
    const uint64_t target = waves * kWaveTiles;
    uint64_t per = (range + spb * target - 1) / (spb * target);
    per = std::max<uint64_t>(kMinPointsPerStream, std::min<uint64_t>(kMaxPointsPerStream, per));
    return (uint32_t)per;
}

inline Geometry geometry(uint64_t range, int mg) {
    Geometry g;
    g.spb = std::max(1, kSumsThreads / mg);
    g.threads = g.spb * mg;
    g.L = points_per_stream(range, (uint64_t)g.spb);
    uint64_t ptile = (uint64_t)g.spb * g.L;
    g.tiles = range ? (range + ptile - 1) / ptile : 0;
    return g;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

inline void fill_integrand(SumsParams &p, const qmc_integrand *f) {
    p.family = f->family;
    p.c = f->c;
    p.w = f->w;
    p.h = f->h;
    p.nu = f->nu;
    p.nf = f->nf;
    p.ucoef = f->ucoef;
    p.fcoef = f->fcoef;
    p.uexp = f->uexp;
    p.fexp = f->fexp;
    p.pa = f->pa;
    p.pb = f->pb;
    p.lam = f->lambda;
}

inline cudaError_t launch_sums_any(int family, int tkind, dim3 g, dim3 b, cudaStream_t s, const SumsParams &p) {
    switch (family) {
    case QMC_GENZ_OSCILLATORY: case QMC_GENZ_PRODUCT_PEAK: case QMC_GENZ_CORNER_PEAK: case QMC_GENZ_GAUSSIAN:
        return launch_sums_genz(family, tkind, g, b, s, p);
    case QMC_GENZ_C0: case QMC_GENZ_DISCONTINUOUS: case QMC_MONOMIAL: case QMC_TRIG:
        return launch_sums_other(family, tkind, g, b, s, p);
    case QMC_SECTOR: case QMC_FEYNMAN:
        return launch_sums_poly(family, tkind, g, b, s, p);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace host
}  // namespace qmc
