// qmc_params.cuh -- launch parameters shared by the host dispatch and the kernels.
#pragma once
#include <cstdint>

#include "qmc_gb300.h"
#include "qmc_lattice.cuh"

namespace qmc {

constexpr int kMaxDim = QMC_MAX_DIM;
constexpr int kMaxKorobov = 8;
constexpr int kMaxSidi = 8;
constexpr int kSumsThreads = 256;   // threads per block of the lattice-sum kernel

// Internal transform kind: symmetric Korobov<r,r>, 1 <= r <= kMaxKorobovInt, evaluated in
// integer fixed point (qmc_fixed.cuh).  The public kind stays QMC_T_KOROBOV.
constexpr int kTKorobovInt = 4;
constexpr int kMaxKorobovInt = 6;

// Korobov<r0,r1> (Eq. (korobov)) as used by the kernels: for u <= 1/2,
//   phi(u) = u^(r0+1) sum_k A[k] u^k,  A[k] = C (-1)^k binom(r1,k) / (r0+k+1), k <= r1,
// and for u > 1/2 the reflection phi(u) = 1 - v^(r1+1) sum_k B[k] v^k with v = 1 - u
// (B: r0 and r1 exchanged).  The weight is C u^r0 (1-u)^r1, C = (r0+r1+1) binom(r0+r1,r0).
struct TransformParams {
    int kind, r0, r1, deg;        // deg = max(r0, r1): Horner length (zero-padded)
    double A[kMaxKorobov + 1];
    double B[kMaxKorobov + 1];
    double C;                     // Korobov constant, or Sidi (pi/2^r) Gamma(r+1)/Gamma((r+1)/2)^2
    double sidi_c[kMaxSidi + 1];  // Sidi: phi = cr * I_r, I_r via the sin-power reduction
};

struct SumsParams {
    uint64_t n;
    uint64_t i_begin, i_end;
    uint64_t tiles;
    uint32_t L;        // points per stream and tile
    int d, m, spb;     // dimension, shifts, streams per block (blockDim = spb * m)
    DimConst dc[kMaxDim];
    const uint64_t *shifts;   // [m][d]
    TransformParams t;
    double cd;                // Korobov C^d, 1 for the other transforms
    const double *fit;        // [d][6] or nullptr
    // integrand (device pointers; the kernel stages them in shared memory)
    int family;
    const double *c, *w;
    const int64_t *h;
    int nu, nf;
    const double *ucoef, *fcoef;
    const int32_t *uexp, *fexp;
    double pa, pb, lam;
    // outputs
    double *partials;                 // [tiles][m] (sum, comp) re, then [tiles][m] im
    unsigned long long *counters;     // [2] or nullptr
};

// One integral of a batch (qmc_batch_sums), built on the host and kept in the workspace.
// Field names match SumsParams so the staging and per-stream code serve both kernels.
struct BatchItem {
    uint64_t n, i_begin, i_end;
    uint64_t tile_begin, tiles;   // global index of the first tile, number of tiles
    uint64_t partial_off;         // offset of this item's partials, in doubles
    uint32_t L;                   // points per stream and tile
    int d;
    double cd;                    // Korobov C^d
    DimConst dc[kMaxDim];
    const uint64_t *shifts;       // [m][d]
    TransformParams t;
    const double *fit;            // [d][6] or nullptr
    int family;
    const double *c, *w;
    const int64_t *h;
    int nu, nf;
    const double *ucoef, *fcoef;
    const int32_t *uexp, *fexp;
    double pa, pb, lam;
};

}  // namespace qmc
