// qmc_sums.cuh -- the persistent lattice-sum kernel (Eq. (lattice)).
//
// Work decomposition.  The i-range [i_begin, i_end) is cut into tiles of spb * L points;
// a block of spb * m threads owns one tile at a time (tiles are dealt round-robin to a
// persistent grid).  Thread (s, k) evaluates shift k on the L consecutive points of
// stream s, so the 32 lanes of a warp are 32 shifts of the same points when m is a
// multiple of 32: the lattice state is shared across the warp (see stream_sums) and the
// instruction stream is uniform.  The transform and, where the integrand allows, the
// integrand's linear and quadratic forms run in integer fixed point (qmc_fixed.cuh,
// qmc_integrands.cuh), and under the cheaper maps so does its final function (qmc_exp.cuh,
// qmc_cos.cuh); FP64 is left to the final function under the higher Korobov orders and to
// the sums.
// Each thread accumulates its L samples in FP64; the tile's per-shift partial is
// the Neumaier-compensated sum over its spb streams in fixed order, written to
// partials[tile][k].  Tiles depend only on the i-range, so the result is bit-identical for
// any grid size, and sharding on tile boundaries reproduces the same partials.
#pragma once
#include <cstdint>

#include "qmc_integrands.cuh"
#include "qmc_transforms.cuh"

namespace qmc {

constexpr uint64_t kInner = 64;   // samples per inner accumulation block (power of two)

__device__ __forceinline__ bool not_finite(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) ==
           0x7FF0000000000000ull;
}

// Neumaier: add v to (s, c).
__device__ __forceinline__ void neumaier_add(double &s, double &c, double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// Fit constants per dimension in shared memory (see apply_fit).
__device__ __forceinline__ void prepare_fit(const double *fit, int d, double *s_fit) {
    const int tid = threadIdx.x;
    if (fit && tid < d) {
        const double *a = fit + 6 * tid;
        double a2 = fabs(a[2]), a3 = fabs(a[3]);
        double *o = s_fit + kFitStride * tid;
        o[0] = a[0];
        o[1] = a[1];
        o[2] = a2 * (a[0] - 1.0);
        o[3] = a3 * (a[1] - 1.0);
        o[4] = a[4];
        o[5] = a[5];
        o[6] = 1.0 - a2 - a3 - a[4] - a[5];
        o[7] = o[2] * a[0];
        o[8] = o[3] * a[1];
        o[9] = 2.0 * o[5];
        o[10] = 3.0 * o[6];
    }
}

// Per-warp lattice state for the shared-state path: two buffers (the state at point t is
// written to buffer t & 1) of one slot per lane, in shared memory.
struct WarpLattice {
    uint64_t fhi[2][32];
    uint64_t flo[2][32];
    uint64_t rem[2][32];
};

// Lanes per stream group of a warp for the shared-state path: 32 when m is a multiple of
// 32, m when m divides 32 and the stream's shifts can hold the d coordinates; 0 otherwise
// (each thread keeps its own state).
__device__ __forceinline__ int lattice_group_lanes(int m, int d) {
    if (m % 32 == 0) return 32;
    if (32 % m == 0 && d <= m) return m;
    return 0;
}

// Shift accessors: dsh(j) is D_kj 2^11, the thread's 53-bit shift of coordinate j in units
// of the lattice state's top word.
struct ShiftsPre {      // values already multiplied by 2^11 (local or shared memory)
    const uint64_t *s;
    __device__ __forceinline__ uint64_t operator()(int j) const { return s[j]; }
};
struct ShiftsGlobal {   // the caller's row of D_kj in global memory, through the read-only path
    const uint64_t *D;
    __device__ __forceinline__ uint64_t operator()(int j) const { return __ldg(D + j) << 11; }
};

// One evaluation of g at the point whose coordinate j has lattice state (fhi(j), flo(j),
// rem(j)); adds it to the two-level accumulator.
template <int FAM, int TK, int R, class P, class Sh, class Hi, class Lo, class Rem>
__device__ __forceinline__ void eval_point(const P &p, const FamilyShared &fsh, const double *s_fit,
                                           bool use_fit, Sh dsh, double cd, Hi fhi,
                                           Lo flo, Rem rem, double &g_re, double &g_im,
                                           unsigned long long &signfail) {
    Weight W{1.0, 1.0, 1.0, Fx{0x8000000000000000ull, 1}};
    FamilyAcc<FAM> fa;
    if constexpr (kFixedTransform<TK> && kHasFixedForm<FAM>) {
        // coordinate and integrand form entirely in fixed point (no fit: the fit map
        // needs x as a double)
        if (!use_fit && fsh.fx.ok) {
            // the final function (exp, power, cos) on the integer pipe where the map leaves
            // it room; under the higher Korobov orders the integer multiply pipe is the
            // bottleneck and the FP64 form, on the otherwise idle FP64 pipe, is faster (the
            // crossover order per family was measured)
            constexpr bool kIntFinish = TK != kTKorobovInt || R <= FamilyAcc<FAM>::kIntFinishMaxR;
            fa.init_fixed();
#pragma unroll 1
            for (int j = 0; j < p.d; ++j)
                fa.template add_fixed<kIntFinish>(j, transform_fixed<TK, R>(fhi(j) + dsh(j), W), fsh);
            const double wt = weight_finish<TK, R>(W, p.t, cd);
            fa.template finish_fixed<kIntFinish>(p.d, fsh, g_re, g_im, signfail);
            g_re *= wt;
            return;
        }
    }
    if constexpr (kFixedTransform<TK> && FAM == QMC_SECTOR) {
        // the real family with F in fixed point takes the coordinates as x 2^64 from the
        // integer-pipe transform (no fit map)
        if (!use_fit && sector_fixed_ok(fsh.poly, p.d)) {
            uint64_t X[8];
#pragma unroll 1
            for (int j = 0; j < p.d; ++j) X[j] = transform_fixed<TK, R>(fhi(j) + dsh(j), W);
            const double wt = weight_finish<TK, R>(W, p.t, cd);
            g_re = sector_value_x(X, p.d, fsh.poly) * wt;
            g_im = 0.0;
            return;
        }
    }
    if constexpr (kFixedTransform<TK> && FAM == QMC_FEYNMAN) {
        // the complex family's fixed-point form likewise takes x 2^64 from the map
        if (!use_fit && feyn_fixed_ok(fsh.poly, p.d)) {
            uint64_t X[kFeynFixedMaxDim];
#pragma unroll 1
            for (int j = 0; j < p.d; ++j) X[j] = transform_fixed<TK, R>(fhi(j) + dsh(j), W);
            const double wt = weight_finish<TK, R>(W, p.t, cd);
            feynman_value_x(X, p.d, fsh.poly, g_re, g_im, signfail);
            g_re *= wt;
            g_im *= wt;
            return;
        }
    }
    fa.init(fsh);
#pragma unroll 1
    for (int j = 0; j < p.d; ++j) {
        Mapped mx;
        if constexpr (TK == kTKorobovInt && (FAM == QMC_SECTOR || FAM == QMC_FEYNMAN)) {
            // the polynomial families use x itself: formed from x 2^64 by integer
            // operations instead of an FP64 conversion and reflection
            mx = Mapped{fixed_u64_to_double(transform_fixed<TK, R>(fhi(j) + dsh(j), W), 64), false};
        } else if constexpr (TK == kTKorobovInt) {
            mx = korobov_int_x<R>(fhi(j) + dsh(j), W);
        } else {
            const double u = fixed_to_double(fhi(j) + dsh(j), flo(j), rem(j), p.n);
            mx = apply_transform<TK>(u, p.t, W);
        }
        if (use_fit) mx = Mapped{apply_fit(reflected(mx), s_fit + kFitStride * j, W.w), false};
        fa.add(j, mx, fsh);
    }
    const double wt = weight_finish<TK, R>(W, p.t, cd);
    fa.finish(p.d, fsh, g_re, g_im, signfail);
    g_re *= wt;
    if constexpr (FamilyAcc<FAM>::kComplex) g_im *= wt;
}

// One stream of one shift: sum of g over points [i0, i0 + cnt) of the lattice described by
// P (fields n, d, dc[], t).  Two-level FP64 accumulation: blocks of kInner samples, then
// the block sums (rounding error ~ (kInner + L/kInner) ulp instead of L ulp).
//
// Lattice state.  When the q = lattice_group_lanes(m, d) lanes of a warp group are q shifts
// of the same stream (wl != nullptr; q = 32 for m a multiple of 32, q = m for m = 2..16
// with d <= m), the state is shared: the group's lane j < d keeps coordinate j in
// registers, computes its start point and steps it, and publishes it to the warp's shared
// buffer once per point; every lane of the group reads the d coordinates from there
// (broadcast loads), with one __syncwarp over the group per point.  That is one lattice
// step per lane and point instead of d.  Otherwise each thread keeps all d coordinates in
// local memory (L1) and steps them itself.
template <int FAM, int TK, int R, class P, class Sh>
__device__ __forceinline__ void stream_sums_r(const P &p, const FamilyShared &fsh, const double *s_fit,
                                              bool use_fit, Sh dsh, double cd,
                                              uint64_t i0, uint64_t cnt, WarpLattice *wl,
                                              int q, double &acc_re, double &acc_im,
                                              unsigned long long &nonfinite,
                                              unsigned long long &signfail) {
    constexpr bool kCplx = FamilyAcc<FAM>::kComplex;
    const int d = p.d;
    const uint64_t n = p.n;
    double in_re = 0.0, in_im = 0.0;
    acc_re = 0.0;
    acc_im = 0.0;
    if (!cnt) return;
    auto accumulate = [&](uint64_t t, double g_re, double g_im) {
        if (not_finite(g_re) || (kCplx && not_finite(g_im))) ++nonfinite;
        in_re += g_re;
        if constexpr (kCplx) in_im += g_im;
        if ((t & (kInner - 1)) == kInner - 1) {
            acc_re += in_re;
            in_re = 0.0;
            if constexpr (kCplx) {
                acc_im += in_im;
                in_im = 0.0;
            }
        }
    };
    if (wl && q == 32) {
        // the warp is one group: lane j < d owns coordinate j
        const int lane = threadIdx.x & 31;
        uint64_t fh = 0, fl = 0, rm = 0;
        if (lane < d) lattice_state_at(i0, p.dc[lane], n, fh, fl, rm);
#pragma unroll 1
        for (uint64_t t = 0; t < cnt; ++t) {
            const int b = (int)(t & 1);
            if (lane < d) {
                wl->fhi[b][lane] = fh;
                if constexpr (TK != kTKorobovInt) {
                    wl->flo[b][lane] = fl;
                    wl->rem[b][lane] = rm;
                }
            }
            __syncwarp();
            double g_re, g_im = 0.0;
            eval_point<FAM, TK, R>(
                p, fsh, s_fit, use_fit, dsh, cd, [&](int j) { return wl->fhi[b][j]; },
                [&](int j) { return wl->flo[b][j]; }, [&](int j) { return wl->rem[b][j]; }, g_re,
                g_im, signfail);
            accumulate(t, g_re, g_im);
            if (lane < d) lattice_step(p.dc[lane], n, fh, fl, rm);
        }
    } else if (wl) {
        // groups of q < 32 lanes (q divides 32): the group's lane j < d owns coordinate j
        const int lane = threadIdx.x & 31;
        const int base = lane & ~(q - 1);
        const int pos = lane - base;
        const unsigned mask = ((1u << q) - 1u) << base;
        uint64_t fh = 0, fl = 0, rm = 0;
        if (pos < d) lattice_state_at(i0, p.dc[pos], n, fh, fl, rm);
#pragma unroll 1
        for (uint64_t t = 0; t < cnt; ++t) {
            const int b = (int)(t & 1);
            if (pos < d) {
                wl->fhi[b][lane] = fh;
                if constexpr (TK != kTKorobovInt) {
                    wl->flo[b][lane] = fl;
                    wl->rem[b][lane] = rm;
                }
            }
            __syncwarp(mask);
            double g_re, g_im = 0.0;
            eval_point<FAM, TK, R>(
                p, fsh, s_fit, use_fit, dsh, cd, [&](int j) { return wl->fhi[b][base + j]; },
                [&](int j) { return wl->flo[b][base + j]; },
                [&](int j) { return wl->rem[b][base + j]; }, g_re, g_im, signfail);
            accumulate(t, g_re, g_im);
            if (pos < d) lattice_step(p.dc[pos], n, fh, fl, rm);
        }
    } else {
        uint64_t fhi[kMaxDim], flo[kMaxDim], rem[kMaxDim];
#pragma unroll 1
        for (int j = 0; j < d; ++j) lattice_state_at(i0, p.dc[j], n, fhi[j], flo[j], rem[j]);
#pragma unroll 1
        for (uint64_t t = 0; t < cnt; ++t) {
            double g_re, g_im = 0.0;
            eval_point<FAM, TK, R>(
                p, fsh, s_fit, use_fit, dsh, cd, [&](int j) { return fhi[j]; },
                [&](int j) { return flo[j]; }, [&](int j) { return rem[j]; }, g_re, g_im, signfail);
            accumulate(t, g_re, g_im);
#pragma unroll 1
            for (int j = 0; j < d; ++j) lattice_step(p.dc[j], n, fhi[j], flo[j], rem[j]);
        }
    }
    acc_re += in_re;
    if constexpr (kCplx) acc_im += in_im;
}

// The integer Korobov is compiled once per order r (uniform branch per stream).
template <int FAM, int TK, class P, class Sh>
__device__ __forceinline__ void stream_sums(const P &p, const FamilyShared &fsh, const double *s_fit,
                                            bool use_fit, Sh dsh, double cd,
                                            uint64_t i0, uint64_t cnt, WarpLattice *wl, int q,
                                            double &acc_re, double &acc_im,
                                            unsigned long long &nonfinite,
                                            unsigned long long &signfail) {
    if constexpr (TK == kTKorobovInt) {
        switch (p.t.r0) {
        case 1:
            stream_sums_r<FAM, TK, 1>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        case 2:
            stream_sums_r<FAM, TK, 2>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        case 3:
            stream_sums_r<FAM, TK, 3>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        case 4:
            stream_sums_r<FAM, TK, 4>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        case 5:
            stream_sums_r<FAM, TK, 5>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        default:
            stream_sums_r<FAM, TK, 6>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                      nonfinite, signfail);
            return;
        }
    } else {
        stream_sums_r<FAM, TK, 0>(p, fsh, s_fit, use_fit, dsh, cd, i0, cnt, wl, q, acc_re, acc_im,
                                  nonfinite, signfail);
    }
}

// Per-shift tile partial: fixed-order compensated sum over the block's spb streams of
// shift k, written as (sum, compensation) to out_re[2k..] (and out_im).  Contains the
// block barriers; every thread of the block must call it.
template <bool CPLX>
__device__ __forceinline__ void tile_partial(double acc_re, double acc_im, double *s_red, int m,
                                             int spb, int s_local, int k, bool active,
                                             double *out_re, double *out_im) {
    const int tid = threadIdx.x;
    s_red[tid] = acc_re;
    if constexpr (CPLX) s_red[kSumsThreads + tid] = acc_im;
    __syncthreads();
    if (s_local == 0 && active) {
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        for (int s = 0; s < spb; ++s) {
            neumaier_add(sr, cr, s_red[s * m + k]);
            if constexpr (CPLX) neumaier_add(si, ci, s_red[kSumsThreads + s * m + k]);
        }
        out_re[2 * k] = sr;
        out_re[2 * k + 1] = cr;
        if constexpr (CPLX) {
            out_im[2 * k] = si;
            out_im[2 * k + 1] = ci;
        }
    }
    __syncthreads();
}

// Blocks per SM the register allocation must allow: five for the separable families (48
// registers; their throughput depends on hiding integer latency), no constraint for the
// polynomial families (their per-thread working set needs the registers).
template <int FAM>
constexpr bool kPolyFamily = FAM == QMC_SECTOR || FAM == QMC_FEYNMAN;
template <int FAM>
constexpr int kSumsMinBlocks = kPolyFamily<FAM> ? 1 : 5;

template <int FAM, int TK>
__global__ void __launch_bounds__(kSumsThreads, kSumsMinBlocks<FAM>)
    sums_kernel(const __grid_constant__ SumsParams p) {
    __shared__ FamilyShared fsh;
    __shared__ double s_fit[kMaxDim * kFitStride];
    __shared__ double s_red[2 * kSumsThreads];
    __shared__ WarpLattice s_lat[kSumsThreads / 32];
    constexpr bool kCplx = FamilyAcc<FAM>::kComplex;

    const int tid = threadIdx.x;
    stage_family<FAM, false>(p, fsh);
    prepare_fit(p.fit, p.d, s_fit);
    __syncthreads();
    if constexpr (kHasFixedForm<FAM>) {
        // the FP64 forms' subset-sum tables (256 FP64 sums per block), only when the
        // fixed-point form does not take every evaluation (uniform over the block)
        if (!(kFixedTransform<TK> && p.fit == nullptr && fsh.fx.ok)) {
            stage_subset_sums<FAM>(p, fsh);
            __syncthreads();
        }
    }

    const int m = p.m, d = p.d;
    const int k = tid % m;
    const int s_local = tid / m;
    const bool active = s_local < p.spb;
    const double cd = p.cd;   // Korobov C^d (host-computed; 1 otherwise)

    // The shifts D_kj, read once per dimension of every evaluation.  Under the cheap maps
    // (baker, none) the separable families stage them, times 2^11 (the 53-bit shift in the
    // high word's units), in shared memory, in the polynomial buffer they do not use, as
    // [k][j] rows of odd length (the warp's lanes hit distinct banks).  Otherwise each
    // thread reads its row of the caller's array through the read-only cache: the block's
    // m rows (m d 8 bytes) are shared by all its warps and stay in L1, where a copy per
    // thread in local memory (spb times as much) missed.
    unsigned long long nonfinite = 0, signfail = 0;
    const uint64_t ptile = (uint64_t)p.spb * p.L;
    const int q = lattice_group_lanes(m, d);
    auto run_tiles = [&](auto dsh) {
        for (uint64_t tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
            const uint64_t i0 = p.i_begin + tile * ptile + (uint64_t)s_local * p.L;
            uint64_t cnt = 0;
            if (active && i0 < p.i_end) cnt = (p.i_end - i0 < p.L) ? (p.i_end - i0) : p.L;
            double acc_re, acc_im;
            stream_sums<FAM, TK>(p, fsh, s_fit, p.fit != nullptr, dsh, cd, i0, cnt,
                                 q ? &s_lat[tid >> 5] : nullptr, q, acc_re, acc_im, nonfinite,
                                 signfail);
            double *out_re = p.partials + 2 * (tile * (uint64_t)m);
            double *out_im = p.partials + 2 * (p.tiles * (uint64_t)m) + 2 * (tile * (uint64_t)m);
            tile_partial<kCplx>(acc_re, acc_im, s_red, m, p.spb, s_local, k, active, out_re, out_im);
        }
    };
    bool staged = false;
    if constexpr (!kPolyFamily<FAM> && (TK == QMC_T_BAKER || TK == QMC_T_NONE)) {
        const int ds = d | 1;
        if (m * ds <= 4 * kMaxTerms) {   // uniform over the block
            uint64_t *s_dsh = fsh.poly.buf.u;
            for (int i = tid; i < m * ds; i += blockDim.x) {
                const int kk = i / ds, j = i - kk * ds;
                s_dsh[i] = j < d ? (p.shifts[(size_t)kk * d + j] << 11) : 0ull;
            }
            __syncthreads();
            run_tiles(ShiftsPre{s_dsh + k * ds});
            staged = true;
        }
    }
    if (!staged) run_tiles(ShiftsGlobal{p.shifts + (size_t)k * d});
    if (p.counters && (nonfinite | signfail)) {
        if (nonfinite) atomicAdd(p.counters, nonfinite);
        if (signfail) atomicAdd(p.counters + 1, signfail);
    }
}

}  // namespace qmc
