// qmc_batch.cuh -- one launch over many integrals (batching of heterogeneous integrands).
//
// The tiles of all integrals form one global tile sequence; block b takes tile b (grid-stride
// for very large batches), finds its integral by binary search over the tiles' prefix sums,
// copies that integral's descriptor into shared memory, stages its coefficients, and runs
// the same per-stream code as the single-integral kernel.  Integrals differ in dimension,
// lattice size, transform, fit and coefficients; they share the family (a template
// parameter) and the number of shifts m (the block shape).  Tiles of small integrals fill
// the GPU alongside large ones, which one launch per integral cannot do.
#pragma once
#include <cstdint>

#include "qmc_sums.cuh"

namespace qmc {

template <int FAM, int TK>
__device__ __forceinline__ void batch_stream(const BatchItem &it, const FamilyShared &fsh,
                                             const double *s_fit, const uint64_t *dsh,
                                             uint64_t i0, uint64_t cnt, WarpLattice *wl,
                                             int q, double &acc_re, double &acc_im,
                                             unsigned long long &nonfinite,
                                             unsigned long long &signfail) {
    stream_sums<FAM, TK>(it, fsh, s_fit, it.fit != nullptr, ShiftsPre{dsh}, it.cd, i0, cnt, wl, q, acc_re,
                         acc_im, nonfinite, signfail);
}

template <int FAM>
__global__ void __launch_bounds__(kSumsThreads)
    batch_kernel(const BatchItem *items, const uint64_t *tile_begin, int count,
                 uint64_t total_tiles, int m, int spb, double *partials,
                 unsigned long long *counters) {
    __shared__ FamilyShared fsh;
    __shared__ double s_fit[kMaxDim * kFitStride];
    __shared__ double s_red[2 * kSumsThreads];
    __shared__ WarpLattice s_lat[kSumsThreads / 32];
    __shared__ BatchItem s_item;
    __shared__ int s_q;
    constexpr bool kCplx = FamilyAcc<FAM>::kComplex;
    const int tid = threadIdx.x;
    const int k = tid % m;
    const int s_local = tid / m;
    const bool active = s_local < spb;

    for (uint64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        if (tid == 0) {
            int lo = 0, hi = count;   // largest q with tile_begin[q] <= tile
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (tile_begin[mid] <= tile) lo = mid;
                else hi = mid;
            }
            s_q = lo;
        }
        __syncthreads();
        const int q = s_q;
        {
            const uint64_t *src = reinterpret_cast<const uint64_t *>(items + q);
            uint64_t *dst = reinterpret_cast<uint64_t *>(&s_item);
            for (int w = tid; w < (int)(sizeof(BatchItem) / 8); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        const BatchItem &it = s_item;
        stage_family<FAM>(it, fsh);
        prepare_fit(it.fit, it.d, s_fit);
        __syncthreads();

        const int d = it.d;
        uint64_t dsh[kMaxDim];
#pragma unroll 1
        for (int j = 0; j < d; ++j) dsh[j] = active ? (it.shifts[(size_t)k * d + j] << 11) : 0ull;
        const uint64_t local = tile - it.tile_begin;
        const uint64_t i0 = it.i_begin + local * (uint64_t)spb * it.L + (uint64_t)s_local * it.L;
        uint64_t cnt = 0;
        if (active && i0 < it.i_end) cnt = (it.i_end - i0 < it.L) ? (it.i_end - i0) : it.L;
        double acc_re = 0.0, acc_im = 0.0;
        unsigned long long nonfinite = 0, signfail = 0;
        const int qlanes = lattice_group_lanes(m, d);
        WarpLattice *wl = qlanes ? &s_lat[tid >> 5] : nullptr;
        switch (it.t.kind) {
        case QMC_T_NONE:
            batch_stream<FAM, QMC_T_NONE>(it, fsh, s_fit, dsh, i0, cnt, wl, qlanes, acc_re, acc_im, nonfinite, signfail);
            break;
        case QMC_T_BAKER:
            batch_stream<FAM, QMC_T_BAKER>(it, fsh, s_fit, dsh, i0, cnt, wl, qlanes, acc_re, acc_im, nonfinite, signfail);
            break;
        case QMC_T_KOROBOV:
            batch_stream<FAM, QMC_T_KOROBOV>(it, fsh, s_fit, dsh, i0, cnt, wl, qlanes, acc_re, acc_im, nonfinite, signfail);
            break;
        case kTKorobovInt:
            batch_stream<FAM, kTKorobovInt>(it, fsh, s_fit, dsh, i0, cnt, wl, qlanes, acc_re, acc_im, nonfinite, signfail);
            break;
        default:
            batch_stream<FAM, QMC_T_SIDI>(it, fsh, s_fit, dsh, i0, cnt, wl, qlanes, acc_re, acc_im, nonfinite, signfail);
            break;
        }
        double *base = partials + it.partial_off;
        double *out_re = base + 2 * (local * (uint64_t)m);
        double *out_im = base + 2 * (it.tiles * (uint64_t)m) + 2 * (local * (uint64_t)m);
        tile_partial<kCplx>(acc_re, acc_im, s_red, m, spb, s_local, k, active, out_re, out_im);
        if (counters && (nonfinite | signfail)) {
            if (nonfinite) atomicAdd(counters + 2 * q, nonfinite);
            if (signfail) atomicAdd(counters + 2 * q + 1, signfail);
        }
    }
}

}  // namespace qmc
