// qmc_internal.h -- host-side declarations shared by the C-ABI and the kernel TUs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "qmc_params.cuh"

namespace qmc {

// Launches sums_kernel<FAM, TK> for the family group compiled in one translation unit.
// Returns cudaErrorInvalidValue when (family, transform) is not in that group.
cudaError_t launch_sums_genz(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                             const SumsParams &p);
cudaError_t launch_sums_other(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                              const SumsParams &p);
cudaError_t launch_sums_poly(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                             const SumsParams &p);

struct PointsParams {
    uint64_t n, i_begin, count;
    int d, m;
    uint32_t L;
    DimConst dc[kMaxDim];
    const uint64_t *shifts;
    double *out;
};
cudaError_t launch_points(const PointsParams &p, cudaStream_t s);

// Reduce per-tile partials [tiles][m] (sum, comp) (and the im block) to double-double
// sums [2m] (and [2m..4m) for im), fixed order.
cudaError_t launch_reduce_tiles(const double *partials, uint64_t tiles, int m, int is_complex,
                                double *sums, cudaStream_t s);
cudaError_t launch_finalize(const double *sums, int m, uint64_t n, int is_complex,
                            double *result, double *Q, cudaStream_t s);

cudaError_t launch_evaluate(const SumsParams &p, double *out, cudaStream_t s);
cudaError_t launch_histogram(const SumsParams &p, int bins, double *hist, double *work,
                             uint32_t nblocks, cudaStream_t s);

int sm_count();

// Batch building blocks shared by qmc_batch_sums and the serving loop.  Item partial
// offsets are relative to `partials`.
int fill_batch_item(BatchItem &it, const qmc_batch_item &b, int m, int spb, uint32_t Lcfg, int fam);
bool batch_family_supported(int fam);
cudaError_t launch_batch(int family, const BatchItem *items, const uint64_t *tile_begin, int count,
                         uint64_t tiles, int m, int spb, double *partials,
                         unsigned long long *counters, cudaStream_t s);
cudaError_t launch_batch_reduce(const BatchItem *d_items, int count, int m, int cplx,
                                const double *partials, double *sums, cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchItem *d_items, int count, int m, int cplx,
                                  const double *sums, double *results, cudaStream_t s);

}  // namespace qmc
