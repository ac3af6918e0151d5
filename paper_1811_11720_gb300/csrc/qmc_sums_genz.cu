// Genz families 1-4 (Sec. 5.2): the benchmark families.
#include "qmc_sums_inst.cuh"

namespace qmc {
cudaError_t launch_sums_genz(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                             const SumsParams &p) {
    switch (family) {
    case QMC_GENZ_OSCILLATORY: return launch_family<QMC_GENZ_OSCILLATORY>(tkind, grid, block, s, p);
    case QMC_GENZ_PRODUCT_PEAK: return launch_family<QMC_GENZ_PRODUCT_PEAK>(tkind, grid, block, s, p);
    case QMC_GENZ_CORNER_PEAK: return launch_family<QMC_GENZ_CORNER_PEAK>(tkind, grid, block, s, p);
    case QMC_GENZ_GAUSSIAN: return launch_family<QMC_GENZ_GAUSSIAN>(tkind, grid, block, s, p);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace qmc
