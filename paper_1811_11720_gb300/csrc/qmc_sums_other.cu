// Genz families 5-6, the minimal-example monomial and the trigonometric test product.
#include "qmc_sums_inst.cuh"

namespace qmc {
cudaError_t launch_sums_other(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                              const SumsParams &p) {
    switch (family) {
    case QMC_GENZ_C0: return launch_family<QMC_GENZ_C0>(tkind, grid, block, s, p);
    case QMC_GENZ_DISCONTINUOUS: return launch_family<QMC_GENZ_DISCONTINUOUS>(tkind, grid, block, s, p);
    case QMC_MONOMIAL: return launch_family<QMC_MONOMIAL>(tkind, grid, block, s, p);
    case QMC_TRIG: return launch_family<QMC_TRIG>(tkind, grid, block, s, p);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace qmc
