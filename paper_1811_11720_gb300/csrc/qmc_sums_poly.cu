// Polynomial families: real sector-like U^a/F^b and the complex deformed-contour integrand.
#include "qmc_sums_inst.cuh"

namespace qmc {
cudaError_t launch_sums_poly(int family, int tkind, dim3 grid, dim3 block, cudaStream_t s,
                             const SumsParams &p) {
    switch (family) {
    case QMC_SECTOR: return launch_family<QMC_SECTOR>(tkind, grid, block, s, p);
    case QMC_FEYNMAN: return launch_family<QMC_FEYNMAN>(tkind, grid, block, s, p);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace qmc
