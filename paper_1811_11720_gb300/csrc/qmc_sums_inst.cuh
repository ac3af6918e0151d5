// qmc_sums_inst.cuh -- per-translation-unit instantiation of sums_kernel over the
// transforms (the four public kinds and the integer-pipe Korobov) for a list of families
// (split across TUs so nvcc compiles them in parallel).
#pragma once
#include "qmc_internal.h"
#include "qmc_sums.cuh"

namespace qmc {

template <int FAM, int TK>
static cudaError_t launch_one(dim3 grid, dim3 block, cudaStream_t s, const SumsParams &p) {
    sums_kernel<FAM, TK><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <int FAM>
static cudaError_t launch_family(int tkind, dim3 grid, dim3 block, cudaStream_t s,
                                 const SumsParams &p) {
    switch (tkind) {
    case QMC_T_NONE: return launch_one<FAM, QMC_T_NONE>(grid, block, s, p);
    case QMC_T_BAKER: return launch_one<FAM, QMC_T_BAKER>(grid, block, s, p);
    case QMC_T_KOROBOV: return launch_one<FAM, QMC_T_KOROBOV>(grid, block, s, p);
    case QMC_T_SIDI: return launch_one<FAM, QMC_T_SIDI>(grid, block, s, p);
    case kTKorobovInt: return launch_one<FAM, kTKorobovInt>(grid, block, s, p);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
