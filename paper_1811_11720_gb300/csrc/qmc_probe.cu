// qmc_probe.cu -- qmc_probe_units(): throughput of the two arithmetic units the lattice
// sums run on, measured on the device at hand (the roofline's denominators).
//
// The lattice-sum kernel spends its time in two places: the FP64 pipe (sums, weights, the
// complex family's whole integrand) and the integer multiply pipe, which executes the
// truncated 64-bit high products (mulhi_trunc: one 32 x 32 -> 64-bit multiply and two
// 32-bit high multiplies) of the exact lattice points' fixed-point transforms and Genz
// forms.  Each probe runs independent dependency chains of exactly that operation on a
// full-occupancy grid covering every SM, so its rate is what the unit sustains for the
// kernel's own instruction mix.  The paper has no counterpart: this is measurement only.
#include <cuda_runtime.h>

#include <cstdint>

#include "qmc_fixed.cuh"
#include "qmc_gb300.h"
#include "qmc_hostutil.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;    // independent chains per thread (hide the pipe latency)
constexpr int kUnroll = 4;    // iterations per loop trip

__global__ void __launch_bounds__(kProbeThreads) probe_fp64_fma(uint32_t trips, double *sink) {
    double a[kChains];
    const double b = 0.999999999;
    const double c = 1e-9 * (double)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (k + 1) + 1e-7 * (double)blockIdx.x;
#pragma unroll 1
    for (uint32_t i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[0] = s;   // never true; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) probe_int_mulhi(uint32_t trips, double *sink) {
    uint64_t x[kChains];
    const uint64_t y = 0x9e3779b97f4a7c15ull ^ ((uint64_t)threadIdx.x << 7);
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = 0x0123456789abcdefull * (uint64_t)(k + 1) + ((uint64_t)blockIdx.x << 20) + threadIdx.x;
#pragma unroll 1
    for (uint32_t i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = qmc::mulhi_trunc(x[k], y) + x[k];
        }
    }
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= x[k];
    if (s == 0x5a5a5a5a5a5a5a5aull) sink[0] = (double)s;   // practically never; keeps them live
}

}  // namespace

extern "C" int qmc_probe_units(int unit, uint32_t trips, double *sink, double *ops_out,
                               void *stream) {
    using namespace qmc::host;
    if (!sink || !ops_out || trips < 1) return QMC_ERR_ARG;
    if (unit != QMC_PROBE_FP64_FMA && unit != QMC_PROBE_INT_MULHI) return QMC_ERR_ARG;
    int st = device_ok();
    if (st) return st;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QMC_ERR_CUDA;
    const void *fn = unit == QMC_PROBE_FP64_FMA ? (const void *)probe_fp64_fma
                                                : (const void *)probe_int_mulhi;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return QMC_ERR_CUDA;
    const unsigned blocks = (unsigned)(sms * per_sm);
    if (unit == QMC_PROBE_FP64_FMA)
        probe_fp64_fma<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(trips, sink);
    else
        probe_int_mulhi<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(trips, sink);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    // operations: FP64 fused multiply-adds, or 32-bit multiplies (three per high product)
    const double per_step = unit == QMC_PROBE_FP64_FMA ? 1.0 : 3.0;
    *ops_out = (double)blocks * kProbeThreads * (double)trips * kUnroll * kChains * per_step;
    return QMC_OK;
}
