// qmc_noalloc.cu -- qmc_sums_noalloc(): per-shift lattice sums without any allocation.
//
// Some callers cannot allocate device memory at the time they integrate: code running
// inside a CUDA-graph capture, a real-time or signal-safe path, a host process whose
// allocator is owned by another runtime (a framework's caching allocator that must not be
// bypassed), or an embedded user that has budgeted all device memory up front.  For them
// this entry point takes the same inputs and outputs as qmc_sums() but no workspace: the
// per-tile partial sums go to a fixed device array that is part of the library image.
//
// The array is QMC_NOALLOC_SCRATCH_BYTES (8 MiB) per device, held by every GPU that loads
// the library until the process exits.  All calls on a device share it and it keeps the last
// call's contents; the lattice-sum kernel overwrites every partial it later reads, so
// nothing in it has to start at zero.  Calls that overlap on the GPU (different streams,
// or host threads, without ordering between them) race on the array.
//
// The array's device address is looked up once per device and kept for the life of the
// process; cudaDeviceReset() unloads the library's device image, so after a reset that
// address is stale and this entry point must not be called again in the same process.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "qmc_gb300.h"
#include "qmc_hostutil.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QMC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  The array's name is only a
// host-side handle; the address has to come from the runtime, once per device, with that
// device current.
int noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMC_ERR_NO_DEVICE;
    if (dev < 0 || dev >= kMaxDevices) return QMC_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return QMC_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return QMC_OK;
}

}  // namespace

extern "C" int qmc_sums_noalloc(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin,
                                uint64_t i_end, double *sums, unsigned long long *counters,
                                void *stream) {
    using namespace qmc::host;
    // the checks of qmc_sums, in its order, so that both entry points report the same code
    int st = check_integrand_shape(f);
    if (st) return st;
    if ((st = check_rule(rule))) return st;
    if (f->dim != rule->dim) return QMC_ERR_DIM;
    if (!sums) return QMC_ERR_ARG;
    if (i_end <= i_begin || i_end > rule->n) return QMC_ERR_RANGE;
    if ((st = device_ok())) return st;
    const size_t need = qmc_sums_workspace_bytes(rule, is_complex_family(f->family), i_begin, i_end);
    if (need == 0) return QMC_ERR_ARG;
    if (need > (size_t)QMC_NOALLOC_SCRATCH_BYTES) return QMC_ERR_WORKSPACE;
    void *scratch = nullptr;
    if ((st = noalloc_scratch(&scratch))) return st;
    return qmc_sums(f, rule, i_begin, i_end, scratch, (size_t)QMC_NOALLOC_SCRATCH_BYTES, sums,
                    counters, stream);
}
