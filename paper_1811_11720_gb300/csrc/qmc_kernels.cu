// qmc_kernels.cu -- lattice points, fixed-order reductions, evaluate() and the fit
// histogram.
#include <cuda_runtime.h>

#include <cstdint>

#include "qmc_integrands.cuh"
#include "qmc_internal.h"
#include "qmc_lattice.cuh"
#include "qmc_transforms.cuh"

namespace qmc {

// ---- lattice points (Eq. (lattice), Fig. 1) --------------------------------------------
// Thread t owns points [i_begin + t L, i_begin + (t+1) L): state from the closed form at
// the chunk start, then lattice_step, exactly as in the sums kernel.
__global__ void __launch_bounds__(128) points_kernel(const PointsParams p) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t off = t * p.L;
    if (off >= p.count) return;
    const uint64_t cnt = (p.count - off < p.L) ? p.count - off : p.L;
    const uint64_t i0 = p.i_begin + off;
    const int d = p.d, m = p.m;
    uint64_t fhi[kMaxDim], flo[kMaxDim], rem[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j)
        if (j < d) lattice_state_at(i0, p.dc[j], p.n, fhi[j], flo[j], rem[j]);
    for (uint64_t q = 0; q < cnt; ++q) {
        double *o = p.out + (off + q) * (uint64_t)m * d;
        for (int k = 0; k < m; ++k) {
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j)
                if (j < d)
                    o[(size_t)k * d + j] = fixed_to_double(fhi[j] + (p.shifts[(size_t)k * d + j] << 11),
                                                           flo[j], rem[j], p.n);
        }
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j)
            if (j < d) lattice_step(p.dc[j], p.n, fhi[j], flo[j], rem[j]);
    }
}

cudaError_t launch_points(const PointsParams &p, cudaStream_t s) {
    uint64_t threads = (p.count + p.L - 1) / p.L;
    uint32_t blocks = (uint32_t)((threads + 127) / 128);
    if (blocks == 0) return cudaSuccess;
    points_kernel<<<blocks, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ---- fixed-order double-double reductions ----------------------------------------------
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bp = s - a;
    double e = (a - (s - bp)) + (b - bp);
    return {s, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    double e = s.lo + a.lo + b.lo;
    double hi = s.hi + e;
    double lo = e - (hi - s.hi);
    return {hi, lo};
}

constexpr int kRedThreads = 256;

// One block per (shift, component): thread t folds tiles t, t+256, ... in order, then a
// fixed binary tree over the block.
__global__ void __launch_bounds__(kRedThreads) reduce_tiles_kernel(const double *partials,
                                                                   uint64_t tiles, int m,
                                                                   double *sums) {
    __shared__ dd red[kRedThreads];
    const int col = blockIdx.x;           // k + m * component
    const int comp = col / m, k = col % m;
    const double *base = partials + 2 * (uint64_t)comp * tiles * m;
    dd acc = {0.0, 0.0};
    for (uint64_t t = threadIdx.x; t < tiles; t += kRedThreads) {
        const double *pp = base + 2 * (t * (uint64_t)m + k);
        acc = dd_add(acc, dd{pp[0], pp[1]});
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = dd_add(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = sums + 2 * (uint64_t)comp * m + 2 * k;
        o[0] = red[0].hi;
        o[1] = red[0].lo;
    }
}

cudaError_t launch_reduce_tiles(const double *partials, uint64_t tiles, int m, int is_complex,
                                double *sums, cudaStream_t s) {
    reduce_tiles_kernel<<<m * (is_complex ? 2 : 1), kRedThreads, 0, s>>>(partials, tiles, m, sums);
    return cudaGetLastError();
}

// Eq. (lattice) and Eq. (lattice-error): Q_k = S_k / n, Qbar, sigma, per component.
// The m divisions run in parallel (one thread per shift and component); the mean and the
// variance are then summed by one thread per component in fixed order k = 0..m-1, the
// order the batched form uses, so both give the same bits.
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads)
    finalize_kernel(const double *__restrict__ sums, int m, uint64_t n, int is_complex,
                    double *__restrict__ result, double *__restrict__ Q) {
    __shared__ double q_s[2 * QMC_MAX_SHIFTS];
    const double dn = (double)n;
    const int ncomp = is_complex ? 2 : 1;
    for (int i = threadIdx.x; i < ncomp * m; i += blockDim.x) {
        const int comp = i / m, k = i - comp * m;
        const double *sc = sums + 2 * (size_t)comp * m;
        const double q = (sc[2 * k] + sc[2 * k + 1]) / dn;
        q_s[i] = q;
        if (Q) Q[i] = q;
    }
    __syncthreads();
    const int comp = threadIdx.x;
    if (comp >= ncomp) return;
    const double *qc = q_s + (size_t)comp * m;
    double mean = 0.0;
#pragma unroll 8
    for (int k = 0; k < m; ++k) mean += qc[k];
    mean /= (double)m;
    double var = 0.0;
#pragma unroll 8
    for (int k = 0; k < m; ++k) {
        const double dq = qc[k] - mean;
        var = fma(dq, dq, var);
    }
    var /= (double)m * (double)(m - 1);
    result[2 * comp] = mean;
    result[2 * comp + 1] = sqrt(var);
    if (!is_complex) {
        result[2] = 0.0;
        result[3] = 0.0;
    }
}

cudaError_t launch_finalize(const double *sums, int m, uint64_t n, int is_complex,
                            double *result, double *Q, cudaStream_t s) {
    const int work = m * (is_complex ? 2 : 1);
    const int threads = work >= kFinThreads ? kFinThreads : ((work + 31) / 32) * 32;
    finalize_kernel<<<1, threads, 0, s>>>(sums, m, n, is_complex, result, Q);
    return cudaGetLastError();
}

// ---- evaluate(): raw f on one shifted lattice, no transform ---------------------------
template <int FAM>
__device__ __forceinline__ void eval_point(const FamilyShared &fsh, const double *x, int d,
                                           double &re, double &im, unsigned long long &sf) {
    FamilyAcc<FAM> fa;
    fa.init(fsh);
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j)
        if (j < d) fa.add(j, Mapped{x[j], false}, fsh);
    fa.finish(d, fsh, re, im, sf);
}

constexpr int kEvalThreads = 128;
constexpr uint32_t kEvalChunk = 32;

template <int FAM>
__global__ void __launch_bounds__(kEvalThreads) evaluate_kernel(const SumsParams p, double *out) {
    __shared__ FamilyShared fsh;
    stage_family<FAM>(p, fsh);
    __syncthreads();
    const int d = p.d;
    const uint64_t count = p.i_end - p.i_begin;
    uint64_t dsh[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) dsh[j] = (j < d) ? (p.shifts[j] << 11) : 0ull;
    for (uint64_t off = ((uint64_t)blockIdx.x * kEvalThreads + threadIdx.x) * kEvalChunk; off < count;
         off += (uint64_t)gridDim.x * kEvalThreads * kEvalChunk) {
        const uint64_t cnt = (count - off < kEvalChunk) ? count - off : kEvalChunk;
        uint64_t fhi[kMaxDim], flo[kMaxDim], rem[kMaxDim];
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j)
            if (j < d) lattice_state_at(p.i_begin + off, p.dc[j], p.n, fhi[j], flo[j], rem[j]);
        for (uint64_t q = 0; q < cnt; ++q) {
            double x[kMaxDim];
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j) {
                x[j] = 0.0;
                if (j < d) {
                    x[j] = fixed_to_double(fhi[j] + dsh[j], flo[j], rem[j], p.n);
                    lattice_step(p.dc[j], p.n, fhi[j], flo[j], rem[j]);
                }
            }
            double re, im;
            unsigned long long sf = 0;
            eval_point<FAM>(fsh, x, d, re, im, sf);
            if constexpr (FamilyAcc<FAM>::kComplex) {
                out[2 * (off + q)] = re;
                out[2 * (off + q) + 1] = im;
            } else {
                out[off + q] = re;
            }
        }
    }
}

// ---- histogram of |f| per dimension (fit data pass, Sec. 2.4) --------------------------
// Each block walks batches of kEvalThreads points; threads evaluate their point, then
// threads j < d add the batch to dimension j's block histogram in point order
// (deterministic).  Block histograms go to work[block][d][bins] and are summed over
// blocks in block order by hist_sum_kernel.
template <int FAM>
__global__ void __launch_bounds__(kEvalThreads) histogram_kernel(const SumsParams p, int bins,
                                                                 double *work) {
    extern __shared__ double hsm[];   // [d][bins]
    __shared__ FamilyShared fsh;
    __shared__ double val[kEvalThreads];
    __shared__ uint16_t bin[kEvalThreads][kMaxDim];
    stage_family<FAM>(p, fsh);
    const int d = p.d;
    for (int q = threadIdx.x; q < d * bins; q += kEvalThreads) hsm[q] = 0.0;
    __syncthreads();
    uint64_t dsh[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) dsh[j] = (j < d) ? (p.shifts[j] << 11) : 0ull;
    const uint64_t n = p.n;
    const uint64_t per_block = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * per_block;
    const uint64_t b1 = (b0 + per_block < n) ? b0 + per_block : n;
    for (uint64_t base = b0; base < b1; base += kEvalThreads) {
        const uint64_t i = base + threadIdx.x;
        double v = 0.0;
        if (i < b1) {
            double x[kMaxDim];
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j) {
                x[j] = 0.0;
                if (j < d) {
                    uint64_t fh, fl, rm;
                    lattice_state_at(i, p.dc[j], n, fh, fl, rm);
                    x[j] = fixed_to_double(fh + dsh[j], fl, rm, n);
                    int b = (int)floor(x[j] * (double)bins);
                    bin[threadIdx.x][j] = (uint16_t)(b >= bins ? bins - 1 : b);
                }
            }
            double re, im;
            unsigned long long sf = 0;
            eval_point<FAM>(fsh, x, d, re, im, sf);
            v = FamilyAcc<FAM>::kComplex ? hypot(re, im) : fabs(re);
        }
        val[threadIdx.x] = v;
        __syncthreads();
        if ((int)threadIdx.x < d) {
            const int j = threadIdx.x;
            const uint64_t lim = (b1 - base < kEvalThreads) ? b1 - base : kEvalThreads;
            for (uint64_t q = 0; q < lim; ++q) hsm[j * bins + bin[q][j]] += val[q];
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < d * bins; q += kEvalThreads)
        work[(size_t)blockIdx.x * d * bins + q] = hsm[q];
}

__global__ void hist_sum_kernel(const double *work, uint32_t nblocks, int cells, double *hist) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cells) return;
    double s = 0.0, c = 0.0;
    for (uint32_t b = 0; b < nblocks; ++b) {
        double v = work[(size_t)b * cells + q];
        double t = s + v;
        c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    hist[q] = s + c;
}

template <int FAM>
static cudaError_t eval_dispatch_one(const SumsParams &p, double *out, cudaStream_t s) {
    uint64_t count = p.i_end - p.i_begin;
    uint64_t chunks = (count + kEvalChunk - 1) / kEvalChunk;
    uint32_t blocks = (uint32_t)((chunks + kEvalThreads - 1) / kEvalThreads);
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    if (blocks == 0) return cudaSuccess;
    evaluate_kernel<FAM><<<blocks, kEvalThreads, 0, s>>>(p, out);
    return cudaGetLastError();
}

template <int FAM>
static cudaError_t hist_dispatch_one(const SumsParams &p, int bins, double *hist, double *work,
                                     uint32_t nblocks, cudaStream_t s) {
    size_t smem = (size_t)p.d * bins * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(histogram_kernel<FAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    histogram_kernel<FAM><<<nblocks, kEvalThreads, smem, s>>>(p, bins, work);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int cells = p.d * bins;
    hist_sum_kernel<<<(cells + 255) / 256, 256, 0, s>>>(work, nblocks, cells, hist);
    return cudaGetLastError();
}

#define QMC_FAMILY_SWITCH(FN, ...)                                                      \
    switch (p.family) {                                                                 \
    case QMC_GENZ_OSCILLATORY: return FN<QMC_GENZ_OSCILLATORY>(__VA_ARGS__);            \
    case QMC_GENZ_PRODUCT_PEAK: return FN<QMC_GENZ_PRODUCT_PEAK>(__VA_ARGS__);          \
    case QMC_GENZ_CORNER_PEAK: return FN<QMC_GENZ_CORNER_PEAK>(__VA_ARGS__);            \
    case QMC_GENZ_GAUSSIAN: return FN<QMC_GENZ_GAUSSIAN>(__VA_ARGS__);                  \
    case QMC_GENZ_C0: return FN<QMC_GENZ_C0>(__VA_ARGS__);                              \
    case QMC_GENZ_DISCONTINUOUS: return FN<QMC_GENZ_DISCONTINUOUS>(__VA_ARGS__);        \
    case QMC_MONOMIAL: return FN<QMC_MONOMIAL>(__VA_ARGS__);                            \
    case QMC_TRIG: return FN<QMC_TRIG>(__VA_ARGS__);                                    \
    case QMC_SECTOR: return FN<QMC_SECTOR>(__VA_ARGS__);                                \
    case QMC_FEYNMAN: return FN<QMC_FEYNMAN>(__VA_ARGS__);                              \
    default: return cudaErrorInvalidValue;                                              \
    }

cudaError_t launch_evaluate(const SumsParams &p, double *out, cudaStream_t s) {
    QMC_FAMILY_SWITCH(eval_dispatch_one, p, out, s)
}

cudaError_t launch_histogram(const SumsParams &p, int bins, double *hist, double *work,
                             uint32_t nblocks, cudaStream_t s) {
    QMC_FAMILY_SWITCH(hist_dispatch_one, p, bins, hist, work, nblocks, s)
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

}  // namespace qmc
