// qmc_batch.cu -- qmc_batch_sums / qmc_batch_autotune: many integrals in one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <cstdint>
#include <cstring>
#include <vector>

#include "qmc_batch.cuh"
#include "qmc_gb300.h"
#include "qmc_hostutil.h"
#include "qmc_internal.h"

using namespace qmc;
using namespace qmc::host;

namespace qmc {

constexpr int kBatchRedThreads = 256;   // as the single-integral reduction: same fold order

// dd helpers (fixed-order double-double folding of the tile partials)
struct dd2 {
    double hi, lo;
};
__device__ __forceinline__ dd2 dd2_add(dd2 a, dd2 b) {
    double s = a.hi + b.hi;
    double bp = s - a.hi;
    double e = (a.hi - (s - bp)) + (b.hi - bp) + a.lo + b.lo;
    double hi = s + e;
    return {hi, e - (hi - s)};
}

// Block (q, component, k): fold item q's tiles for shift k in fixed order.
__global__ void __launch_bounds__(kBatchRedThreads)
    batch_reduce_kernel(const BatchItem *items, int m, int cplx, const double *partials,
                        double *sums) {
    __shared__ dd2 red[kBatchRedThreads];
    const int per_item = m * (cplx ? 2 : 1);
    const int q = blockIdx.x / per_item;
    const int rest = blockIdx.x % per_item;
    const int comp = rest / m, k = rest % m;
    const uint64_t tiles = items[q].tiles;
    const double *base = partials + items[q].partial_off + 2 * (uint64_t)comp * tiles * m;
    dd2 acc = {0.0, 0.0};
    for (uint64_t t = threadIdx.x; t < tiles; t += kBatchRedThreads) {
        const double *pp = base + 2 * (t * (uint64_t)m + k);
        acc = dd2_add(acc, dd2{pp[0], pp[1]});
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kBatchRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = dd2_add(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = sums + (size_t)q * 4 * m + 2 * (size_t)comp * m + 2 * k;
        o[0] = red[0].hi;
        o[1] = red[0].lo;
    }
}

// One thread per item: Qbar and sigma (Eq. (lattice), Eq. (lattice-error)).
__global__ void batch_finalize_kernel(const BatchItem *__restrict__ items, int count, int m, int cplx,
                                      const double *__restrict__ sums, double *__restrict__ results) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const double dn = (double)items[q].n;
    double *res = results + 4 * (size_t)q;
    for (int comp = 0; comp < 2; ++comp) {
        if (comp == 1 && !cplx) {
            res[2] = 0.0;
            res[3] = 0.0;
            break;
        }
        const double *__restrict__ sc = sums + (size_t)q * 4 * m + 2 * (size_t)comp * m;
        double mean = 0.0;
#pragma unroll 8
        for (int k = 0; k < m; ++k) mean += (sc[2 * k] + sc[2 * k + 1]) / dn;
        mean /= (double)m;
        double var = 0.0;
#pragma unroll 8
        for (int k = 0; k < m; ++k) {
            double dq = (sc[2 * k] + sc[2 * k + 1]) / dn - mean;
            var = fma(dq, dq, var);
        }
        var /= (double)m * (double)(m - 1);
        res[2 * comp] = mean;
        res[2 * comp + 1] = sqrt(var);
    }
}

template <int FAM>
cudaError_t launch_batch_fam(const BatchItem *items, const uint64_t *tb, int count, uint64_t tiles,
                             int m, int spb, double *partials, unsigned long long *counters,
                             cudaStream_t s) {
    const uint64_t grid = std::min<uint64_t>(tiles, 0x7FFFFFFFull);
    batch_kernel<FAM><<<(unsigned)grid, spb * m, 0, s>>>(items, tb, count, tiles, m, spb, partials, counters);
    return cudaGetLastError();
}

cudaError_t launch_batch(int family, const BatchItem *items, const uint64_t *tb, int count,
                         uint64_t tiles, int m, int spb, double *partials,
                         unsigned long long *counters, cudaStream_t s) {
    switch (family) {
    case QMC_GENZ_OSCILLATORY: return launch_batch_fam<QMC_GENZ_OSCILLATORY>(items, tb, count, tiles, m, spb, partials, counters, s);
    case QMC_GENZ_PRODUCT_PEAK: return launch_batch_fam<QMC_GENZ_PRODUCT_PEAK>(items, tb, count, tiles, m, spb, partials, counters, s);
    case QMC_GENZ_CORNER_PEAK: return launch_batch_fam<QMC_GENZ_CORNER_PEAK>(items, tb, count, tiles, m, spb, partials, counters, s);
    case QMC_GENZ_GAUSSIAN: return launch_batch_fam<QMC_GENZ_GAUSSIAN>(items, tb, count, tiles, m, spb, partials, counters, s);
    case QMC_SECTOR: return launch_batch_fam<QMC_SECTOR>(items, tb, count, tiles, m, spb, partials, counters, s);
    case QMC_FEYNMAN: return launch_batch_fam<QMC_FEYNMAN>(items, tb, count, tiles, m, spb, partials, counters, s);
    default: return cudaErrorInvalidValue;
    }
}

bool batch_family_supported(int fam) {
    return fam == QMC_GENZ_OSCILLATORY || fam == QMC_GENZ_PRODUCT_PEAK || fam == QMC_GENZ_CORNER_PEAK ||
           fam == QMC_GENZ_GAUSSIAN || fam == QMC_SECTOR || fam == QMC_FEYNMAN;
}

cudaError_t launch_batch_reduce(const BatchItem *d_items, int count, int m, int cplx,
                                const double *partials, double *sums, cudaStream_t s) {
    const uint64_t blocks = (uint64_t)count * m * (cplx ? 2 : 1);
    batch_reduce_kernel<<<(unsigned)blocks, kBatchRedThreads, 0, s>>>(d_items, m, cplx, partials, sums);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchItem *d_items, int count, int m, int cplx,
                                  const double *sums, double *results, cudaStream_t s) {
    batch_finalize_kernel<<<(count + 127) / 128, 128, 0, s>>>(d_items, count, m, cplx, sums, results);
    return cudaGetLastError();
}

int fill_batch_item(BatchItem &it, const qmc_batch_item &b, int m, int spb, uint32_t Lcfg, int fam) {
    int st = check_integrand_shape(&b.f);
    if (st) return st;
    if ((st = check_rule(&b.rule))) return st;
    if (b.f.family != fam || (int)b.rule.m != m) return QMC_ERR_ARG;
    if (b.f.dim != b.rule.dim) return QMC_ERR_DIM;
    if (b.i_end <= b.i_begin || b.i_end > b.rule.n) return QMC_ERR_RANGE;
    const uint64_t range = b.i_end - b.i_begin;
    uint32_t L = Lcfg;
    if (L == 0) {
        Geometry g = geometry(range, m);
        L = (g.spb == spb) ? g.L : points_per_stream(range, (uint64_t)spb);
    }
    const uint64_t ptile = (uint64_t)spb * L;
    std::memset(&it, 0, sizeof(it));
    it.n = b.rule.n;
    it.i_begin = b.i_begin;
    it.i_end = b.i_end;
    it.tiles = (range + ptile - 1) / ptile;
    it.L = L;
    it.d = b.rule.dim;
    for (int j = 0; j < it.d; ++j) it.dc[j] = dim_const(b.rule.z[j] % b.rule.n, b.rule.n);
    it.shifts = b.rule.shifts;
    it.t = make_transform(b.rule.transform);
    it.cd = korobov_cd(b.rule.transform, it.t, it.d);
    it.fit = b.rule.fit;
    it.family = fam;
    it.c = b.f.c;
    it.w = b.f.w;
    it.h = b.f.h;
    it.nu = b.f.nu;
    it.nf = b.f.nf;
    it.ucoef = b.f.ucoef;
    it.fcoef = b.f.fcoef;
    it.uexp = b.f.uexp;
    it.fexp = b.f.fexp;
    it.pa = b.f.pa;
    it.pb = b.f.pb;
    it.lam = b.f.lambda;
    return QMC_OK;
}

}  // namespace qmc

namespace {

struct BatchPlan {
    std::vector<BatchItem> items;
    std::vector<uint64_t> tile_begin;   // count + 1
    uint64_t total_tiles = 0;
    uint64_t partial_doubles = 0;
    int m = 0, spb = 0, family = 0, cplx = 0;
    size_t off_items = 0, off_tb = 0, off_partials = 0, bytes = 0;
};

// Validates the batch and lays out descriptors, tile prefix sums and partials.
int plan_batch(const qmc_batch_item *in, int count, const qmc_batch_config *cfg, BatchPlan &P) {
    if (!in || count < 1) return QMC_ERR_ARG;
    const int m = (int)in[0].rule.m;
    const int fam = in[0].f.family;
    if (m < 1 || m > kMaxShiftGroup) return QMC_ERR_M;
    if (!batch_family_supported(fam)) return QMC_ERR_INTEGRAND;
    int spb = (cfg && cfg->streams_per_block > 0) ? cfg->streams_per_block : std::max(1, kSumsThreads / m);
    if (spb * m > kSumsThreads) return QMC_ERR_ARG;
    const uint32_t Lcfg = cfg ? cfg->points_per_stream : 0;
    P.m = m;
    P.spb = spb;
    P.family = fam;
    P.cplx = is_complex_family(fam);
    P.items.resize(count);
    P.tile_begin.resize(count + 1);
    uint64_t tiles = 0, poff = 0;
    for (int q = 0; q < count; ++q) {
        BatchItem &it = P.items[q];
        int st = fill_batch_item(it, in[q], m, spb, Lcfg, fam);
        if (st) return st;
        it.tile_begin = tiles;
        it.partial_off = poff;
        P.tile_begin[q] = tiles;
        tiles += it.tiles;
        poff += it.tiles * (uint64_t)m * 2 * (P.cplx ? 2 : 1);
    }
    P.tile_begin[count] = tiles;
    P.total_tiles = tiles;
    P.partial_doubles = poff;
    size_t o = 0;
    P.off_items = o;
    o += align256(sizeof(BatchItem) * count);
    P.off_tb = o;
    o += align256(sizeof(uint64_t) * (count + 1));
    P.off_partials = o;
    o += align256(sizeof(double) * poff);
    P.bytes = o;
    return QMC_OK;
}

// Kernels only (descriptors already in the workspace): capturable in a CUDA graph.
int launch_planned(const BatchPlan &P, int count, void *workspace, double *sums, double *results,
                   unsigned long long *counters, cudaStream_t s) {
    char *ws = (char *)workspace;
    BatchItem *d_items = (BatchItem *)(ws + P.off_items);
    uint64_t *d_tb = (uint64_t *)(ws + P.off_tb);
    double *d_part = (double *)(ws + P.off_partials);
    if (launch_batch(P.family, d_items, d_tb, count, P.total_tiles, P.m, P.spb, d_part, counters, s) != cudaSuccess)
        return QMC_ERR_CUDA;
    if (launch_batch_reduce(d_items, count, P.m, P.cplx, d_part, sums, s) != cudaSuccess) return QMC_ERR_CUDA;
    if (results) {
        if (P.m < 2) return QMC_ERR_M;
        if (launch_batch_finalize(d_items, count, P.m, P.cplx, sums, results, s) != cudaSuccess)
            return QMC_ERR_CUDA;
    }
    return QMC_OK;
}

int run_batch(const BatchPlan &P, int count, void *workspace, double *sums, double *results,
              unsigned long long *counters, cudaStream_t s) {
    char *ws = (char *)workspace;
    if (cudaMemcpyAsync(ws + P.off_items, P.items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + P.off_tb, P.tile_begin.data(), sizeof(uint64_t) * (count + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return QMC_ERR_CUDA;
    return launch_planned(P, count, workspace, sums, results, counters, s);
}

}  // namespace

struct qmc_batch_plan {
    BatchPlan P;
    int count;
    void *workspace;
};

extern "C" int qmc_batch_plan_create(const qmc_batch_item *items, int count,
                                     const qmc_batch_config *cfg, void *workspace,
                                     size_t workspace_bytes, void *stream, qmc_batch_plan **out) {
    if (!workspace || !out) return QMC_ERR_ARG;
    qmc_batch_plan *plan = new (std::nothrow) qmc_batch_plan;
    if (!plan) return QMC_ERR_ARG;
    int st = plan_batch(items, count, cfg, plan->P);
    if (!st && workspace_bytes < plan->P.bytes) st = QMC_ERR_WORKSPACE;
    if (!st) st = device_ok();
    if (!st) {
        cudaStream_t s = (cudaStream_t)stream;
        char *ws = (char *)workspace;
        if (cudaMemcpyAsync(ws + plan->P.off_items, plan->P.items.data(), sizeof(BatchItem) * count,
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(ws + plan->P.off_tb, plan->P.tile_begin.data(),
                            sizeof(uint64_t) * (count + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = QMC_ERR_CUDA;
    }
    if (st) {
        delete plan;
        return st;
    }
    plan->count = count;
    plan->workspace = workspace;
    *out = plan;
    return QMC_OK;
}

extern "C" int qmc_batch_plan_run(const qmc_batch_plan *plan, double *sums, double *results,
                                  unsigned long long *counters, void *stream) {
    if (!plan || !sums) return QMC_ERR_ARG;
    return launch_planned(plan->P, plan->count, plan->workspace, sums, results, counters,
                          (cudaStream_t)stream);
}

extern "C" void qmc_batch_plan_destroy(qmc_batch_plan *plan) { delete plan; }

extern "C" size_t qmc_batch_workspace_bytes(const qmc_batch_item *items, int count,
                                            const qmc_batch_config *cfg) {
    BatchPlan P;
    if (plan_batch(items, count, cfg, P) != QMC_OK) return 0;
    return P.bytes;
}

extern "C" int qmc_batch_sums(const qmc_batch_item *items, int count, const qmc_batch_config *cfg,
                              void *workspace, size_t workspace_bytes, double *sums,
                              double *results, unsigned long long *counters, void *stream) {
    if (!workspace || !sums) return QMC_ERR_ARG;
    BatchPlan P;
    int st = plan_batch(items, count, cfg, P);
    if (st) return st;
    if (workspace_bytes < P.bytes) return QMC_ERR_WORKSPACE;
    if ((st = device_ok())) return st;
    return run_batch(P, count, workspace, sums, results, counters, (cudaStream_t)stream);
}

extern "C" int qmc_batch_autotune(const qmc_batch_item *items, int count, void *workspace,
                                  size_t workspace_bytes, double *sums, void *stream,
                                  qmc_batch_config *best) {
    if (!workspace || !sums || !best || !items || count < 1) return QMC_ERR_ARG;
    int st = device_ok();
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // a sample of the batch: every step-th item, at most 256 items
    const int step = std::max(1, count / 256);
    std::vector<qmc_batch_item> sample;
    for (int q = 0; q < count; q += step) sample.push_back(items[q]);
    // bounded cost per candidate: at most ~2^23 points in all, each item's range cut to its
    // share from its start (the candidates are compared on the same work)
    const uint64_t share = std::max<uint64_t>(1u << 16, (1u << 23) / sample.size());
    for (auto &it : sample)
        if (it.i_end > it.i_begin + share) it.i_end = it.i_begin + share;
    const int m = (int)items[0].rule.m;
    if (m < 1 || m > kMaxShiftGroup) return QMC_ERR_M;
    const int spb_max = std::max(1, kSumsThreads / m);
    const int spbs[] = {spb_max, std::max(1, spb_max / 2), std::max(1, spb_max / 4)};
    const uint32_t Ls[] = {16, 32, 64, 128, 256, 512};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QMC_ERR_CUDA;
    float best_ms = -1.0f;
    qmc_batch_config cand;
    for (int si = 0; si < 3; ++si) {
        if (si > 0 && spbs[si] == spbs[si - 1]) continue;
        for (uint32_t L : Ls) {
            cand.streams_per_block = spbs[si];
            cand.points_per_stream = L;
            BatchPlan P;
            if ((st = plan_batch(sample.data(), (int)sample.size(), &cand, P))) break;
            if (P.bytes > workspace_bytes) continue;
            // warm once, then time one run
            if ((st = run_batch(P, (int)sample.size(), workspace, sums, nullptr, nullptr, s))) break;
            cudaEventRecord(e0, s);
            if ((st = run_batch(P, (int)sample.size(), workspace, sums, nullptr, nullptr, s))) break;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = QMC_ERR_CUDA; break; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                *best = cand;
            }
        }
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    return best_ms < 0.0f ? QMC_ERR_WORKSPACE : QMC_OK;
}
