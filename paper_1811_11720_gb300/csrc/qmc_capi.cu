// qmc_capi.cu -- the C ABI declared in include/qmc_gb300.h.
//
// Host responsibilities: argument validation, lattice constants (Fz, remz) in exact
// 128-bit host arithmetic, SplitMix64 shifts, Korobov/Sidi coefficient tables, the tile
// geometry, kernel dispatch, and the host-buffer integrate() with its adaptive loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "qmc_gb300.h"
#include "qmc_hostutil.h"
#include "qmc_internal.h"

using namespace qmc;

namespace {

using namespace qmc::host;

uint64_t splitmix64_output(uint64_t seed, uint64_t t) {
    // SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden-ratio increment,
    // the output is the state passed through the published finaliser.
    uint64_t x = seed + (t + 1) * 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

}  // namespace

// ======================================================================================
extern "C" {

const char *qmc_strerror(int code) {
    switch (code) {
    case QMC_OK: return "ok";
    case QMC_ERR_ARG: return "invalid argument";
    case QMC_ERR_DIM: return "dimension out of range";
    case QMC_ERR_N: return "lattice size out of range or not in the table";
    case QMC_ERR_GENVEC: return "generating vector component not coprime to n";
    case QMC_ERR_M: return "number of shifts out of range (m >= 2 needed for an error)";
    case QMC_ERR_FIT_PARAMS: return "PolySingular parameters violate a0 >= 1.001, a1 <= -0.001";
    case QMC_ERR_INTEGRAND: return "unknown integrand family or bad coefficient arrays";
    case QMC_ERR_TRANSFORM: return "unknown transform or order out of range";
    case QMC_ERR_CUDA: return "CUDA runtime error";
    case QMC_ERR_WORKSPACE: return "workspace too small";
    case QMC_ERR_NONFINITE: return "integrand produced NaN or Inf";
    case QMC_ERR_RANGE: return "index range or bin count out of range";
    case QMC_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    default: return "unknown error";
    }
}

int qmc_abi_version(void) { return QMC_ABI_VERSION; }

int qmc_get_next_n(const qmc_genvec_table *t, uint64_t preferred, uint64_t *n_out) {
    if (!t || !t->n || !n_out || t->count < 1) return QMC_ERR_ARG;
    for (int c = 0; c < t->count; ++c)
        if (t->n[c] >= preferred) {
            *n_out = t->n[c];
            return QMC_OK;
        }
    return QMC_ERR_N;
}

int qmc_make_shifts(uint64_t seed, uint64_t m, int dim, uint64_t *D_out) {
    if (!D_out) return QMC_ERR_ARG;
    if (dim < 1 || dim > QMC_MAX_DIM) return QMC_ERR_DIM;
    if (m < 1 || m > QMC_MAX_SHIFTS) return QMC_ERR_M;
    for (uint64_t k = 0; k < m; ++k)
        for (int j = 0; j < dim; ++j)
            D_out[k * dim + j] = splitmix64_output(seed, k * (uint64_t)dim + j) >> 11;
    return QMC_OK;
}

int qmc_points(const qmc_rule *rule, uint64_t i_begin, uint64_t count, double *out, void *stream) {
    int st = check_rule(rule);
    if (st) return st;
    if (!out) return QMC_ERR_ARG;
    if (i_begin > rule->n || count > rule->n - i_begin) return QMC_ERR_RANGE;
    if ((st = device_ok())) return st;
    PointsParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = rule->n;
    p.i_begin = i_begin;
    p.count = count;
    p.d = rule->dim;
    p.m = (int)rule->m;
    p.L = 64;
    for (int j = 0; j < rule->dim; ++j) p.dc[j] = dim_const(rule->z[j] % rule->n, rule->n);
    p.shifts = rule->shifts;
    p.out = out;
    return cuda_status(launch_points(p, (cudaStream_t)stream));
}

size_t qmc_sums_workspace_bytes(const qmc_rule *rule, int is_complex, uint64_t i_begin,
                                uint64_t i_end) {
    if (!rule || i_end <= i_begin || rule->m < 1) return 0;
    size_t total = 0;
    for (uint64_t k0 = 0; k0 < rule->m; k0 += kMaxShiftGroup) {
        int mg = (int)std::min<uint64_t>(kMaxShiftGroup, rule->m - k0);
        Geometry g = geometry(i_end - i_begin, mg);
        total += align256(g.tiles * (uint64_t)mg * 2 * sizeof(double) * (is_complex ? 2 : 1));
    }
    return total;
}

int qmc_sums(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin, uint64_t i_end,
             void *workspace, size_t workspace_bytes, double *sums, unsigned long long *counters,
             void *stream) {
    int st = check_integrand_shape(f);
    if (st) return st;
    if ((st = check_rule(rule))) return st;
    if (f->dim != rule->dim) return QMC_ERR_DIM;
    if (!sums || !workspace) return QMC_ERR_ARG;
    if (i_end <= i_begin || i_end > rule->n) return QMC_ERR_RANGE;
    const int cplx = is_complex_family(f->family);
    if (workspace_bytes < qmc_sums_workspace_bytes(rule, cplx, i_begin, i_end)) return QMC_ERR_WORKSPACE;
    if ((st = device_ok())) return st;
    cudaStream_t s = (cudaStream_t)stream;

    SumsParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = rule->n;
    p.i_begin = i_begin;
    p.i_end = i_end;
    p.d = rule->dim;
    for (int j = 0; j < rule->dim; ++j) p.dc[j] = dim_const(rule->z[j] % rule->n, rule->n);
    p.t = make_transform(rule->transform);
    p.cd = korobov_cd(rule->transform, p.t, rule->dim);
    p.fit = rule->fit;
    fill_integrand(p, f);
    p.counters = counters;

    char *ws = (char *)workspace;
    const uint64_t m = rule->m;
    for (uint64_t k0 = 0; k0 < m; k0 += kMaxShiftGroup) {
        const int mg = (int)std::min<uint64_t>(kMaxShiftGroup, m - k0);
        Geometry g = geometry(i_end - i_begin, mg);
        p.m = mg;
        p.spb = g.spb;
        p.L = g.L;
        p.tiles = g.tiles;
        p.shifts = rule->shifts + k0 * rule->dim;
        p.partials = (double *)ws;
        cudaError_t e = launch_sums_any(f->family, p.t.kind, dim3((unsigned)g.tiles),
                                        dim3(g.threads), s, p);
        if (e != cudaSuccess) return QMC_ERR_CUDA;
        // sums layout: re pairs for all m, then im pairs for all m; group k0 writes its slice
        double *grp = sums + 2 * k0;
        if (!cplx) {
            e = launch_reduce_tiles(p.partials, g.tiles, mg, 0, grp, s);
        } else {
            // the reduce kernel writes [re (2 mg)] [im (2 mg)] contiguously; reduce each
            // component separately so that im lands at sums + 2m + 2 k0
            e = launch_reduce_tiles(p.partials, g.tiles, mg, 0, grp, s);
            if (e == cudaSuccess)
                e = launch_reduce_tiles(p.partials + 2 * g.tiles * (uint64_t)mg, g.tiles, mg, 0,
                                        sums + 2 * m + 2 * k0, s);
        }
        if (e != cudaSuccess) return QMC_ERR_CUDA;
        ws += align256(g.tiles * (uint64_t)mg * 2 * sizeof(double) * (cplx ? 2 : 1));
    }
    return QMC_OK;
}

int qmc_sums_tile_count(uint64_t range_len, uint64_t m, uint64_t *tiles,
                        uint64_t *points_per_tile) {
    if (!tiles || !points_per_tile) return QMC_ERR_ARG;
    if (m < 1 || m > (uint64_t)kMaxShiftGroup) return QMC_ERR_M;
    const Geometry g = geometry(range_len, (int)m);
    *tiles = g.tiles;
    *points_per_tile = (uint64_t)g.spb * g.L;
    return QMC_OK;
}

int qmc_sums_tiles(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin,
                   uint64_t i_end, uint64_t tile_begin, uint64_t tile_end, double *partials,
                   unsigned long long *counters, void *stream) {
    int st = check_integrand_shape(f);
    if (st) return st;
    if ((st = check_rule(rule))) return st;
    if (f->dim != rule->dim) return QMC_ERR_DIM;
    if (!partials) return QMC_ERR_ARG;
    if (rule->m > (uint64_t)kMaxShiftGroup) return QMC_ERR_M;
    if (i_end <= i_begin || i_end > rule->n) return QMC_ERR_RANGE;
    const int mg = (int)rule->m;
    const Geometry g = geometry(i_end - i_begin, mg);
    if (tile_begin >= tile_end || tile_end > g.tiles) return QMC_ERR_RANGE;
    if ((st = device_ok())) return st;

    // the tiles of the whole range's decomposition: same L and streams per block, the
    // first point moved to tile_begin, the global end kept for the ragged last tile
    SumsParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = rule->n;
    p.i_begin = i_begin + tile_begin * (uint64_t)g.spb * g.L;
    p.i_end = i_end;
    p.d = rule->dim;
    for (int j = 0; j < rule->dim; ++j) p.dc[j] = dim_const(rule->z[j] % rule->n, rule->n);
    p.t = make_transform(rule->transform);
    p.cd = korobov_cd(rule->transform, p.t, rule->dim);
    p.fit = rule->fit;
    fill_integrand(p, f);
    p.counters = counters;
    p.m = mg;
    p.spb = g.spb;
    p.L = g.L;
    p.tiles = tile_end - tile_begin;
    p.shifts = rule->shifts;
    p.partials = partials;
    cudaError_t e = launch_sums_any(f->family, p.t.kind, dim3((unsigned)p.tiles), dim3(g.threads),
                                    (cudaStream_t)stream, p);
    return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int qmc_reduce_tiles(const double *partials, uint64_t tiles, uint64_t m, int is_complex,
                     double *sums, void *stream) {
    if (!partials || !sums || tiles < 1) return QMC_ERR_ARG;
    if (m < 1 || m > (uint64_t)kMaxShiftGroup) return QMC_ERR_M;
    int st = device_ok();
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_reduce_tiles(partials, tiles, (int)m, 0, sums, s);
    if (e == cudaSuccess && is_complex)
        e = launch_reduce_tiles(partials + 2 * tiles * m, tiles, (int)m, 0, sums + 2 * m, s);
    return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

int qmc_merge_sums(const double *parts, uint64_t nparts, uint64_t len, double *out) {
    if (!parts || !out || nparts < 1 || len < 2 || (len & 1)) return QMC_ERR_ARG;
    // (hi, lo) += (a_hi, a_lo) per slot: TwoSum of the high words, the low words added to its
    // error, renormalised with Fast2Sum; parts are taken in their order (deterministic)
    for (uint64_t k = 0; k < len; k += 2) {
        double hi = parts[k], lo = parts[k + 1];
        for (uint64_t p = 1; p < nparts; ++p) {
            const double a_hi = parts[p * len + k], a_lo = parts[p * len + k + 1];
            const double s = hi + a_hi;
            const double bp = s - hi;
            double e = (hi - (s - bp)) + (a_hi - bp);
            e = e + (lo + a_lo);
            hi = s + e;
            lo = e - (hi - s);
        }
        out[k] = hi;
        out[k + 1] = lo;
    }
    return QMC_OK;
}

int qmc_finalize(const double *sums, uint64_t m, uint64_t n, int is_complex, double *result,
                 double *Q, void *stream) {
    if (!sums || !result) return QMC_ERR_ARG;
    if (m < 2 || m > QMC_MAX_SHIFTS) return QMC_ERR_M;
    if (n < 1) return QMC_ERR_N;
    int st = device_ok();
    if (st) return st;
    return cuda_status(launch_finalize(sums, (int)m, n, is_complex ? 1 : 0, result, Q, (cudaStream_t)stream));
}

int qmc_evaluate(const qmc_integrand *f, uint64_t n, const uint64_t *z, int dim,
                 const uint64_t *shift, uint64_t i_begin, uint64_t count, double *out, void *stream) {
    int st = check_integrand_shape(f);
    if (st) return st;
    if (!z || !shift || !out) return QMC_ERR_ARG;
    if (dim != f->dim) return QMC_ERR_DIM;
    if (n < 2 || n >= kNMax) return QMC_ERR_N;
    if (i_begin > n || count > n - i_begin) return QMC_ERR_RANGE;
    for (int j = 0; j < dim; ++j)
        if (z[j] % n == 0 || gcd_u64(z[j] % n, n) != 1) return QMC_ERR_GENVEC;
    if ((st = device_ok())) return st;
    if (count == 0) return QMC_OK;
    SumsParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    p.i_begin = i_begin;
    p.i_end = i_begin + count;
    p.d = dim;
    p.m = 1;
    for (int j = 0; j < dim; ++j) p.dc[j] = dim_const(z[j] % n, n);
    p.shifts = shift;
    fill_integrand(p, f);
    return cuda_status(launch_evaluate(p, out, (cudaStream_t)stream));
}

static uint32_t hist_blocks(uint64_t n) {
    uint64_t b = (n + 4095) / 4096;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, 1024));
}

size_t qmc_histogram_workspace_bytes(uint64_t n, int dim, int bins) {
    if (dim < 1 || dim > QMC_MAX_DIM || bins < 1 || n < 1) return 0;
    return (size_t)hist_blocks(n) * dim * bins * sizeof(double);
}

int qmc_histogram(const qmc_integrand *f, uint64_t n, const uint64_t *z, int dim,
                  const uint64_t *shift, int bins, double *hist, void *workspace,
                  size_t workspace_bytes, void *stream) {
    int st = check_integrand_shape(f);
    if (st) return st;
    if (!z || !shift || !hist || !workspace) return QMC_ERR_ARG;
    if (dim != f->dim) return QMC_ERR_DIM;
    if (n < 2 || n >= kNMax) return QMC_ERR_N;
    if (bins < 1 || (size_t)dim * bins > 20480) return QMC_ERR_RANGE;
    for (int j = 0; j < dim; ++j)
        if (z[j] % n == 0 || gcd_u64(z[j] % n, n) != 1) return QMC_ERR_GENVEC;
    uint32_t nb = hist_blocks(n);
    if (workspace_bytes < (size_t)nb * dim * bins * sizeof(double)) return QMC_ERR_WORKSPACE;
    if ((st = device_ok())) return st;
    SumsParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = n;
    p.i_begin = 0;
    p.i_end = n;
    p.d = dim;
    p.m = 1;
    for (int j = 0; j < dim; ++j) p.dc[j] = dim_const(z[j] % n, n);
    p.shifts = shift;
    fill_integrand(p, f);
    return cuda_status(launch_histogram(p, bins, hist, (double *)workspace, nb, (cudaStream_t)stream));
}

}  // extern "C"
