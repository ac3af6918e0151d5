// qmc_host.cu -- qmc_integrate(): the host-buffer entry point (App. A.2 integrate()).
//
// Uploads the integrand and the shifts into a library-owned device arena (one per device,
// grown on demand and reused), optionally runs the variance-reduction fit (histogram
// kernel + host Levenberg-Marquardt), then the lattice sums, the fixed-order tile reduction
// and the shift reduction, and reads back the four result numbers and two counters.  With
// options it repeats on larger lattices until the error goal is met (Sec. 3.3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "qmc_gb300.h"
#include "qmc_internal.h"

namespace {

struct Arena {
    int device = -1;
    char *base = nullptr;
    size_t cap = 0;
};

std::mutex g_mutex;
std::vector<Arena> g_arenas;

// Returns a device buffer of at least `bytes` for the current device (caller holds g_mutex).
char *arena_get(size_t bytes, int *status) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *status = QMC_ERR_NO_DEVICE;
        return nullptr;
    }
    Arena *a = nullptr;
    for (auto &x : g_arenas)
        if (x.device == dev) a = &x;
    if (!a) {
        g_arenas.push_back(Arena{dev, nullptr, 0});
        a = &g_arenas.back();
    }
    if (a->cap < bytes) {
        if (a->base) cudaFree(a->base);
        a->base = nullptr;
        a->cap = 0;
        size_t want = std::max(bytes, (size_t)1 << 20);
        if (cudaMalloc(&a->base, want) != cudaSuccess) {
            *status = QMC_ERR_CUDA;
            return nullptr;
        }
        a->cap = want;
    }
    *status = QMC_OK;
    return a->base;
}

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
    size_t off_c, off_w, off_h, off_uc, off_fc, off_ue, off_fe, off_shift, off_fit, off_sums,
        off_res, off_cnt, off_hist, off_hws, off_ws, total;
};

bool goal_met(const double *res, int cplx, const qmc_options *o) {
    double tol_re = std::max(o->epsabs, o->epsrel * std::fabs(res[0]));
    if (!cplx) return res[1] <= tol_re;
    double tol_im = std::max(o->epsabs, o->epsrel * std::fabs(res[2]));
    if (o->errormode == QMC_ERRORMODE_LARGEST) {
        double big = std::max(std::fabs(res[0]), std::fabs(res[2]));
        return std::max(res[1], res[3]) <= std::max(o->epsabs, o->epsrel * big);
    }
    return res[1] <= tol_re && res[3] <= tol_im;
}

double error_ratio(const double *res, int cplx, const qmc_options *o) {
    double r = res[1] / std::max(std::max(o->epsabs, o->epsrel * std::fabs(res[0])), 1e-300);
    if (cplx) r = std::max(r, res[3] / std::max(std::max(o->epsabs, o->epsrel * std::fabs(res[2])), 1e-300));
    return r;
}

}  // namespace

extern "C" int qmc_integrate(const qmc_integrand *f, const qmc_genvec_table *table,
                             uint64_t n_or_minn, uint64_t m, qmc_transform transform,
                             const qmc_fit_opts *fit, uint64_t seed, const qmc_options *opts,
                             void *stream, qmc_result *out) {
    if (!f || !table || !out || !table->n || !table->z) return QMC_ERR_ARG;
    if (f->dim < 1 || f->dim > QMC_MAX_DIM || f->dim > table->s_max) return QMC_ERR_DIM;
    if (m < 2 || m > QMC_MAX_SHIFTS) return QMC_ERR_M;
    const int d = f->dim;
    const int cplx = (f->family == QMC_FEYNMAN);
    const bool use_fit = fit && fit->enabled;
    const int bins = use_fit ? (fit->bins > 0 ? fit->bins : 1000) : 0;
    cudaStream_t s = (cudaStream_t)stream;

    uint64_t n = 0;
    int st = qmc_get_next_n(table, n_or_minn, &n);
    if (st) return st;
    const uint64_t n_max = table->n[table->count - 1];
    uint64_t n_fit = 0;
    if (use_fit) {
        st = qmc_get_next_n(table, fit->evaluateminn ? fit->evaluateminn : 100000, &n_fit);
        if (st) return st;
    }
    const uint64_t m_cap = opts ? QMC_MAX_SHIFTS : m;

    // device layout (worst case over the adaptive loop: largest n, m_cap shifts)
    Layout L;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al(std::max<size_t>(b, 8)); return r; };
    L.off_c = take(d * sizeof(double));
    L.off_w = take(d * sizeof(double));
    L.off_h = take(d * sizeof(int64_t));
    L.off_uc = take((size_t)std::max(f->nu, 0) * sizeof(double));
    L.off_fc = take((size_t)std::max(f->nf, 0) * sizeof(double));
    L.off_ue = take((size_t)std::max(f->nu, 0) * d * sizeof(int32_t));
    L.off_fe = take((size_t)std::max(f->nf, 0) * d * sizeof(int32_t));
    L.off_shift = take(m_cap * d * sizeof(uint64_t));
    L.off_fit = take(6 * d * sizeof(double));
    L.off_sums = take(4 * m_cap * sizeof(double));
    L.off_res = take(4 * sizeof(double));
    L.off_cnt = take(2 * sizeof(unsigned long long));
    L.off_hist = take(use_fit ? (size_t)d * bins * sizeof(double) : 8);
    L.off_hws = take(use_fit ? qmc_histogram_workspace_bytes(n_fit, d, bins) : 8);
    // lattice-sum workspace: the largest over the (n, m) pairs the loop may visit, i.e. n
    // with m, and with options every table size up to n_max with m and then n_max with
    // m doubled up to QMC_MAX_SHIFTS.  The tile count is not monotone in n (whole waves),
    // so neither the largest n nor the largest m alone bounds it.
    qmc_rule probe;
    std::memset(&probe, 0, sizeof(probe));
    probe.dim = d;
    auto ws_need = [&](uint64_t v, uint64_t mm) {
        probe.n = v;
        probe.m = mm;
        return qmc_sums_workspace_bytes(&probe, cplx, 0, v);
    };
    size_t ws_bytes = 0;
    for (int c = 0; c < table->count; ++c) {
        const uint64_t v = table->n[c];
        if (v >= n && v <= (opts ? n_max : n)) ws_bytes = std::max(ws_bytes, ws_need(v, m));
    }
    if (opts)
        for (uint64_t mm = 2 * m; mm <= QMC_MAX_SHIFTS; mm *= 2) ws_bytes = std::max(ws_bytes, ws_need(n_max, mm));
    L.off_ws = take(ws_bytes);
    L.total = o;

    std::lock_guard<std::mutex> lock(g_mutex);
    char *base = arena_get(L.total, &st);
    if (st) return st;

    qmc_integrand df = *f;   // device copy of the description
    auto up = [&](size_t off, const void *src, size_t bytes) -> cudaError_t {
        if (!src || !bytes) return cudaSuccess;
        return cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = cudaSuccess;
    if (f->c) { e = up(L.off_c, f->c, d * sizeof(double)); df.c = (const double *)(base + L.off_c); }
    if (e == cudaSuccess && f->w) { e = up(L.off_w, f->w, d * sizeof(double)); df.w = (const double *)(base + L.off_w); }
    if (e == cudaSuccess && f->h) { e = up(L.off_h, f->h, d * sizeof(int64_t)); df.h = (const int64_t *)(base + L.off_h); }
    if (e == cudaSuccess && f->ucoef) { e = up(L.off_uc, f->ucoef, f->nu * sizeof(double)); df.ucoef = (const double *)(base + L.off_uc); }
    if (e == cudaSuccess && f->fcoef) { e = up(L.off_fc, f->fcoef, f->nf * sizeof(double)); df.fcoef = (const double *)(base + L.off_fc); }
    if (e == cudaSuccess && f->uexp) { e = up(L.off_ue, f->uexp, (size_t)f->nu * d * sizeof(int32_t)); df.uexp = (const int32_t *)(base + L.off_ue); }
    if (e == cudaSuccess && f->fexp) { e = up(L.off_fe, f->fexp, (size_t)f->nf * d * sizeof(int32_t)); df.fexp = (const int32_t *)(base + L.off_fe); }
    if (e != cudaSuccess) return QMC_ERR_CUDA;

    // generating vector of a table size
    auto zrow = [&](uint64_t nn, uint64_t *z) -> int {
        for (int c = 0; c < table->count; ++c)
            if (table->n[c] == nn) {
                for (int j = 0; j < d; ++j) z[j] = table->z[(size_t)c * table->s_max + j];
                return QMC_OK;
            }
        return QMC_ERR_N;
    };

    // variance-reduction fit (Sec. 2.4; Sec. 3.3.1: fit first, then periodize the fitted
    // integrand).  The fit lattice uses one shift: outputs 0..d-1 of the SplitMix64 stream
    // seeded with seed + 1.
    double *d_fit = nullptr;
    if (use_fit) {
        uint64_t zf[QMC_MAX_DIM], sh[QMC_MAX_DIM];
        if ((st = zrow(n_fit, zf))) return st;
        qmc_make_shifts(seed + 1, 1, d, sh);
        uint64_t *d_sh = (uint64_t *)(base + L.off_shift);
        if (cudaMemcpyAsync(d_sh, sh, d * sizeof(uint64_t), cudaMemcpyHostToDevice, s) != cudaSuccess) return QMC_ERR_CUDA;
        double *d_hist = (double *)(base + L.off_hist);
        st = qmc_histogram(&df, n_fit, zf, d, d_sh, bins, d_hist, base + L.off_hws,
                           qmc_histogram_workspace_bytes(n_fit, d, bins), stream);
        if (st) return st;
        std::vector<double> hist((size_t)d * bins), params(6 * d);
        if (cudaMemcpyAsync(hist.data(), d_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return QMC_ERR_CUDA;
        if ((st = qmc_fit_polysingular(hist.data(), d, bins, fit, params.data()))) return st;
        d_fit = (double *)(base + L.off_fit);
        if (cudaMemcpyAsync(d_fit, params.data(), params.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return QMC_ERR_CUDA;
    }

    uint64_t cur_m = m;
    uint64_t evals = 0, iters = 0;
    unsigned long long counters_total[2] = {0, 0};
    double res[4] = {0, 0, 0, 0};
    std::vector<uint64_t> sh;
    uint64_t shifts_m = 0;
    for (;;) {
        qmc_rule rule;
        std::memset(&rule, 0, sizeof(rule));
        rule.n = n;
        rule.dim = d;
        if ((st = zrow(n, rule.z))) return st;
        rule.m = cur_m;
        rule.transform = transform;
        rule.fit = d_fit;
        if (shifts_m != cur_m) {
            sh.resize(cur_m * d);
            qmc_make_shifts(seed, cur_m, d, sh.data());
            if (cudaMemcpyAsync(base + L.off_shift, sh.data(), sh.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return QMC_ERR_CUDA;
            shifts_m = cur_m;
        }
        rule.shifts = (const uint64_t *)(base + L.off_shift);
        unsigned long long *d_cnt = (unsigned long long *)(base + L.off_cnt);
        if (cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return QMC_ERR_CUDA;
        double *d_sums = (double *)(base + L.off_sums);
        // the reservation, so that qmc_sums' size check guards it
        st = qmc_sums(&df, &rule, 0, n, base + L.off_ws, ws_bytes, d_sums, d_cnt, stream);
        if (st) return st;
        double *d_res = (double *)(base + L.off_res);
        if ((st = qmc_finalize(d_sums, cur_m, n, cplx, d_res, nullptr, stream))) return st;
        unsigned long long cnt[2];
        if (cudaMemcpyAsync(res, d_res, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return QMC_ERR_CUDA;
        counters_total[0] += cnt[0];
        counters_total[1] += cnt[1];
        evals += n * cur_m;
        ++iters;
        if (!opts || goal_met(res, cplx, opts) || evals >= opts->maxeval) break;
        // Larger lattice (results of this iteration are discarded, Sec. 3.3.1).  The error
        // is assumed to fall at least like 1/n: n_next = n * (error / goal).
        double ratio = std::max(error_ratio(res, cplx, opts), 1.0);
        double pref = (double)n * ratio;
        uint64_t n_next;
        if (pref >= (double)n_max || n == n_max) {
            if (n == n_max) {
                if (cur_m * 2 > QMC_MAX_SHIFTS) break;
                cur_m *= 2;   // beyond the table: more shifts (Monte Carlo scaling)
                n_next = n_max;
            } else {
                n_next = n_max;
            }
        } else if (qmc_get_next_n(table, (uint64_t)pref + 1, &n_next) != QMC_OK) {
            n_next = n_max;
        }
        if (n_next <= n && cur_m == shifts_m) {
            if (qmc_get_next_n(table, n + 1, &n_next) != QMC_OK) break;
        }
        // stay within maxeval where a smaller admissible lattice exists
        uint64_t remaining = opts->maxeval > evals ? opts->maxeval - evals : 0;
        if (n_next * cur_m > remaining) {
            uint64_t best = 0;
            for (int c = 0; c < table->count; ++c)
                if (table->n[c] > n && table->n[c] * cur_m <= remaining) best = table->n[c];
            if (best == 0) break;
            n_next = best;
        }
        n = n_next;
    }
    out->integral.re = res[0];
    out->error.re = res[1];
    out->integral.im = cplx ? res[2] : 0.0;
    out->error.im = cplx ? res[3] : 0.0;
    out->n = n;
    out->m = cur_m;
    out->iterations = iters;
    out->evaluations = evals;
    out->nonfinite = counters_total[0];
    out->signfail = counters_total[1];
    return counters_total[0] ? QMC_ERR_NONFINITE : QMC_OK;
}
