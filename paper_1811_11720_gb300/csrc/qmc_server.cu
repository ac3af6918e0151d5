// qmc_server.cu -- serving loop: continuous batching of adaptive integrations.
//
// Requests (an integrand and an error goal) are queued on the host.  Each qmc_server_step:
//   1. admits queued requests in arrival order while device memory (a pool of the
//      configured budget) and slots allow: the request's coefficients, shifts and the
//      tile partials of its largest admissible lattice are reserved and uploaded once;
//   2. runs every admitted request on its current lattice in one batched launch per
//      integrand family (same kernels as qmc_batch_sums, default launch shape, so a
//      request's numbers do not depend on what else is in the batch);
//   3. reads back each request's mean and error, applies the error goal of the adaptive
//      mode (Sec. 3.3.1): met, or out of evaluations, completes the request and frees its
//      memory; otherwise the request moves to a larger table size for the next step
//      (results of the smaller lattice are discarded).
// Requests arriving while others run join at the next step: work of different requests
// overlaps on the device inside each launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "qmc_gb300.h"
#include "qmc_hostutil.h"
#include "qmc_internal.h"

using namespace qmc;
using namespace qmc::host;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    int state = QMC_REQ_PENDING;
    int status = QMC_OK;
    qmc_integrand fh{};      // scalars; host arrays below
    std::vector<double> c, w, ucoef, fcoef;
    std::vector<int64_t> h;
    std::vector<int32_t> uexp, fexp;
    double epsrel = 0, epsabs = 0;
    uint64_t minn = 0, maxeval = 0, seed = 0;
    // device reservation
    size_t off = 0, bytes = 0;
    qmc_integrand fd{};
    uint64_t *d_shifts = nullptr;
    double *d_partials = nullptr;
    uint64_t tiles_cap = 0;  // tiles of partials reserved
    std::vector<uint64_t> shifts;
    // progress
    uint64_t n = 0, evaluations = 0, iterations = 0;
    uint64_t waited = 0;     // steps spent waiting since the request last ran
    unsigned long long nonfinite = 0, signfail = 0;
    double res[4] = {0, 0, 0, 0};
    double t_submit = 0, t_done = 0;
};

}  // namespace

struct qmc_server {
    qmc_server_config cfg{};
    std::vector<uint64_t> tn, tz;
    int s_max = 0;
    cudaStream_t stream = nullptr;
    char *pool = nullptr;
    size_t pool_bytes = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size
    // fixed regions
    size_t fixed_bytes = 0;
    BatchItem *d_items = nullptr;
    uint64_t *d_tb = nullptr;
    double *d_sums = nullptr, *d_results = nullptr;
    unsigned long long *d_counters = nullptr;
    BatchItem *h_items = nullptr;
    uint64_t *h_tb = nullptr;
    double *h_results = nullptr;
    unsigned long long *h_counters = nullptr;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> active;
    std::deque<uint64_t> completed;   // finished, not yet reported by qmc_server_completed
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    std::mutex mu;
};

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

bool pool_alloc(qmc_server *s, size_t bytes, size_t *off) {
    bytes = al256(bytes);
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            size_t rest = it->second - bytes;
            size_t roff = it->first + bytes;
            s->free_blocks.erase(it);
            if (rest) s->free_blocks[roff] = rest;
            return true;
        }
    }
    return false;
}

void pool_free(qmc_server *s, size_t off, size_t bytes) {
    bytes = al256(bytes);
    auto it = s->free_blocks.emplace(off, bytes).first;
    // merge with the next and previous blocks
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

int next_table_n(const qmc_server *s, uint64_t preferred, uint64_t *n) {
    for (uint64_t v : s->tn)
        if (v >= preferred) {
            *n = v;
            return QMC_OK;
        }
    return QMC_ERR_N;
}

// Largest table size whose lattice still fits the request's evaluation budget.
uint64_t largest_admissible_n(const qmc_server *s, const Request &r) {
    uint64_t n0 = 0;
    if (next_table_n(s, r.minn, &n0)) return 0;
    uint64_t best = n0;
    for (uint64_t v : s->tn)
        if (v >= n0 && v * s->cfg.m <= std::max<uint64_t>(r.maxeval, n0 * s->cfg.m)) best = v;
    return best;
}

size_t request_bytes(const qmc_server *s, const Request &r, uint64_t nmax, uint64_t *tiles_cap) {
    const int d = r.fh.dim;
    const int cplx = is_complex_family(r.fh.family);
    // the partials of the largest tile count over the lattices the request may visit: the
    // count is not monotone in n (whole waves; e.g. 2261 tiles at n = 886,097 against 2257
    // at n = 974,707 for m = 32), so the largest lattice alone would under-reserve
    uint64_t n0 = 0;
    if (next_table_n(s, r.minn, &n0)) n0 = nmax;
    uint64_t tiles = 0;
    for (uint64_t v : s->tn)
        if (v >= n0 && v <= nmax) tiles = std::max(tiles, geometry(v, (int)s->cfg.m).tiles);
    size_t b = 0;
    b += al256(r.c.size() * 8) + al256(r.w.size() * 8) + al256(r.h.size() * 8);
    b += al256(r.ucoef.size() * 8) + al256(r.fcoef.size() * 8);
    b += al256(r.uexp.size() * 4) + al256(r.fexp.size() * 4);
    b += al256(s->cfg.m * d * 8);
    b += al256(tiles * s->cfg.m * 2 * sizeof(double) * (cplx ? 2 : 1));
    *tiles_cap = tiles;
    return b;
}

bool goal_met_req(const Request &r, int cplx) {
    double tre = std::max(r.epsabs, r.epsrel * std::fabs(r.res[0]));
    if (!cplx) return r.res[1] <= tre;
    double tim = std::max(r.epsabs, r.epsrel * std::fabs(r.res[2]));
    return r.res[1] <= tre && r.res[3] <= tim;
}

int admit(qmc_server *s, Request &r) {
    const uint64_t nmax = largest_admissible_n(s, r);
    if (!nmax) {
        r.state = QMC_REQ_DONE;
        r.status = QMC_ERR_N;
        r.t_done = now_s();
        return 1;
    }
    const size_t bytes = request_bytes(s, r, nmax, &r.tiles_cap);
    size_t off;
    if (!pool_alloc(s, bytes, &off)) return 0;
    r.off = off;
    r.bytes = bytes;
    char *p = s->pool + off;
    auto place = [&](const void *src, size_t nbytes) -> void * {
        void *dst = p;
        if (nbytes && src) cudaMemcpyAsync(dst, src, nbytes, cudaMemcpyHostToDevice, s->stream);
        p += al256(nbytes);
        return nbytes ? dst : nullptr;
    };
    r.fd = r.fh;
    r.fd.c = (const double *)place(r.c.data(), r.c.size() * 8);
    r.fd.w = (const double *)place(r.w.data(), r.w.size() * 8);
    r.fd.h = (const int64_t *)place(r.h.data(), r.h.size() * 8);
    r.fd.ucoef = (const double *)place(r.ucoef.data(), r.ucoef.size() * 8);
    r.fd.fcoef = (const double *)place(r.fcoef.data(), r.fcoef.size() * 8);
    r.fd.uexp = (const int32_t *)place(r.uexp.data(), r.uexp.size() * 4);
    r.fd.fexp = (const int32_t *)place(r.fexp.data(), r.fexp.size() * 4);
    r.shifts.resize(s->cfg.m * r.fh.dim);
    qmc_make_shifts(r.seed, s->cfg.m, r.fh.dim, r.shifts.data());
    r.d_shifts = (uint64_t *)place(r.shifts.data(), r.shifts.size() * 8);
    r.d_partials = (double *)p;
    next_table_n(s, r.minn, &r.n);
    r.state = QMC_REQ_ACTIVE;
    return 2;
}

qmc_rule rule_of(const qmc_server *s, const Request &r) {
    qmc_rule rule;
    std::memset(&rule, 0, sizeof(rule));
    rule.n = r.n;
    rule.dim = r.fh.dim;
    for (size_t c = 0; c < s->tn.size(); ++c)
        if (s->tn[c] == r.n)
            for (int j = 0; j < r.fh.dim; ++j) rule.z[j] = s->tz[c * s->s_max + j];
    rule.m = s->cfg.m;
    rule.shifts = r.d_shifts;
    rule.transform = s->cfg.transform;
    rule.fit = nullptr;
    return rule;
}

}  // namespace

extern "C" int qmc_server_create(const qmc_genvec_table *table, const qmc_server_config *cfg,
                                 void *stream, qmc_server **out) {
    if (!table || !cfg || !out || !table->n || !table->z || table->count < 1) return QMC_ERR_ARG;
    if (cfg->m < 2 || cfg->m > 256) return QMC_ERR_M;
    if (cfg->max_slots < 1 || cfg->max_slots > 65536) return QMC_ERR_ARG;
    int st = check_transform(cfg->transform);
    if (st) return st;
    if ((st = device_ok())) return st;
    qmc_server *s = new (std::nothrow) qmc_server;
    if (!s) return QMC_ERR_ARG;
    s->cfg = *cfg;
    s->s_max = table->s_max;
    s->tn.assign(table->n, table->n + table->count);
    s->tz.assign(table->z, table->z + (size_t)table->count * table->s_max);
    s->stream = (cudaStream_t)stream;
    const size_t slots = cfg->max_slots;
    s->fixed_bytes = al256(sizeof(BatchItem) * slots) + al256(sizeof(uint64_t) * (slots + 1)) +
                     al256(sizeof(double) * 4 * cfg->m * slots) + al256(sizeof(double) * 4 * slots) +
                     al256(sizeof(unsigned long long) * 2 * slots);
    if (cfg->memory_budget <= s->fixed_bytes) {
        delete s;
        return QMC_ERR_WORKSPACE;
    }
    s->pool_bytes = cfg->memory_budget;
    if (cudaMalloc(&s->pool, s->pool_bytes) != cudaSuccess) {
        delete s;
        return QMC_ERR_CUDA;
    }
    if (cudaMallocHost(&s->h_items, sizeof(BatchItem) * slots) != cudaSuccess ||
        cudaMallocHost(&s->h_tb, sizeof(uint64_t) * (slots + 1)) != cudaSuccess ||
        cudaMallocHost(&s->h_results, sizeof(double) * 4 * slots) != cudaSuccess ||
        cudaMallocHost(&s->h_counters, sizeof(unsigned long long) * 2 * slots) != cudaSuccess) {
        qmc_server_destroy(s);
        return QMC_ERR_CUDA;
    }
    char *p = s->pool;
    s->d_items = (BatchItem *)p;
    p += al256(sizeof(BatchItem) * slots);
    s->d_tb = (uint64_t *)p;
    p += al256(sizeof(uint64_t) * (slots + 1));
    s->d_sums = (double *)p;
    p += al256(sizeof(double) * 4 * cfg->m * slots);
    s->d_results = (double *)p;
    p += al256(sizeof(double) * 4 * slots);
    s->d_counters = (unsigned long long *)p;
    s->free_blocks[s->fixed_bytes] = s->pool_bytes - s->fixed_bytes;
    *out = s;
    return QMC_OK;
}

extern "C" void qmc_server_destroy(qmc_server *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->pool) cudaFree(s->pool);
    if (s->h_items) cudaFreeHost(s->h_items);
    if (s->h_tb) cudaFreeHost(s->h_tb);
    if (s->h_results) cudaFreeHost(s->h_results);
    if (s->h_counters) cudaFreeHost(s->h_counters);
    delete s;
}

extern "C" int qmc_server_submit(qmc_server *s, const qmc_integrand *f, double epsrel,
                                 double epsabs, uint64_t minn, uint64_t maxeval, uint64_t seed,
                                 uint64_t *id) {
    if (!s || !f || !id) return QMC_ERR_ARG;
    int st = check_integrand_shape(f);
    if (st) return st;
    if (!batch_family_supported(f->family)) return QMC_ERR_INTEGRAND;
    if (f->dim > s->s_max) return QMC_ERR_DIM;
    Request r;
    r.fh = *f;
    const int d = f->dim;
    if (f->c) r.c.assign(f->c, f->c + d);
    if (f->w) r.w.assign(f->w, f->w + d);
    if (f->h) r.h.assign(f->h, f->h + d);
    if (f->ucoef) r.ucoef.assign(f->ucoef, f->ucoef + f->nu);
    if (f->fcoef) r.fcoef.assign(f->fcoef, f->fcoef + f->nf);
    if (f->uexp) r.uexp.assign(f->uexp, f->uexp + (size_t)f->nu * d);
    if (f->fexp) r.fexp.assign(f->fexp, f->fexp + (size_t)f->nf * d);
    r.epsrel = epsrel;
    r.epsabs = epsabs;
    r.minn = minn;
    r.maxeval = maxeval;
    r.seed = seed;
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    r.id = s->next_id++;
    *id = r.id;
    s->reqs.emplace(r.id, std::move(r));
    s->pending.push_back(*id);
    return QMC_OK;
}

extern "C" int qmc_server_step(qmc_server *s, int *completed) {
    if (!s) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    int done = 0;
    // 1. admission in arrival order
    while (!s->pending.empty() && (int)s->active.size() < s->cfg.max_slots) {
        Request &r = s->reqs[s->pending.front()];
        int a = admit(s, r);
        if (a == 0) break;   // out of memory: wait for completions
        s->pending.pop_front();
        if (a == 1) {
            ++done;
            s->completed.push_back(r.id);
        } else {
            s->active.push_back(r.id);
        }
    }
    if (s->active.empty()) {
        if (completed) *completed = done;
        return QMC_OK;
    }
    // 2. the requests of this step: all, or shortest (aged) first within the budget
    std::vector<uint64_t> run = s->active, idle;
    if (s->cfg.step_evaluations) {
        std::vector<std::pair<double, size_t>> key;
        for (size_t q = 0; q < s->active.size(); ++q) {
            const Request &r = s->reqs[s->active[q]];
            key.push_back({(double)r.n * (double)s->cfg.m / (1.0 + (double)r.waited), q});
        }
        std::stable_sort(key.begin(), key.end());
        run.clear();
        uint64_t spent = 0;
        size_t nchosen = 0;
        std::vector<char> chosen(s->active.size(), 0);
        for (const auto &kv : key) {
            const Request &r = s->reqs[s->active[kv.second]];
            const uint64_t cost = r.n * s->cfg.m;
            if (nchosen && spent + cost > s->cfg.step_evaluations) continue;
            spent += cost;
            chosen[kv.second] = 1;
            ++nchosen;
        }
        for (size_t q = 0; q < s->active.size(); ++q) {
            Request &r = s->reqs[s->active[q]];
            if (chosen[q]) {
                run.push_back(r.id);
                r.waited = 0;
            } else {
                idle.push_back(r.id);
                ++r.waited;
            }
        }
    }
    // one batched launch per family over the requests of this step
    std::vector<int> fams;
    for (uint64_t id : run) {
        int fam = s->reqs[id].fh.family;
        if (std::find(fams.begin(), fams.end(), fam) == fams.end()) fams.push_back(fam);
    }
    const int m = (int)s->cfg.m;
    const int spb = std::max(1, kSumsThreads / m);
    if (cudaMemsetAsync(s->d_counters, 0, sizeof(unsigned long long) * 2 * run.size(), s->stream) != cudaSuccess)
        return QMC_ERR_CUDA;
    std::vector<uint64_t> order;   // request id per batch slot
    size_t base = 0;
    for (int fam : fams) {
        const size_t g0 = base;
        uint64_t tiles = 0;
        for (uint64_t id : run) {
            Request &r = s->reqs[id];
            if (r.fh.family != fam) continue;
            qmc_batch_item b;
            b.f = r.fd;
            b.rule = rule_of(s, r);
            b.i_begin = 0;
            b.i_end = r.n;
            BatchItem &it = s->h_items[base];
            int st = fill_batch_item(it, b, m, spb, 0, fam);
            if (st) return st;
            if (it.tiles > r.tiles_cap) return QMC_ERR_WORKSPACE;   // never: see request_bytes
            it.tile_begin = tiles;
            it.partial_off = (uint64_t)(r.d_partials - (double *)s->pool);
            s->h_tb[base - g0] = tiles;
            tiles += it.tiles;
            order.push_back(id);
            ++base;
        }
        const int cnt = (int)(base - g0);
        s->h_tb[cnt] = tiles;
        const int cplx = is_complex_family(fam);
        BatchItem *di = s->d_items + g0;
        if (cudaMemcpyAsync(di, s->h_items + g0, sizeof(BatchItem) * cnt, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(s->d_tb, s->h_tb, sizeof(uint64_t) * (cnt + 1), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return QMC_ERR_CUDA;
        if (launch_batch(fam, di, s->d_tb, cnt, tiles, m, spb, (double *)s->pool, s->d_counters + 2 * g0, s->stream) != cudaSuccess ||
            launch_batch_reduce(di, cnt, m, cplx, (double *)s->pool, s->d_sums + g0 * 4 * m, s->stream) != cudaSuccess ||
            launch_batch_finalize(di, cnt, m, cplx, s->d_sums + g0 * 4 * m, s->d_results + 4 * g0, s->stream) != cudaSuccess)
            return QMC_ERR_CUDA;
        // the tile prefix array is reused by the next family: order the host writes
        if (fams.size() > 1 && cudaStreamSynchronize(s->stream) != cudaSuccess) return QMC_ERR_CUDA;
    }
    const size_t na = order.size();
    if (cudaMemcpyAsync(s->h_results, s->d_results, sizeof(double) * 4 * na, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->h_counters, s->d_counters, sizeof(unsigned long long) * 2 * na, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return QMC_ERR_CUDA;
    // 3. goals, escalation, completion
    std::vector<uint64_t> still = idle;
    const double t = now_s();
    for (size_t q = 0; q < na; ++q) {
        Request &r = s->reqs[order[q]];
        const int cplx = is_complex_family(r.fh.family);
        std::memcpy(r.res, s->h_results + 4 * q, sizeof(r.res));
        r.nonfinite += s->h_counters[2 * q];
        r.signfail += s->h_counters[2 * q + 1];
        r.evaluations += r.n * s->cfg.m;
        r.iterations += 1;
        bool finish = goal_met_req(r, cplx) || r.evaluations >= r.maxeval;
        if (!finish) {
            double goal = std::max(std::max(r.epsabs, r.epsrel * std::fabs(r.res[0])), 1e-300);
            double ratio = r.res[1] / goal;
            if (cplx) ratio = std::max(ratio, r.res[3] / std::max(std::max(r.epsabs, r.epsrel * std::fabs(r.res[2])), 1e-300));
            ratio = std::max(ratio, 1.0);
            uint64_t nn = 0;
            const double pref = (double)r.n * ratio;
            if (pref >= (double)s->tn.back() || next_table_n(s, (uint64_t)pref + 1, &nn) != QMC_OK) nn = s->tn.back();
            if (nn <= r.n && next_table_n(s, r.n + 1, &nn) != QMC_OK) nn = 0;
            // stay within the evaluation budget and the reserved partials
            const uint64_t cap = largest_admissible_n(s, r);
            const uint64_t remaining = r.maxeval > r.evaluations ? r.maxeval - r.evaluations : 0;
            if (nn && (nn > cap || nn * s->cfg.m > remaining)) {
                uint64_t best = 0;
                for (uint64_t v : s->tn)
                    if (v > r.n && v <= cap && v * s->cfg.m <= remaining) best = v;
                nn = best;
            }
            if (nn) r.n = nn;
            else finish = true;
        }
        if (finish) {
            r.state = QMC_REQ_DONE;
            r.status = r.nonfinite ? QMC_ERR_NONFINITE : QMC_OK;
            r.t_done = t;
            pool_free(s, r.off, r.bytes);
            ++done;
            s->completed.push_back(r.id);
        } else {
            still.push_back(r.id);
        }
    }
    s->active.swap(still);
    if (completed) *completed = done;
    return QMC_OK;
}

extern "C" int qmc_server_status(qmc_server *s, uint64_t id, int *state, qmc_result *result,
                                 double *latency_s) {
    if (!s) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return QMC_ERR_ARG;
    const Request &r = it->second;
    if (state) *state = r.state;
    if (result) {
        const int cplx = is_complex_family(r.fh.family);
        result->integral.re = r.res[0];
        result->error.re = r.res[1];
        result->integral.im = cplx ? r.res[2] : 0.0;
        result->error.im = cplx ? r.res[3] : 0.0;
        result->n = r.n;
        result->m = s->cfg.m;
        result->iterations = r.iterations;
        result->evaluations = r.evaluations;
        result->nonfinite = r.nonfinite;
        result->signfail = r.signfail;
    }
    if (latency_s) *latency_s = r.state == QMC_REQ_DONE ? r.t_done - r.t_submit : -1.0;
    return r.state == QMC_REQ_DONE ? r.status : QMC_OK;
}

extern "C" int qmc_server_completed(qmc_server *s, uint64_t *ids, int cap, int *count) {
    if (!s || !ids || !count || cap < 0) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    int k = 0;
    while (k < cap && !s->completed.empty()) {
        ids[k++] = s->completed.front();
        s->completed.pop_front();
    }
    *count = k;
    return QMC_OK;
}

extern "C" int qmc_server_counts(qmc_server *s, int *pending, int *active, size_t *free_bytes) {
    if (!s) return QMC_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    if (pending) *pending = (int)s->pending.size();
    if (active) *active = (int)s->active.size();
    if (free_bytes) {
        size_t f = 0;
        for (auto &b : s->free_blocks) f += b.second;
        *free_bytes = f;
    }
    return QMC_OK;
}
