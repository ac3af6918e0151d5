/*
 * qmc_gb300.h -- C ABI of a GB300 (sm_103a) implementation of randomly shifted rank-1
 * lattice quadrature, the quasi-Monte Carlo method of Borowka, Heinrich, Jahn, Jones,
 * Kerner, Schlenk, "A GPU compatible quasi-Monte Carlo integrator interfaced to pySecDec"
 * (arXiv:1811.11720).
 *
 * The estimator (Sec. 2.1, Eq. (lattice)) is
 *     Q^(k) = (1/n) sum_{i<n} g({ i z / n + Delta_k }),    Qbar = (1/m) sum_{k<m} Q^(k),
 * and its error (Eq. (lattice-error)) is sigma = sqrt( sum_k (Q^(k) - Qbar)^2 / (m (m-1)) ),
 * per real component.  g is the integrand f after the optional PolySingular
 * variance-reduction map (Sec. 2.4, Eq. (ISfit)) and a periodizing transform (Sec. 2.3).
 *
 * Conventions used by every entry point
 *   - Return value: QMC_OK (0) on success, a negative QMC_ERR_* code otherwise; nothing is
 *     written to outputs on argument errors.  qmc_strerror() gives a message.
 *   - Pointers documented as "device" must be CUDA device (or managed) memory on the
 *     current device; "host" pointers are ordinary host memory.  The caller owns every
 *     input and output buffer; the library never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device entry points only
 *     enqueue work and return; results are valid after the stream is synchronised.
 *   - Lattice points are exact: r = i z_j mod n in integer arithmetic and
 *     u = RN( frac(r/n + D 2^-53) ), the exact rational rounded once to the nearest
 *     double (ties to even), where the shift Delta_{k,j} = D_{k,j} 2^-53 and D is a 53-bit
 *     integer.  u can equal 1.0 when the fraction lies within half an ulp of 1.
 *   - Sums are deterministic: the same inputs and i-range give bit-identical results.
 */
#ifndef QMC_GB300_H
#define QMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMC_ABI_VERSION 1
#define QMC_MAX_DIM 16      /* integration variables per integrand */
#define QMC_MAX_SHIFTS 1024 /* random shifts m (the paper's maxmperpackage default) */
#define QMC_MAX_TERMS 512   /* monomials per polynomial (U and F each) */
#define QMC_NOALLOC_SCRATCH_BYTES (8u << 20) /* fixed device scratch of qmc_sums_noalloc */

/* ---- status codes ------------------------------------------------------------------ */
enum {
    QMC_OK = 0,
    QMC_ERR_ARG = -1,        /* NULL pointer, unknown enum, inconsistent sizes          */
    QMC_ERR_DIM = -2,        /* dim < 1, dim > QMC_MAX_DIM, or dim > table s_max         */
    QMC_ERR_N = -3,          /* n < 2, n >= 2^63, or no table size >= the request        */
    QMC_ERR_GENVEC = -4,     /* some z_j = 0 (mod n) or gcd(z_j, n) != 1                  */
    QMC_ERR_M = -5,          /* m < 2 (sigma undefined) or m > QMC_MAX_SHIFTS            */
    QMC_ERR_FIT_PARAMS = -6, /* PolySingular a0 < 1.001 or a1 > -0.001 (Sec. 2.4)         */
    QMC_ERR_INTEGRAND = -7,  /* unknown family or bad coefficient arrays                 */
    QMC_ERR_TRANSFORM = -8,  /* unknown transform or orders out of range                 */
    QMC_ERR_CUDA = -9,       /* a CUDA runtime call failed                               */
    QMC_ERR_WORKSPACE = -10, /* workspace smaller than qmc_sums_workspace_bytes()         */
    QMC_ERR_NONFINITE = -11, /* the integrand produced NaN or Inf (result still returned) */
    QMC_ERR_RANGE = -12,     /* empty or out-of-range i-range / bins                     */
    QMC_ERR_NO_DEVICE = -13  /* no CUDA device, or the device is not sm_103             */
};

/* ---- value types -------------------------------------------------------------------- */
typedef struct { double re, im; } qmc_c64;

/* Result of an integration (the paper's result struct, App. A.2 integrate()). */
typedef struct {
    qmc_c64 integral;      /* Qbar (imaginary part 0 for real integrands)              */
    qmc_c64 error;         /* sigma per component                                     */
    uint64_t n;            /* size of the last lattice                                  */
    uint64_t m;            /* shifts of the last lattice                                */
    uint64_t iterations;   /* lattices evaluated (Case 1 escalation)                    */
    uint64_t evaluations;  /* integrand evaluations in total                            */
    uint64_t nonfinite;    /* samples that were NaN or Inf (excluded from nothing)       */
    uint64_t signfail;     /* complex family: samples with Im F(z) > 0                  */
} qmc_result;

/* Integrand families.  The paper's integrand is a C++ functor compiled into the kernel
 * (Sec. 3.2, minimal example); across a C ABI it is described by data instead. */
enum {
    QMC_GENZ_OSCILLATORY = 1,   /* cos(2 pi w_1 + sum c_i x_i)          Sec. 5.2 table */
    QMC_GENZ_PRODUCT_PEAK = 2,  /* prod (c_i^-2 + (x_i - w_i)^2)^-1                 */
    QMC_GENZ_CORNER_PEAK = 3,   /* (1 + sum c_i x_i)^-(d+1)                         */
    QMC_GENZ_GAUSSIAN = 4,      /* exp(-sum c_i^2 (x_i - w_i)^2)                   */
    QMC_GENZ_C0 = 5,            /* exp(-sum c_i |x_i - w_i|)                        */
    QMC_GENZ_DISCONTINUOUS = 6, /* 0 if x_1 > w_1 or x_2 > w_2 else exp(sum c_i x_i) */
    QMC_MONOMIAL = 10,          /* prod x_i (the minimal example of Sec. 3.2)       */
    QMC_TRIG = 11,              /* prod (1 + c_i cos(2 pi (h_i x_i + w_i)))          */
    QMC_FEYNMAN = 20,           /* complex U(z)^a F(z)^-b det(dz/dx), deformed contour */
    QMC_SECTOR = 21             /* real U(x)^a F(x)^-b                               */
};

/* Integrand description.  For host entry points the arrays are host memory, for device
 * entry points device memory.  Unused arrays may be NULL.
 *   Genz / trig:  c[dim], w[dim]; trig also h[dim] (integer frequencies).
 *   Polynomial families: U = sum_m ucoef[m] prod_k x_k^uexp[m*dim+k] (nu terms), F likewise
 *   (nf terms), exponents 0..15; the value is U^pa F^-pb (principal branch) times, for
 *   QMC_FEYNMAN, det(dz/dx) at z_k = x_k - i lambda x_k (1 - x_k) dF/dx_k (real x).
 *   Arithmetic is FP64 except for two integer-pipe forms in 64-bit fixed point, chosen at
 *   staging: QMC_SECTOR's dense F when its coefficients are non-negative with a constant
 *   term c0 > 0 and the bound 4.5 N (sum of coefficients / c0) 2^-62 on its relative error
 *   (N products) is at most 2^-42; QMC_FEYNMAN's Hessian, dF and dU for dim 3..6 (deg U <= 2,
 *   deg F <= 3), each within 2^-49 of the sum of |coefficients|.  U(x), F(x) of QMC_FEYNMAN,
 *   and everything else, stay FP64. */
typedef struct {
    int family;
    int dim;
    const double *c, *w;
    const int64_t *h;
    int nu, nf;
    const double *ucoef, *fcoef;
    const int32_t *uexp, *fexp;
    double pa, pb, lambda;
} qmc_integrand;

/* Periodizing transforms (Sec. 2.3; table of integral transforms, App. A.4). */
enum { QMC_T_NONE = 0, QMC_T_BAKER = 1, QMC_T_KOROBOV = 2, QMC_T_SIDI = 3 };
typedef struct {
    int kind;
    int r0, r1;   /* Korobov<r0,r1>: weight ~ u^r0 (1-u)^r1, 0 <= r <= 8; Sidi<r0>, 1 <= r0 <= 8 */
} qmc_transform;

/* Generating-vector table (App. A.1 field generatingvectors; App. A.3): count sizes n[]
 * in ascending order, row c of z[] (count x s_max, row-major) is the vector for n[c]. */
typedef struct {
    const uint64_t *n;
    const uint64_t *z;
    int s_max;
    int count;
} qmc_genvec_table;

/* One shifted lattice rule with its inputs resident on the device. */
typedef struct {
    uint64_t n;                 /* lattice size, 2 <= n < 2^63                          */
    int dim;                    /* integration variables                                */
    uint64_t z[QMC_MAX_DIM];    /* generating vector (host copy), gcd(z_j, n) = 1       */
    uint64_t m;                 /* shifts, 1 <= m <= QMC_MAX_SHIFTS                     */
    const uint64_t *shifts;     /* device [m][dim] 53-bit integers D, Delta = D 2^-53   */
    qmc_transform transform;
    const double *fit;          /* device [dim][6] PolySingular a0..a5 or NULL (no fit) */
} qmc_rule;

/* Variance-reduction fit options (App. A.1 fields evaluateminn, fitstepsize, fitmaxiter,
 * fitxtol, fitgtol, fitftol). */
typedef struct {
    int enabled;
    uint64_t evaluateminn;  /* default 100000 */
    int bins;               /* histogram bins per dimension, default 1000 */
    int maxiter;            /* default 40 */
    double xtol, gtol, ftol;/* defaults 3e-3, 1e-8, 1e-8 */
    int stepsize;           /* every stepsize-th CDF point enters the fit, default 10 */
} qmc_fit_opts;

/* Error goal for the adaptive mode (App. A.1 fields minn, minm, epsrel, epsabs, maxeval,
 * errormode). */
enum { QMC_ERRORMODE_ALL = 0, QMC_ERRORMODE_LARGEST = 1 };
typedef struct {
    double epsrel, epsabs;
    uint64_t maxeval;
    int errormode;
} qmc_options;

/* ---- host helpers ------------------------------------------------------------------- */
const char *qmc_strerror(int code);
int qmc_abi_version(void);

/* Smallest table size >= preferred (App. A.2 get_next_n).  Errors: QMC_ERR_ARG,
 * QMC_ERR_N when every size is smaller. */
int qmc_get_next_n(const qmc_genvec_table *table, uint64_t preferred, uint64_t *n_out);

/* Random shifts (Sec. 2.1: Delta_k i.i.d. uniform on [0,1)^d).  D_out[k*dim + j] (host,
 * m*dim entries) = output number k*dim + j of the SplitMix64 generator seeded with `seed`,
 * shifted right by 11 bits.  Errors: QMC_ERR_ARG, QMC_ERR_DIM, QMC_ERR_M. */
int qmc_make_shifts(uint64_t seed, uint64_t m, int dim, uint64_t *D_out);

/* ---- device entry points (inputs resident on the device) --------------------------- */

/* Lattice points u[(i - i_begin)*m*dim + k*dim + j] for i_begin <= i < i_begin + count
 * (Eq. (lattice), Fig. 1), written to device memory out[count*m*dim].  No transform.
 * Errors: QMC_ERR_ARG/N/GENVEC/DIM/M/RANGE, QMC_ERR_CUDA. */
int qmc_points(const qmc_rule *rule, uint64_t i_begin, uint64_t count, double *out, void *stream);

/* Device scratch needed by qmc_sums for the i-range [i_begin, i_end) (per-tile partial
 * sums; the tiling is fixed by the range, not by the device).  For m <= 256 a qmc_sums
 * call leaves its tile partials at the start of the workspace in the layout of
 * qmc_sums_tiles (tiles x m (sum, compensation) pairs, then the imaginary block), so a
 * caller can check or reuse them. */
size_t qmc_sums_workspace_bytes(const qmc_rule *rule, int is_complex, uint64_t i_begin,
                                uint64_t i_end);

/* Per-shift sums S_k = sum_{i_begin <= i < i_end} g(x_{i,k}) (Eq. (lattice) before the 1/n).
 * `f` holds device pointers.  sums (device) receives double-double pairs:
 * sums[2k], sums[2k+1] = (hi, lo) of Re S_k, and for complex integrands
 * sums[2m + 2k], sums[2m + 2k + 1] = (hi, lo) of Im S_k.  counters (device, may be NULL)
 * receives [0] += samples that were NaN/Inf and [1] += complex sign-check failures.
 * Errors: argument codes, QMC_ERR_WORKSPACE, QMC_ERR_CUDA. */
int qmc_sums(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin, uint64_t i_end,
             void *workspace, size_t workspace_bytes, double *sums,
             unsigned long long *counters, void *stream);

/* qmc_sums without a workspace argument and without any allocation.  The paper has no
 * counterpart: it is for callers that cannot allocate device memory when they integrate
 * -- code running under CUDA-graph capture, latency- or signal-critical paths, hosts whose
 * device memory belongs to another allocator, or deployments that fix all device memory
 * in advance.  Same inputs, outputs and results as qmc_sums (bit-identical sums); the
 * per-tile partials live in a fixed device array of QMC_NOALLOC_SCRATCH_BYTES (8 MiB) that
 * every GPU loading the library holds until the process exits.
 *   - Problems whose partials need more than that (qmc_sums_workspace_bytes() >
 *     QMC_NOALLOC_SCRATCH_BYTES, e.g. real m = 32 beyond n ~ 1.1e9) are rejected with
 *     QMC_ERR_WORKSPACE before anything is launched.
 *   - The first call on a device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture.  The
 *     address is kept for the life of the process: after cudaDeviceReset() it is stale,
 *     so do not call this entry point again in that process.
 *   - Argument checks and their codes are those of qmc_sums, in the same order; only then
 *     is the size compared with the array.
 *   - All calls on a device share the array and it keeps the last call's contents; the
 *     kernel overwrites every partial it reads, so nothing has to be cleared first.  Calls
 *     that overlap on the GPU (unordered streams or threads) race on it: order them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine. */
int qmc_sums_noalloc(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin,
                     uint64_t i_end, double *sums, unsigned long long *counters, void *stream);

/* Shift reduction (Eq. (lattice) and Eq. (lattice-error)) from device sums laid out as
 * above over a lattice of size n: result (device) [4] = Qbar_re, sigma_re, Qbar_im,
 * sigma_im, and Q (device, may be NULL) [m] or [2m] = per-shift Q^(k) re (then im).
 * m >= 2.  Errors: QMC_ERR_ARG, QMC_ERR_M, QMC_ERR_CUDA. */
int qmc_finalize(const double *sums, uint64_t m, uint64_t n, int is_complex, double *result,
                 double *Q, void *stream);

/* Raw samples f(x_i) on one shifted lattice (App. A.2 evaluate()): out (device) [count]
 * (real) or [2*count] interleaved (complex), x_i = {i z/n + Delta} with shift (device)
 * [dim] 53-bit integers; no transform, no fit. */
int qmc_evaluate(const qmc_integrand *f, uint64_t n, const uint64_t *z, int dim,
                 const uint64_t *shift, uint64_t i_begin, uint64_t count, double *out,
                 void *stream);

/* Per-dimension histogram of |f| over all n points of one shifted lattice (the data pass
 * of the fit, Sec. 2.4): hist (device) [dim][bins] += |f(x_i)| at bin floor(x_ij * bins)
 * (clamped to bins-1); hist is zeroed first.  workspace (device) must hold
 * qmc_histogram_workspace_bytes(n, dim, bins) bytes (per-block partial histograms, summed
 * in block order: the result is deterministic).  dim * bins <= 20480. */
size_t qmc_histogram_workspace_bytes(uint64_t n, int dim, int bins);
int qmc_histogram(const qmc_integrand *f, uint64_t n, const uint64_t *z, int dim,
                  const uint64_t *shift, int bins, double *hist, void *workspace,
                  size_t workspace_bytes, void *stream);

/* ---- batches: many integrals in one launch -------------------------------------------- */

/* One integral of a batch: integrand and rule with device arrays (as for qmc_sums) and
 * its i-range.  All items of one batch share the integrand family and m (1 <= m <= 256);
 * dimension, n, z, shifts, transform, fit and coefficients may differ per item.  Families:
 * Genz 1-4, QMC_SECTOR, QMC_FEYNMAN. */
typedef struct {
    qmc_integrand f;
    qmc_rule rule;
    uint64_t i_begin, i_end;
} qmc_batch_item;

/* Launch shape: streams_per_block (block = streams_per_block * m threads, <= 256) and
 * points_per_stream (points per thread and tile).  0 selects the defaults of qmc_sums
 * (256/m streams, range-dependent tile length), with which every item's sums are
 * bit-identical to a qmc_sums call on that item. */
typedef struct {
    int streams_per_block;
    uint32_t points_per_stream;
} qmc_batch_config;

/* Device workspace for qmc_batch_sums (item descriptors, tile offsets, tile partials);
 * 0 when the batch is invalid. */
size_t qmc_batch_workspace_bytes(const qmc_batch_item *items, int count,
                                 const qmc_batch_config *cfg);

/* Per-shift sums of every item in one kernel launch, then one reduction launch and
 * (results != NULL) one finalize launch (Eq. (lattice), Eq. (lattice-error)).
 *   items: host array of count items.  sums (device) [count][4m]: item q's double-double
 *   sums at q*4m in the qmc_sums layout.  results (device, may be NULL) [count][4]:
 *   Qbar_re, sigma_re, Qbar_im, sigma_im (needs m >= 2).  counters (device, may be NULL)
 *   [count][2]: NaN/Inf samples and complex sign-check failures per item, added to.
 * Errors: argument codes of qmc_sums per item, QMC_ERR_ARG for mixed families or m,
 * QMC_ERR_WORKSPACE, QMC_ERR_CUDA. */
int qmc_batch_sums(const qmc_batch_item *items, int count, const qmc_batch_config *cfg,
                   void *workspace, size_t workspace_bytes, double *sums, double *results,
                   unsigned long long *counters, void *stream);

/* The same in two steps, for replaying a batch (e.g. from a captured CUDA graph):
 * qmc_batch_plan_create validates the items, uploads their descriptors into `workspace`
 * (stream-ordered, then synchronises `stream`) and returns a host handle; the items' device
 * arrays and the workspace must outlive the plan.  qmc_batch_plan_run enqueues only kernel
 * launches (batch kernel, reduction, optional finalize), so it can be captured.
 * qmc_batch_plan_destroy frees the handle (host memory). */
typedef struct qmc_batch_plan qmc_batch_plan;
int qmc_batch_plan_create(const qmc_batch_item *items, int count, const qmc_batch_config *cfg,
                          void *workspace, size_t workspace_bytes, void *stream,
                          qmc_batch_plan **out);
int qmc_batch_plan_run(const qmc_batch_plan *plan, double *sums, double *results,
                       unsigned long long *counters, void *stream);
void qmc_batch_plan_destroy(qmc_batch_plan *plan);

/* Chooses the launch shape for a batch by timing candidate configurations
 * (streams_per_block in {256/m, 128/m, 64/m} x points_per_stream in {16..512}) on a sample
 * of at most 256 items, each cut to the first max(2^16, 2^23 / items) points of its range
 * so that a candidate costs a bounded time (CUDA events on `stream`).  workspace and sums as for
 * qmc_batch_sums of the same items (the sample needs no more).  best receives the fastest
 * configuration.  Overwrites sums. */
int qmc_batch_autotune(const qmc_batch_item *items, int count, void *workspace,
                       size_t workspace_bytes, double *sums, void *stream,
                       qmc_batch_config *best);

/* ---- serving: continuous batching of adaptive integrations ---------------------------- */

/* A server owns a device memory pool of memory_budget bytes (one cudaMalloc at creation)
 * and runs at most max_slots requests at a time, all with m shifts (2..256) and the given
 * transform.  Requests are integrals with an error goal (epsrel, epsabs, the rule of the
 * adaptive mode, Sec. 3.3.1, errormode all) and an evaluation budget maxeval, starting
 * at get_next_n(minn).  Each qmc_server_step admits queued requests in arrival order
 * while memory and slots allow (reserving coefficients, shifts and the tile partials of
 * the largest tile count among the lattices up to the request's largest admissible
 * one; the count is not monotone in n), runs the admitted requests (all of them, or
 * those chosen within step_evaluations) on their current lattices in one batched launch
 * per integrand family, and then completes requests whose
 * goal is met or whose budget is spent, moving the others to larger table sizes.  A
 * request's result does not depend on the other requests: it equals qmc_integrate with
 * the same arguments as long as neither needs more shifts than m.
 * Families: as for batches.  The server is not thread-safe across steps of one server
 * from several threads (calls are serialised by a lock). */
enum { QMC_REQ_PENDING = 0, QMC_REQ_ACTIVE = 1, QMC_REQ_DONE = 2 };
typedef struct {
    size_t memory_budget;
    int max_slots;
    uint64_t m;
    qmc_transform transform;
    /* Evaluations one step may spend (0: every running request each step).  When set, a
     * step runs the running requests in order of their current lattice's cost divided by
     * one plus the steps they have waited (shortest first, aged so that none starves),
     * while the sum of their evaluations stays within the budget (at least one request
     * per step).  The choice changes when a request runs, never its numbers. */
    uint64_t step_evaluations;
} qmc_server_config;
typedef struct qmc_server qmc_server;

/* table: host, copied.  stream: the server's CUDA stream (NULL = default).  Errors:
 * QMC_ERR_ARG/M/TRANSFORM, QMC_ERR_WORKSPACE (budget below the fixed per-slot buffers),
 * QMC_ERR_CUDA, QMC_ERR_NO_DEVICE. */
int qmc_server_create(const qmc_genvec_table *table, const qmc_server_config *cfg,
                      void *stream, qmc_server **out);
void qmc_server_destroy(qmc_server *s);

/* Queue a request; f has host arrays (copied).  *id receives its identifier. */
int qmc_server_submit(qmc_server *s, const qmc_integrand *f, double epsrel, double epsabs,
                      uint64_t minn, uint64_t maxeval, uint64_t seed, uint64_t *id);

/* One scheduling round (synchronises the server's stream); *completed (may be NULL)
 * receives the number of requests that finished in it. */
int qmc_server_step(qmc_server *s, int *completed);

/* State of a request (QMC_REQ_*), its result so far (final once done) and, when done, the
 * seconds from submission to completion.  Returns the request's status once done
 * (QMC_OK, QMC_ERR_NONFINITE, QMC_ERR_N when no table size fits), QMC_OK before. */
int qmc_server_status(qmc_server *s, uint64_t id, int *state, qmc_result *result,
                      double *latency_s);

/* Queued and running requests and the free bytes of the pool. */
int qmc_server_counts(qmc_server *s, int *pending, int *active, size_t *free_bytes);

/* Identifiers of the requests that finished since the previous call, in completion order:
 * up to cap of them are written to ids (host, caller-owned), *count receives how many;
 * the rest stay queued for the next call.  A serving loop reads these after each step
 * instead of polling every open request.  Errors: QMC_ERR_ARG (s, ids or count NULL,
 * cap < 0). */
int qmc_server_completed(qmc_server *s, uint64_t *ids, int cap, int *count);

/* ---- tile-aligned sharding --------------------------------------------------------- */

/* qmc_sums cuts an i-range into tiles that depend only on the range's length and m (one
 * shift group, m <= 256) and folds the per-tile partial sums in tile order in double-double.
 * A range split at tile boundaries, its tiles' partials gathered in tile order and folded
 * by qmc_reduce_tiles gives the per-shift sums of qmc_sums bit for bit (Sec. 2.1: the
 * points of one rule are independent, so shards need no other exchange). */

/* Number of tiles of the decomposition of an i-range of range_len points with m shifts,
 * and the points per tile (the last tile may be shorter).  Errors: QMC_ERR_ARG,
 * QMC_ERR_M (m outside 1..256). */
int qmc_sums_tile_count(uint64_t range_len, uint64_t m, uint64_t *tiles,
                        uint64_t *points_per_tile);

/* Per-tile partial sums of tiles [tile_begin, tile_end) of the decomposition of
 * [i_begin, i_end): partials[t][k] = (sum, compensation) of shift k over tile
 * tile_begin + t, for t < T = tile_end - tile_begin, then (complex family) the same T x m
 * block for the imaginary part.  partials: device, 2 m T doubles (4 m T complex), written
 * entirely.  counters: as qmc_sums.  The values equal those qmc_sums forms for the same
 * tiles.  Errors: as qmc_sums; QMC_ERR_M (m > 256); QMC_ERR_RANGE (empty or out-of-range
 * tile range). */
int qmc_sums_tiles(const qmc_integrand *f, const qmc_rule *rule, uint64_t i_begin,
                   uint64_t i_end, uint64_t tile_begin, uint64_t tile_end, double *partials,
                   unsigned long long *counters, void *stream);

/* The fold qmc_sums applies to its tiles: sums[2k], sums[2k+1] = double-double sum of shift
 * k's partials over the tiles in order (complex: the imaginary part at sums[2m + 2k..]).
 * partials: device, the layout of qmc_sums_tiles for `tiles` tiles.  sums: device, 2 m
 * (4 m complex) doubles.  Errors: QMC_ERR_ARG, QMC_ERR_M, QMC_ERR_CUDA. */
int qmc_reduce_tiles(const double *partials, uint64_t tiles, uint64_t m, int is_complex,
                     double *sums, void *stream);

/* Merge of per-shift sums computed on separate i-ranges of one rule (Sec. 2.1: the sum
 * over a lattice is the sum of its parts' sums).  parts (host) holds nparts arrays of len
 * doubles back to back, each in the qmc_sums layout of (hi, lo) double-double pairs (len
 * even: 2m real, 4m complex); out (host, len doubles, may alias parts' first array)
 * receives their double-double sum, pairs added in part order with TwoSum and a Fast2Sum
 * renormalisation: deterministic, equal to the whole range's sums within the rounding of
 * the double-double format.  No device work.  Errors: QMC_ERR_ARG (NULL, nparts < 1, len
 * odd or < 2). */
int qmc_merge_sums(const double *parts, uint64_t nparts, uint64_t len, double *out);

/* ---- generating vectors: fast CBC on the device -------------------------------------- */

/* Component-by-component construction (App. A.3 of the paper; the fast algorithm of
 * Nuyens and Cools) of a rank-1 lattice generating vector for a prime number of points n,
 * in the Korobov space of smoothness alpha = 2 with kernel omega(x) = 2 pi^2 (x^2 - x + 1/6),
 * product weights gamma and parameter beta: z_1 = 1, then each z_j in 1..(n-1)/2 minimises
 *   e^2(z_1..z_j) = -1 + (1/n) sum_{k<n} prod_{l<=j} (beta + gamma omega({k z_l / n})).
 * The candidate sums are cyclic convolutions over the multiplicative group of n, folded to
 * length (n-1)/2 and evaluated with cuFFT (FP64); sums within 1e-14 omega(0) sum_k p(k) of
 * the minimum are ties, won by the smallest z.  The shipped tables use gamma = 1/s_max,
 * beta = 1.
 * z_out: host, s entries.  e2_out: host, s entries (the squared worst-case error after each
 * component), or NULL.  stream: NULL = default.  Device memory (about qmc_cbc_device_bytes(n)
 * plus cuFFT's work area) is allocated here and freed before returning.
 * Errors: QMC_ERR_ARG (n not a prime in [5, 2^53), s outside 1..1024, beta <= 0,
 * gamma < 0), QMC_ERR_CUDA (allocation, FFT or launch failure), QMC_ERR_NO_DEVICE. */
size_t qmc_cbc_device_bytes(uint64_t n);
int qmc_cbc_korobov(uint64_t n, int s, double gamma, double beta, uint64_t *z_out,
                    double *e2_out, void *stream);

/* ---- measurement: unit throughput probes ------------------------------------------- */

/* The paper has no counterpart: these measure the two arithmetic units the lattice sums
 * run on, for the roofline of qmc_sums on the device at hand.  QMC_PROBE_FP64_FMA runs
 * chains of FP64 fused multiply-adds; QMC_PROBE_INT_MULHI runs chains of the truncated
 * 64-bit high product the kernel's fixed-point transforms and Genz forms use (one
 * 32 x 32 -> 64-bit multiply and two 32-bit high multiplies).  One launch of
 * SMs x (resident blocks per SM) blocks of 256 threads, each thread running trips x 32
 * operations on 8 independent chains; *ops_out (host) receives the operations launched
 * (FMAs, or 32-bit multiplies).  sink: device, one double (written only in a case that
 * does not occur; it keeps the chains live).  The call only enqueues: time it with events
 * on `stream`.  Errors: QMC_ERR_ARG (unknown unit, NULL, trips < 1), QMC_ERR_NO_DEVICE,
 * QMC_ERR_CUDA. */
enum { QMC_PROBE_FP64_FMA = 1, QMC_PROBE_INT_MULHI = 2 };
int qmc_probe_units(int unit, uint32_t trips, double *sink, double *ops_out, void *stream);

/* ---- host entry points -------------------------------------------------------------- */

/* Fit the PolySingular map (Eq. (ISfit), |a2|, |a3| form of App. A.5) per dimension to
 * the inverse CDF taken from a host histogram hist[dim][bins]: data pairs
 * (CDF(b/bins), b/bins) for every stepsize-th edge, Levenberg-Marquardt with
 * a0 >= 1.001, a1 <= -0.001.  params (host) [dim][6]. */
int qmc_fit_polysingular(const double *hist, int dim, int bins, const qmc_fit_opts *opts,
                         double *params);

/* Integrate with host buffers (the paper's integrate(), App. A.2).
 *   f: host arrays.  table: host.  m: shifts (the paper's minm).
 *   opts == NULL: fixed lattice (Sec. 3.3.2, Case 2): n = get_next_n(n_or_minn), one pass.
 *   opts != NULL: adaptive (Sec. 3.3.1, Case 1): start at get_next_n(n_or_minn); while the
 *     error goal (|E - I| <= max(epsabs, epsrel |I|), per component or by errormode) fails
 *     and evaluations stay below maxeval, discard the result and take a larger table size;
 *     past the largest size, double m.  The last result is returned.
 *   fit: NULL or enabled == 0 for no variance reduction; else fit on a lattice of
 *     >= evaluateminn points first and integrate the fitted, then periodized, integrand.
 *   Shifts come from qmc_make_shifts(seed, m, dim).  Device memory is library-owned and
 *   reused across calls on the same device.
 * Returns QMC_OK, an error code, or QMC_ERR_NONFINITE when samples were NaN/Inf (out is
 * filled, out->nonfinite counts them). */
int qmc_integrate(const qmc_integrand *f, const qmc_genvec_table *table, uint64_t n_or_minn,
                  uint64_t m, qmc_transform transform, const qmc_fit_opts *fit, uint64_t seed,
                  const qmc_options *opts, void *stream, qmc_result *out);

#ifdef __cplusplus
}
#endif
#endif /* QMC_GB300_H */
