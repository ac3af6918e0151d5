// qmc_cbc.cu -- fast component-by-component construction of rank-1 lattice generating
// vectors on the GPU (App. A.3 table of generating vectors; the fast CBC of Nuyens and
// Cools, with cuFFT for the cyclic convolutions).
//
// Korobov space of smoothness alpha = 2 with product weights: the squared worst-case error
// of z = (z_1..z_s) on n points is
//     e^2(z) = -1 + (1/n) sum_{k=0}^{n-1} prod_{l<=s} (beta + gamma omega({k z_l / n})),
//     omega(x) = 2 pi^2 (x^2 - x + 1/6),
// and CBC fixes z_1 = 1, then picks each z_j in 1..n-1 minimising e^2 given z_1..z_(j-1).
// Only T(z) = sum_k p(k) omega({k z / n}) depends on the candidate, with p(k) the product of
// the factors of the earlier components.  For prime n and a primitive root g, z = g^a and
// k = g^-b give {k z / n} = {g^(a-b) / n}: T is a cyclic convolution over the group of
// units.  Because g^((n-1)/2) = -1, omega(x) = omega(1 - x) and p(k) = p(n - k), it folds to
// length H = (n-1)/2:
//     T(g^a) = p(0) omega(0) + 2 sum_{b<H} p(g^-b) omega({g^(a-b) / n}),   a < H,
// and the candidates are the representatives min(g^a, n - g^a) <= H.  The cyclic
// convolution of length H is taken from a linear one: with W2 = (W, W) of length 2H and
// P zero-padded, (P * W2)[a + H] = sum_b P[b] W[(a - b) mod H] for a < H, and any transform
// length L >= 2H keeps those indices free of wrap-around; L is chosen 7-smooth so that
// cuFFT runs its mixed-radix kernels whatever the factors of H.  Each component costs one
// real-to-complex FFT of length L, a pointwise product with the (once transformed) W2, one
// complex-to-real FFT, a minimum search and an update of p.
//
// Ties: sums within 1e-14 omega(0) sum_k p(k) of the minimum are ties, and the smallest
// candidate wins (the same reading as the CPU construction that wrote the shipped table).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "qmc_gb300.h"
#include "qmc_hostutil.h"

namespace qmc {
namespace {

constexpr double kTwoPi2 = 19.739208802178717237668981999752;   // 2 pi^2
constexpr double kTieRtol = 1e-14;
constexpr int kCbcThreads = 256;

__host__ __device__ inline double omega_k(double x) { return kTwoPi2 * (x * x - x + 1.0 / 6.0); }

// a b mod n for a, b < n < 2^53: the quotient estimated in FP64 is within 2 of the exact
// one, and the remainder is corrected exactly in 64-bit two's complement.
__device__ __forceinline__ uint64_t mulmod_dev(uint64_t a, uint64_t b, uint64_t n) {
    const uint64_t lo = a * b;
    const double qd = floor((double)a * (double)b / (double)n);
    const uint64_t q = qd <= 0.0 ? 0ull : (uint64_t)qd;
    long long r = (long long)(lo - q * n);   // the exact a b - q n, within (-2n, 3n)
#pragma unroll 1
    for (int it = 0; it < 4 && r < 0; ++it) r += (long long)n;
#pragma unroll 1
    for (int it = 0; it < 4 && r >= (long long)n; ++it) r -= (long long)n;
    return (uint64_t)r;
}

__device__ __forceinline__ uint64_t powmod_dev(uint64_t g, uint64_t e, uint64_t n) {
    uint64_t r = 1 % n, b = g % n;
#pragma unroll 1
    while (e) {
        if (e & 1) r = mulmod_dev(r, b, n);
        b = mulmod_dev(b, b, n);
        e >>= 1;
    }
    return r;
}

inline uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t n) {
    return (uint64_t)((unsigned __int128)a * b % n);
}
inline uint64_t powmod_host(uint64_t g, uint64_t e, uint64_t n) {
    uint64_t r = 1 % n, b = g % n;
    while (e) {
        if (e & 1) r = mulmod_host(r, b, n);
        b = mulmod_host(b, b, n);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for 64-bit integers (the first 12 primes as bases).
bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n % p == 0) return n == p;
    }
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++r;
    }
    for (uint64_t a : small) {
        uint64_t x = powmod_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

// Smallest primitive root of the prime n: g is one when g^((n-1)/q) != 1 for every prime
// factor q of n - 1.
uint64_t primitive_root(uint64_t n) {
    std::vector<uint64_t> qs;
    uint64_t m = n - 1;
    for (uint64_t q = 2; q * q <= m; ++q) {
        if (m % q == 0) {
            qs.push_back(q);
            while (m % q == 0) m /= q;
        }
    }
    if (m > 1) qs.push_back(m);
    for (uint64_t g = 2; g < n; ++g) {
        bool ok = true;
        for (uint64_t q : qs) {
            if (powmod_host(g, (n - 1) / q, n) == 1) {
                ok = false;
                break;
            }
        }
        if (ok) return g;
    }
    return 0;
}

// gp[c] = g^c mod n for c < H; thread t fills [t B, t B + B).
__global__ void cbc_powers_kernel(uint64_t g, uint64_t n, uint64_t H, uint64_t B, uint64_t *gp) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t c0 = t * B;
    if (c0 >= H) return;
    uint64_t x = powmod_dev(g, c0, n);
    const uint64_t c1 = c0 + B < H ? c0 + B : H;
#pragma unroll 1
    for (uint64_t c = c0; c < c1; ++c) {
        gp[c] = x;
        x = mulmod_dev(x, g, n);
    }
}

// w[c] = w[c + H] = omega(g^c / n) for c < H, zero on [2H, L)
__global__ void cbc_omega_kernel(const uint64_t *gp, uint64_t H, uint64_t L, uint64_t n, double *w) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < L;
         c += (uint64_t)gridDim.x * blockDim.x) {
        if (c < 2 * H) {
            const uint64_t c0 = c < H ? c : c - H;
            w[c] = omega_k((double)gp[c0] / (double)n);
        } else {
            w[c] = 0.0;
        }
    }
}

// p[k] *= beta + gamma omega({k z / n}) for k <= H (p[k] = 1 first when init).
__global__ void cbc_update_kernel(double *p, uint64_t H, uint64_t n, uint64_t z, double beta,
                                  double gamma, int init) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= H;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const double f = fma(gamma, omega_k((double)mulmod_dev(k, z, n) / (double)n), beta);
        p[k] = init ? f : p[k] * f;
    }
}

// P[b] = p(min(g^-b, n - g^-b)) for b < H (g^-b = n - g^(H - b) for b >= 1, g^0 = 1), zero
// on [H, L).
__global__ void cbc_gather_kernel(const uint64_t *gp, const double *p, uint64_t H, uint64_t L,
                                  uint64_t n, double *P) {
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < L;
         b += (uint64_t)gridDim.x * blockDim.x) {
        if (b >= H) {
            P[b] = 0.0;
            continue;
        }
        uint64_t k = 1;
        if (b) {
            const uint64_t v = gp[H - b];
            k = v < n - v ? v : n - v;
        }
        P[b] = p[k];
    }
}

__global__ void cbc_pointwise_kernel(cufftDoubleComplex *a, const cufftDoubleComplex *b,
                                     uint64_t m) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const cufftDoubleComplex x = a[i], y = b[i];
        a[i] = make_cuDoubleComplex(fma(x.x, y.x, -x.y * y.y), fma(x.x, y.y, x.y * y.x));
    }
}

// Block sums of p[1..H] (fixed order within a block, blocks in order on the host).
__global__ void cbc_sum_kernel(const double *p, uint64_t H, uint64_t per_block, double *out) {
    __shared__ double s[kCbcThreads];
    const uint64_t lo = 1 + (uint64_t)blockIdx.x * per_block;
    const uint64_t hi = lo + per_block < H + 1 ? lo + per_block : H + 1;
    double acc = 0.0;
    for (uint64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) acc += p[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kCbcThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// Per-block minimum of T[a] = scale raw[a] + off over a < H.
__global__ void cbc_min_kernel(const double *raw, uint64_t H, double scale, double off,
                               uint64_t per_block, double *out) {
    __shared__ double s[kCbcThreads];
    const uint64_t lo = (uint64_t)blockIdx.x * per_block;
    const uint64_t hi = lo + per_block < H ? lo + per_block : H;
    double m = INFINITY;
    for (uint64_t a = lo + threadIdx.x; a < hi; a += blockDim.x) m = fmin(m, fma(scale, raw[a], off));
    s[threadIdx.x] = m;
    __syncthreads();
    for (int w = kCbcThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// Per block: the smallest representative min(g^a, n - g^a) among a with T[a] <= bound,
// and its T (representative n when none).
__global__ void cbc_pick_kernel(const double *raw, const uint64_t *gp, uint64_t H, uint64_t n,
                                double scale, double off, double bound, uint64_t per_block,
                                uint64_t *rep_out, double *t_out) {
    __shared__ uint64_t sr[kCbcThreads];
    __shared__ double st[kCbcThreads];
    const uint64_t lo = (uint64_t)blockIdx.x * per_block;
    const uint64_t hi = lo + per_block < H ? lo + per_block : H;
    uint64_t best = n;
    double bt = INFINITY;
    for (uint64_t a = lo + threadIdx.x; a < hi; a += blockDim.x) {
        const double t = fma(scale, raw[a], off);
        if (t <= bound) {
            const uint64_t v = gp[a];
            const uint64_t rep = v < n - v ? v : n - v;
            if (rep < best) {
                best = rep;
                bt = t;
            }
        }
    }
    sr[threadIdx.x] = best;
    st[threadIdx.x] = bt;
    __syncthreads();
    for (int w = kCbcThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w && sr[threadIdx.x + w] < sr[threadIdx.x]) {
            sr[threadIdx.x] = sr[threadIdx.x + w];
            st[threadIdx.x] = st[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rep_out[blockIdx.x] = sr[0];
        t_out[blockIdx.x] = st[0];
    }
}

struct DeviceBuffers {
    std::vector<void *> ptrs;
    ~DeviceBuffers() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    bool alloc(T **p, size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return false;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return true;
    }
};

struct Plans {
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    ~Plans() {
        if (have_fwd) cufftDestroy(fwd);
        if (have_inv) cufftDestroy(inv);
    }
};

// Smallest 2^a 3^b 5^c 7^d >= x.
uint64_t smooth_at_least(uint64_t x) {
    uint64_t best = ~0ull;
    for (uint64_t p7 = 1; p7 < 2 * x; p7 *= 7)
        for (uint64_t p5 = p7; p5 < 2 * x; p5 *= 5)
            for (uint64_t p3 = p5; p3 < 2 * x; p3 *= 3) {
                uint64_t v = p3;
                while (v < x) v *= 2;
                if (v < best) best = v;
            }
    return best;
}

unsigned grid_for(uint64_t work) {
    const uint64_t g = (work + kCbcThreads - 1) / kCbcThreads;
    return (unsigned)(g < 152ull * 64 ? (g ? g : 1) : 152ull * 64);
}

}  // namespace
}  // namespace qmc

using namespace qmc;

extern "C" size_t qmc_cbc_device_bytes(uint64_t n) {
    if (n < 5) return 0;
    const uint64_t H = (n - 1) / 2;
    const uint64_t L = smooth_at_least(2 * H);
    // gp (8 H), p (8 (H + 1)), P/T (8 L), FP and FW (16 (L/2 + 1) each)
    return (size_t)(8 * H + 8 * (H + 1) + 8 * L + 32 * (L / 2 + 1));
}

extern "C" int qmc_cbc_korobov(uint64_t n, int s, double gamma, double beta, uint64_t *z_out,
                               double *e2_out, void *stream) {
    if (!z_out || s < 1 || s > 1024 || n < 5 || n >= (1ull << 53) || !(beta > 0.0) ||
        !(gamma >= 0.0) || !is_prime_u64(n))
        return QMC_ERR_ARG;
    if (const int e = host::device_ok()) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t H = (n - 1) / 2;
    const uint64_t L = smooth_at_least(2 * H);   // transform length
    const uint64_t nc = L / 2 + 1;               // complex outputs of a real FFT of length L
    const uint64_t g = primitive_root(n);
    if (!g) return QMC_ERR_ARG;

    DeviceBuffers buf;
    uint64_t *gp = nullptr;
    double *p = nullptr, *P = nullptr, *part = nullptr, *tpart = nullptr;
    uint64_t *rpart = nullptr;
    cufftDoubleComplex *FP = nullptr, *FW = nullptr;
    const unsigned nblk = 152 * 8;
    if (!buf.alloc(&gp, H) || !buf.alloc(&p, H + 1) || !buf.alloc(&P, L) || !buf.alloc(&FP, nc) ||
        !buf.alloc(&FW, nc) || !buf.alloc(&part, nblk) || !buf.alloc(&tpart, nblk) ||
        !buf.alloc(&rpart, nblk))
        return QMC_ERR_CUDA;

    Plans plans;
    long long len = (long long)L;
    size_t work = 0;
    if (cufftCreate(&plans.fwd) != CUFFT_SUCCESS) return QMC_ERR_CUDA;
    plans.have_fwd = true;
    if (cufftCreate(&plans.inv) != CUFFT_SUCCESS) return QMC_ERR_CUDA;
    plans.have_inv = true;
    if (cufftMakePlanMany64(plans.fwd, 1, &len, nullptr, 1, 0, nullptr, 1, 0, CUFFT_D2Z, 1, &work) !=
            CUFFT_SUCCESS ||
        cufftMakePlanMany64(plans.inv, 1, &len, nullptr, 1, 0, nullptr, 1, 0, CUFFT_Z2D, 1, &work) !=
            CUFFT_SUCCESS ||
        cufftSetStream(plans.fwd, st) != CUFFT_SUCCESS || cufftSetStream(plans.inv, st) != CUFFT_SUCCESS)
        return QMC_ERR_CUDA;

    // powers of g, the transformed omega sequence (P is scratch here)
    const uint64_t B = 64;
    const uint64_t nthr = (H + B - 1) / B;
    cbc_powers_kernel<<<(unsigned)((nthr + kCbcThreads - 1) / kCbcThreads), kCbcThreads, 0, st>>>(g, n, H, B, gp);
    cbc_omega_kernel<<<grid_for(L), kCbcThreads, 0, st>>>(gp, H, L, n, P);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    if (cufftExecD2Z(plans.fwd, P, FW) != CUFFT_SUCCESS) return QMC_ERR_CUDA;

    // component 1: z_1 = 1
    cbc_update_kernel<<<grid_for(H + 1), kCbcThreads, 0, st>>>(p, H, n, 1, beta, gamma, 1);
    const uint64_t per_sum = (H + nblk - 1) / nblk;
    const uint64_t per_min = (H + nblk - 1) / nblk;
    std::vector<double> hpart(nblk), htp(nblk);
    std::vector<uint64_t> hrp(nblk);

    auto total = [&](double &tot) -> bool {
        double p0 = 0.0;
        cbc_sum_kernel<<<nblk, kCbcThreads, 0, st>>>(p, H, per_sum, part);
        if (cudaMemcpyAsync(hpart.data(), part, nblk * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(&p0, p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return false;
        double acc = 0.0;
        for (unsigned b = 0; b < nblk; ++b) acc += hpart[b];
        tot = p0 + 2.0 * acc;
        return true;
    };
    double tot = 0.0;
    if (!total(tot)) return QMC_ERR_CUDA;
    z_out[0] = 1;
    if (e2_out) e2_out[0] = -1.0 + tot / (double)n;
    const double w0 = omega_k(0.0);

    for (int j = 1; j < s; ++j) {
        double p0 = 0.0;
        if (cudaMemcpyAsync(&p0, p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return QMC_ERR_CUDA;
        cbc_gather_kernel<<<grid_for(L), kCbcThreads, 0, st>>>(gp, p, H, L, n, P);
        if (cufftExecD2Z(plans.fwd, P, FP) != CUFFT_SUCCESS) return QMC_ERR_CUDA;
        cbc_pointwise_kernel<<<grid_for(nc), kCbcThreads, 0, st>>>(FP, FW, nc);
        if (cufftExecZ2D(plans.inv, FP, P) != CUFFT_SUCCESS) return QMC_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return QMC_ERR_CUDA;
        // T[a] = 2 raw[a + H] / L + p(0) omega(0)  (the inverse transform is unnormalised)
        const double scale = 2.0 / (double)L, off = p0 * w0;
        const double *raw = P + H;
        cbc_min_kernel<<<nblk, kCbcThreads, 0, st>>>(raw, H, scale, off, per_min, part);
        if (cudaMemcpyAsync(hpart.data(), part, nblk * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QMC_ERR_CUDA;
        double tmin = INFINITY;
        for (unsigned b = 0; b < nblk; ++b) tmin = std::fmin(tmin, hpart[b]);
        const double bound = tmin + kTieRtol * w0 * tot;
        cbc_pick_kernel<<<nblk, kCbcThreads, 0, st>>>(raw, gp, H, n, scale, off, bound, per_min, rpart,
                                                      tpart);
        if (cudaMemcpyAsync(hrp.data(), rpart, nblk * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(htp.data(), tpart, nblk * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QMC_ERR_CUDA;
        uint64_t zj = n;
        double tj = 0.0;
        for (unsigned b = 0; b < nblk; ++b)
            if (hrp[b] < zj) {
                zj = hrp[b];
                tj = htp[b];
            }
        if (zj >= n) return QMC_ERR_CUDA;   // non-finite sums
        z_out[j] = zj;
        if (e2_out) e2_out[j] = -1.0 + (beta * tot + gamma * tj) / (double)n;
        cbc_update_kernel<<<grid_for(H + 1), kCbcThreads, 0, st>>>(p, H, n, zj, beta, gamma, 0);
        if (!total(tot)) return QMC_ERR_CUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}
