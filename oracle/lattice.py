"""Lattice sizes and component-by-component (CBC) generating vectors -- oracle side.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain Python/NumPy; shares no code with
the CUDA path.

* Lattice sizes (App. A.1, field ``generatingvectors``; App. A.3): the next prime strictly
  above ``1020 * 1.1**i`` (computed in double, then floored) for ``i = 0..152``, plus
  ``2**31 - 1``.
* ``get_next_n`` (App. A.2): the smallest available size ``>= preferred``.
* CBC (Sec. 2.2; App. A.3): Korobov space with smoothness alpha = 2 in Nuyens' notation,
  kernel ``omega(x) = 2 pi^2 (x^2 - x + 1/6)``, product weights ``gamma_j = 1/s`` and
  ``beta_j = 1``.  Component j minimises the shift-averaged squared worst-case error
  ``e^2(z_1..z_j) = -1 + (1/n) sum_{k<n} prod_{l<=j} (beta + gamma omega({k z_l / n}))``
  over ``z_j`` in ``1..(n-1)/2`` (``z`` and ``n - z`` give the same error), taking the
  smallest minimiser; ``z_1 = 1``.  Only the candidate-dependent sum
  ``T(z) = sum_k p(k) omega({k z / n})`` is compared (no ``-1 + ...`` cancellation), and
  sums within ``TIE_RTOL * omega(0) * sum_k p(k)`` of the minimum count as ties.
  - ``cbc_naive``: the definition evaluated for every candidate, O(s n^2).
  - ``cbc_fast``: the same minimisation with the candidate sums computed as one cyclic
    convolution of length ``n - 1`` over the multiplicative group of ``Z_n`` (generator
    ``g``; Nuyens & Cools 2006), by FFT.  Prime ``n`` only.
"""
from __future__ import annotations

import math

import numpy as np

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (the first 12 prime bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def next_prime_above(x: int) -> int:
    p = x + 1
    while not is_prime(p):
        p += 1
    return p


def lattice_sizes(imax: int = 152, include_int_max: bool = True) -> list[int]:
    sizes = {next_prime_above(math.floor(1020.0 * 1.1 ** i)) for i in range(imax + 1)}
    if include_int_max:
        sizes.add(2 ** 31 - 1)
    return sorted(sizes)


def get_next_n(sizes, preferred: int) -> int:
    for n in sorted(sizes):
        if n >= preferred:
            return n
    raise ValueError(f"no lattice size >= {preferred}")


def omega(x):
    """Korobov-space kernel for alpha = 2: 2 pi^2 B_2(x) = 2 pi^2 (x^2 - x + 1/6)."""
    return 2.0 * np.pi ** 2 * (x * x - x + 1.0 / 6.0)


def worst_case_error_sq(n: int, z, s_weights: int | None = None, beta: float = 1.0) -> float:
    """e^2(z) by its definition: -1 + (1/n) sum_k prod_j (beta + gamma omega({k z_j / n})).
    ``gamma = 1/s_weights`` (default: 1/len(z))."""
    z = [int(v) for v in z]
    s = len(z) if s_weights is None else s_weights
    gamma = 1.0 / s
    k = np.arange(n, dtype=np.int64)
    prod = np.ones(n)
    for zj in z:
        frac = ((k * zj) % n).astype(np.float64) / n
        prod *= beta + gamma * omega(frac)
    return float(-1.0 + prod.sum() / n)


def cbc_naive(n: int, s: int, beta: float = 1.0, gamma: float | None = None):
    """Return (z, e2 per component) by evaluating the definition for every candidate."""
    gamma = 1.0 / s if gamma is None else gamma
    k = np.arange(n, dtype=np.int64)
    cand = np.arange(1, (n - 1) // 2 + 1, dtype=np.int64)
    cand = cand[np.gcd(cand, n) == 1]
    p = np.ones(n)
    z = [1]
    p *= beta + gamma * omega(((k * 1) % n) / n)
    e2 = [float(-1.0 + p.sum() / n)]
    for _ in range(1, s):
        # rows: candidates, cols: k
        fr = (np.outer(cand, k) % n).astype(np.float64) / n
        T = (p[None, :] * omega(fr)).sum(axis=1)
        best = _pick(T, cand, omega(0.0) * p.sum())
        zj = int(cand[best])
        z.append(zj)
        e2.append(float(-1.0 + (beta * p.sum() + gamma * T[best]) / n))
        p *= beta + gamma * omega(((k * zj) % n) / n)
    return z, e2


TIE_RTOL = 1e-14


def _pick(T: np.ndarray, cand: np.ndarray, scale: float) -> int:
    """Index of the smallest candidate z among those whose candidate sum
    T(z) = sum_k p(k) omega({k z / n}) lies within TIE_RTOL * scale of the minimum, where
    scale = omega(0) sum_k p(k) bounds the size of the summed terms.  Symmetric lattices
    (e.g. z and z^-1 mod n in two dimensions) give mathematically equal sums that differ
    in the last bits, so exact float equality would let rounding pick the winner; sums
    carry cancellation (omega has mean zero), hence the absolute scale."""
    tmin = T.min()
    near = T <= tmin + TIE_RTOL * scale
    idx = np.nonzero(near)[0]
    return int(idx[np.argmin(cand[idx])])


def _prime_factors(m: int) -> list[int]:
    out, q = [], 2
    while q * q <= m:
        if m % q == 0:
            out.append(q)
            while m % q == 0:
                m //= q
        q += 1
    if m > 1:
        out.append(m)
    return out


def primitive_root(n: int) -> int:
    """Smallest generator of the multiplicative group mod prime n."""
    fac = _prime_factors(n - 1)
    g = 2
    while True:
        if all(pow(g, (n - 1) // q, n) != 1 for q in fac):
            return g
        g += 1


def cbc_fast(n: int, s: int, beta: float = 1.0, gamma: float | None = None, workers: int = -1,
             chunk: int = 1 << 24):
    """CBC for prime n via FFT convolution over the cyclic group Z_n^* (Nuyens-Cools).

    With z = g^a and k = g^-b, {k z / n} depends on a - b only, so the candidate sums
    T(g^a) = sum_{k=1}^{n-1} p(k) omega({k g^a / n}) form a cyclic convolution.  Because
    g^((n-1)/2) = -1 (mod n), p(k) = p(n-k) and omega(x) = omega(1-x), the convolution
    folds to length (n-1)/2: T(g^a) = 2 sum_{b<(n-1)/2} p(g^-b) omega({g^(a-b)/n}).
    The k = 0 term (omega(0) for every candidate) is added separately.  Only
    p(k), k = 0..(n-1)/2, is stored.
    """
    import scipy.fft as sfft

    if not is_prime(n) or n < 5:
        raise ValueError("cbc_fast needs a prime n >= 5")
    gamma = 1.0 / s if gamma is None else gamma
    H = (n - 1) // 2
    g = primitive_root(n)
    gp = _power_table(g, n, H)                      # g^c mod n, c < H
    # Cyclic convolution of length H computed as a linear one: with W2 = [W, W],
    # (P * W2)[a + H] = sum_b P[b] W[(a - b) mod H] for a < H, and a transform length
    # L >= 2H - 1 keeps indices H..2H-1 free of wrap-around.  L is 5-smooth (fast FFT).
    L_fft = sfft.next_fast_len(2 * H, real=True)
    W = omega(gp.astype(np.float64) / n)
    FW = sfft.rfft(np.concatenate([W, W]), n=L_fft, workers=workers)
    del W
    # representatives of +-g^-b: g^-b = g^(2H - b); fold to min(x, n - x)
    ginv = np.empty(H, dtype=np.int64)
    ginv[0] = 1
    if H > 1:
        # g^(2H-b) = -g^(H-b) mod n
        ginv[1:] = n - gp[H - np.arange(1, H)]
    np.minimum(ginv, n - ginv, out=ginv)
    crep = np.minimum(gp, n - gp)                    # candidate representatives <= (n-1)/2

    ph = np.ones(H + 1)                              # p(k) for k = 0..H

    def update(zj):
        for lo in range(0, H + 1, chunk):
            k = np.arange(lo, min(H + 1, lo + chunk), dtype=np.int64)
            ph[lo:lo + k.size] *= beta + gamma * omega(((k * zj) % n).astype(np.float64) / n)

    def total():                                     # sum_{k<n} p(k) = p(0) + 2 sum_{1..H} p(k)
        return ph[0] + 2.0 * ph[1:].sum()

    update(1)
    z = [1]
    e2 = [float(-1.0 + total() / n)]
    w0 = omega(0.0)
    for _ in range(1, s):
        P = ph[ginv]
        T = 2.0 * sfft.irfft(sfft.rfft(P, n=L_fft, workers=workers) * FW, n=L_fft,
                             workers=workers)[H:2 * H]
        del P
        T += ph[0] * w0
        best = _pick(T, crep, w0 * total())
        zj = int(crep[best])
        z.append(zj)
        e2.append(float(-1.0 + (beta * total() + gamma * T[best]) / n))
        del T
        update(zj)
    return z, e2


def _power_table(g: int, n: int, N: int) -> np.ndarray:
    """g^c mod n for c = 0..N-1 with exact int64 arithmetic, built by doubling blocks:
    gp[B:2B] = gp[0:B] * g^B mod n (products stay below 2^63 for n < 2^31)."""
    if n >= (1 << 31):
        raise ValueError("power table needs n < 2^31")
    gp = np.empty(N, dtype=np.int64)
    gp[0] = 1
    filled = 1
    while filled < N:
        take = min(filled, N - filled)
        mult = pow(g, filled, n)
        gp[filled:filled + take] = (gp[:take] * mult) % n
        filled += take
    return gp
