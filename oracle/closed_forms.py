"""Exact values that pin the oracle -- test infrastructure (see oracle/__init__.py).

* Genz integrals (Sec. 5.2, table of test functions) in closed form, evaluated with
  mpmath at 50 digits.
* The minimal example of Sec. 3.2: int x0 x1 x2 = 1/8.
* The lattice character sum: for a rank-1 lattice with shift Delta,
  (1/n) sum_i exp(2 pi i h.({i z/n} + Delta)) = exp(2 pi i h.Delta) if h.z = 0 (mod n),
  else 0.  Expanding prod_j (1 + a_j cos(2 pi (h_j x_j + theta_j))) into Fourier modes
  gives the exact lattice-rule value of that product (untransformed).
* Korobov weights as the explicit polynomials obtained by integrating
  C u^r (1-u)^r by hand, and the Sidi<1>, Sidi<2> maps in closed form.
"""
from __future__ import annotations

import itertools
import math

import mpmath as mp

mp.mp.dps = 50


def genz_exact(family: int, c, w) -> float:
    c = [mp.mpf(float(v)) for v in c]
    w = [mp.mpf(float(v)) for v in w]
    d = len(c)
    if family == 1:   # cos(2 pi w1 + sum c x)
        val = mp.cos(2 * mp.pi * w[0] + sum(c) / 2)
        for cj in c:
            val *= 2 * mp.sin(cj / 2) / cj
        return float(val)
    if family == 2:   # prod 1/(c^-2 + (x-w)^2)
        val = mp.mpf(1)
        for cj, wj in zip(c, w):
            val *= cj * (mp.atan(cj * (1 - wj)) + mp.atan(cj * wj))
        return float(val)
    if family == 3:   # (1 + sum c x)^-(d+1): alternating vertex sum
        s = mp.mpf(0)
        for v in itertools.product((0, 1), repeat=d):
            s += (-1) ** sum(v) / (1 + sum(cj for cj, vj in zip(c, v) if vj))
        den = mp.factorial(d)
        for cj in c:
            den *= cj
        return float(s / den)
    if family == 4:   # exp(-sum c^2 (x-w)^2)
        val = mp.mpf(1)
        for cj, wj in zip(c, w):
            val *= mp.sqrt(mp.pi) / (2 * cj) * (mp.erf(cj * (1 - wj)) + mp.erf(cj * wj))
        return float(val)
    if family == 5:   # exp(-sum c |x-w|)
        val = mp.mpf(1)
        for cj, wj in zip(c, w):
            val *= (2 - mp.exp(-cj * wj) - mp.exp(-cj * (1 - wj))) / cj
        return float(val)
    if family == 6:   # 0 if x1 > w1 or x2 > w2 else exp(sum c x)
        val = mp.mpf(1)
        for j, (cj, wj) in enumerate(zip(c, w)):
            upper = wj if j < 2 else mp.mpf(1)
            val *= (mp.exp(cj * upper) - 1) / cj
        return float(val)
    raise ValueError(family)


def monomial_exact(d: int) -> float:
    return 0.5 ** d


def trig_lattice_exact(amp, h, theta, n: int, z, delta) -> complex:
    """Exact (1/n) sum_i prod_j (1 + a_j cos(2 pi (h_j x_ij + theta_j))) on the shifted
    lattice x_i = {i z / n + delta} (real points, no rounding), via the character sum."""
    d = len(amp)
    total = 0j
    for s in itertools.product((-1, 0, 1), repeat=d):
        k = [sj * int(hj) for sj, hj in zip(s, h)]
        if sum(kj * int(zj) for kj, zj in zip(k, z)) % n != 0:
            continue
        coef = 1.0 + 0j
        phase = 0.0
        for sj, aj, tj, kj, dj in zip(s, amp, theta, k, delta):
            if sj != 0:
                coef *= aj / 2.0
                phase += sj * tj + kj * dj
        total += coef * complex(math.cos(2 * math.pi * phase), math.sin(2 * math.pi * phase))
    return total


KOROBOV_PHI = {  # phi_r(u) = int_0^u (2r+1) C(2r, r) t^r (1-t)^r dt, expanded
    1: [0, 0, 3, -2],
    2: [0, 0, 0, 10, -15, 6],
    3: [0, 0, 0, 0, 35, -84, 70, -20],
    4: [0, 0, 0, 0, 0, 126, -420, 540, -315, 70],
}


def korobov_phi_exact(r: int, u) -> mp.mpf:
    u = mp.mpf(u)
    return sum(cf * u ** k for k, cf in enumerate(KOROBOV_PHI[r]))


def korobov_w_exact(r: int, u) -> mp.mpf:
    u = mp.mpf(u)
    return sum(k * cf * u ** (k - 1) for k, cf in enumerate(KOROBOV_PHI[r]) if k > 0)


def sidi_phi_exact(r: int, u) -> mp.mpf:
    u = mp.mpf(u)
    if r == 1:
        return (1 - mp.cos(mp.pi * u)) / 2
    if r == 2:
        return u - mp.sin(2 * mp.pi * u) / (2 * mp.pi)
    raise ValueError(r)
