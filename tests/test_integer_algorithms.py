"""Error bounds of the kernels' integer-pipe algorithms, checked on the CPU in exact
integer arithmetic against 300-bit references (mpmath).  Each test restates the integer
steps of one device routine (with the constants read from the CUDA headers, so a changed
literal is caught here too) and checks the bound that the routine's comment and the design
notes state:

* exp_fixed (qmc_exp.cuh): e^(+-A 2^-E) within 2^-55 relatively before rounding;
* cos_turns_fixed (qmc_cos.cuh): cos(2 pi T 2^-64) within 1e-17 absolutely;
* fx_recip (qmc_fixed.cuh): 2^127 / m within 4 units (first-order branch near 2^63);
* korobov_P + phi (qmc_fixed.cuh): Korobov<r,r> phi within 2^-(61 - 1.7 r) absolutely,
  the Estrin form with w^2 from v^2.

The GPU parity tests check the compiled kernels themselves against the oracle."""
from __future__ import annotations

import os
import random
import re
import struct
from fractions import Fraction
from math import comb

import pytest

mp = pytest.importorskip("mpmath")
mp.mp.prec = 300

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1811_11720_gb300", "csrc")
M64 = (1 << 64) - 1


def _src(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _table(src, name):
    m = re.search(name + r"\[\d+\]\s*=\s*\{(.*?)\};", src, re.S)
    return [int(v, 16) for v in re.findall(r"0x([0-9a-fA-F]+)ull", m.group(1))]


def _const(src, name):
    return int(re.search(r"constexpr uint64_t " + name + r"\s*=\s*0x([0-9a-fA-F]+)ull", src).group(1), 16)


def mulhi_trunc(a, b):
    ah, al, bh, bl = a >> 32, a & 0xFFFFFFFF, b >> 32, b & 0xFFFFFFFF
    return ah * bh + ((ah * bl) >> 32) + ((al * bh) >> 32)


def sqhi_trunc(a):
    ah, al = a >> 32, a & 0xFFFFFFFF
    return ah * ah + (((ah * al) >> 32) << 1)


def test_exp_fixed_error_bound():
    src = _src("qmc_exp.cuh")
    tab = _table(src, "kExp2Fixed")
    L, LN2 = _const(src, "kLog2e"), _const(src, "kLn2")
    D = {k: _const(src, "kD%d" % k) for k in range(2, 7)}

    def exp_fixed(A, E, neg):
        P = A * L
        hi, lo = P >> 64, P & M64
        sh = E - 1
        k = min(hi >> sh, 4096)
        F = ((hi << (64 - sh)) | (lo >> sh)) & M64
        ke = k
        if neg:
            ke = -k - (1 if F else 0)
            F = (-F) & M64
        Y = mulhi_trunc((F << 6) & M64, LN2)
        G = D[6]
        for j in (5, 4, 3, 2):
            G = D[j] + mulhi_trunc(G, Y)
        em1 = Y + mulhi_trunc(Y, mulhi_trunc(Y, G))
        t = tab[F >> 58]
        M = t + (mulhi_trunc(t, em1) >> 6)
        assert (1 << 63) <= M < (1 << 64)
        return Fraction(M, 1 << 63) * Fraction(2) ** ke

    rng = random.Random(7)
    worst = 0
    for _ in range(4000):
        E = rng.randint(2, 64)
        A = rng.getrandbits(rng.randint(1, 63))
        neg = rng.random() < 0.7
        a = mp.mpf(A) / mp.mpf(2) ** E
        if a > 700:
            continue
        got = exp_fixed(A, E, neg)
        ref = mp.exp(-a if neg else a)
        worst = max(worst, abs(mp.mpf(got.numerator) / got.denominator / ref - 1))
    assert worst < mp.mpf(2) ** -55, float(worst)


def test_cos_turns_fixed_error_bound():
    src = _src("qmc_cos.cuh")
    tab = _table(src, "kCos256")
    k2pi, c6, c24 = _const(src, "k2Pi"), _const(src, "kC6"), _const(src, "kC24")
    k120, k720 = _const(src, "kK120"), _const(src, "kK720")

    def cos_fixed(T):
        u = (T + (1 << 55)) & M64
        j = u >> 56
        r = (u & ((1 << 56) - 1)) - (1 << 55)
        neg = r < 0
        a = -r if neg else r
        Y = mulhi_trunc(a << 8, k2pi)
        Z = sqhi_trunc(Y)
        Ps = mulhi_trunc(Z, c6 - mulhi_trunc(Z, k120))
        Sy = Y - (mulhi_trunc(Y, Ps) >> 10)
        Q2 = (1 << 63) - (mulhi_trunc(Z, c24 - mulhi_trunc(Z, k720)) >> 10)
        Cm = mulhi_trunc(Z, Q2)
        q, i = j >> 6, j & 63
        ca, sa = tab[i], tab[64 - i]
        even = not (q & 1)
        P, Q = (ca, sa) if even else (sa, ca)
        ysin = mulhi_trunc(Q, Sy) >> 5
        v = P - (mulhi_trunc(P, Cm) >> 10) + (-ysin if even != neg else ysin)
        return -v if q in (1, 2) else v

    rng = random.Random(11)
    worst = 0
    for t in range(4000):
        T = rng.getrandbits(64) if t % 5 else ((rng.randint(0, 1023) << 54) + rng.randint(-3, 3)) & M64
        err = abs(mp.mpf(cos_fixed(T)) / mp.mpf(2) ** 62 - mp.cos(2 * mp.pi * mp.mpf(T) / mp.mpf(2) ** 64))
        worst = max(worst, err)
    assert worst < 1e-17, float(worst)


def test_fx_recip_error_bound():
    def f32(x):
        return struct.unpack("f", struct.pack("f", x))[0]

    def recip(m, ulps):
        mh = m >> 32
        if mh == 0x80000000:
            dl = m - (1 << 63)
            return (1 << 64) if dl == 0 else (-2 * dl) & M64
        r = f32(1.0 / f32(float(mh)))
        bits = struct.unpack("I", struct.pack("f", r))[0] + ulps   # rcp.approx: a few ulps
        E = ((bits >> 23) & 0xFF) - 127
        mant = (bits & 0x7FFFFF) | 0x800000
        R = M64 if E >= -31 else mant << (72 + E)
        for _ in range(2):
            plo, phi = (m * R) & M64, (m * R) >> 64
            ehi = ((1 << 63) - phi - (1 if plo else 0)) & M64
            neg = ehi >= (1 << 63)
            c = ((R * (((-ehi) & M64) if neg else ehi)) >> 64) << 1
            R = (R - c) & M64 if neg else (R + c) & M64
        return R

    rng = random.Random(3)
    for t in range(20000):
        kind = t % 5
        if kind == 0:
            m = (1 << 63) + rng.getrandbits(rng.randint(0, 40))
        elif kind == 1:
            m = M64 - rng.getrandbits(rng.randint(0, 40))
        else:
            m = (1 << 63) | rng.getrandbits(63)
        R = recip(m, rng.randint(-3, 3))
        exact = Fraction(1 << 127, m)
        assert abs(R - exact) <= 4, (hex(m), float(R - exact))


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_korobov_phi_estrin_error_bound(r):
    S = sum(comb(r + k, k) for k in range(r + 1))
    F = 0
    while S * 2 ** (F + 1) < 2 ** 64:
        F += 1
    c = [comb(r + k, k) for k in range(r + 1)] + [0]

    def fixed_pow(E, V, V2):
        if E == 2:
            return V2
        if E == 3:
            return mulhi_trunc(V2, V)
        h = fixed_pow(E // 2, V, V2)
        sq = sqhi_trunc(h)
        return mulhi_trunc(sq, V) if E % 2 else sq

    def phi(V):
        V2 = sqhi_trunc(V)
        W = (~V) & M64
        ws = W >> (64 - F)
        pair = [(c[2 * j] << F) + c[2 * j + 1] * ws for j in range(r // 2 + 1)]
        P = pair[0]
        if r >= 2:
            W2 = (V2 - 2 * V - 2) & M64
            P += mulhi_trunc(pair[1], W2)
            if r >= 4:
                W4 = sqhi_trunc(W2)
                P += mulhi_trunc(pair[2], W4)
                if r >= 6:
                    P += mulhi_trunc(pair[3], mulhi_trunc(W4, W2))
        assert P < 2 ** 64
        return (mulhi_trunc(fixed_pow(r + 1, V, V2), P) << (64 - F)) & M64

    C = (2 * r + 1) * comb(2 * r, r)

    def exact(v):   # phi(v) = C int_0^v (t (1 - t))^r dt, v <= 1/2
        return sum(Fraction(C * comb(r, k) * (-1) ** k, r + 1 + k) * v ** (r + 1 + k) for k in range(r + 1))

    rng = random.Random(r)
    worst = Fraction(0)
    for V in [0, 1, 2, (1 << 63) - 1, 1 << 40] + [rng.getrandbits(63) for _ in range(600)]:
        worst = max(worst, abs(Fraction(phi(V), 1 << 64) - exact(Fraction(V, 1 << 64))))
    assert float(worst) < 2.0 ** -(61 - 1.7 * r), float(worst)
