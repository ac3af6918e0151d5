"""Error bounds of the polynomial families' fixed-point forms (qmc_poly.cuh), checked on
the CPU in exact rational arithmetic.  Each test restates the integer steps of one device
routine and checks the bound its comment states:

* dense_eval_fixed (real sector family, F with non-negative coefficients and constant
  term c0 > 0): within 4.5 N units of 2^-s for N products, every partial sum below 2^63;
  with the staging's guard 4.5 N (B / c0) <= 2^20 that is a relative error <= 2^-42;
* feyn_fixed_parts (complex family, d = 3..6): Hessian, gradient and grad U within 2^-49
  of the sum B of the polynomial's |entries|, partial sums below 3 B 2^s < 2^62;
* feyn_add_horner: the nested-form coefficient slots give the polynomial's value;
* the symmetric elimination of det J (feynman_jacobian_det_sym) gives det J;
* unit_to_fixed64 / fixed_u64_to_double / fixed_s64_to_double: x 2^64 truncated and
  v 2^-s truncated to 53 bits.

The GPU parity tests check the compiled kernels against the oracle."""
from __future__ import annotations

import math
import random
import struct
from fractions import Fraction

import numpy as np

M64 = 1 << 64


def mulhi_trunc(a, b):
    ah, al, bh, bl = a >> 32, a & 0xFFFFFFFF, b >> 32, b & 0xFFFFFFFF
    return (ah * bh + ((ah * bl) >> 32) + ((al * bh) >> 32)) % M64


def smulhi_x(c, X):
    """Signed c times X / 2^64 as the device forms it (two's complement wrap)."""
    h = mulhi_trunc(c % M64, X)
    r = (h - X) % M64 if c < 0 else h
    return r - M64 if r >= 1 << 63 else r


def ilogb(v):
    return math.frexp(v)[1] - 1


def d2b(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def b2d(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def unit_to_fixed64(x):
    b = d2b(x)
    if b >= 0x3FF0000000000000 and b < 1 << 63:
        return M64 - 1
    if b == 0 or b >= 1 << 63:
        return 0
    r = 1022 - (b >> 52)
    m = ((b << 11) % M64) | (1 << 63)
    return 0 if r >= 64 else m >> r


def fixed_u64_to_double(u, s):
    if u == 0:
        return 0.0
    lz = 64 - u.bit_length()
    m = (u << lz) % M64
    return b2d((((1085 - lz - s) << 52) + (m >> 11)) % M64)


def fixed_s64_to_double(v, s):
    sign = 1 << 63 if v < 0 else 0
    return b2d(sign | d2b(fixed_u64_to_double(abs(v), s)))


# --- real sector family: dense Horner in unsigned fixed point -------------------------

def dense_fixed(X, V, D, C):
    """dense_eval_fixed with the x_(V-1) = 1 iterations as additions; returns the value
    and the largest partial sum."""
    F, idx, peak = 0, 0, 0
    if D == 3:
        for a in range(V - 1):
            sa = 0
            for b in range(a, V - 1):
                t = 0
                for c in range(b, V - 1):
                    t += mulhi_trunc(C[idx], X[c]); idx += 1
                t += C[idx]; idx += 1
                sa += mulhi_trunc(X[b], t)
                peak = max(peak, t, sa)
            sa += C[idx]; idx += 1
            F += mulhi_trunc(X[a], sa)
            peak = max(peak, sa, F)
    else:
        for a in range(V - 1):
            t = 0
            for b in range(a, V - 1):
                t += mulhi_trunc(C[idx], X[b]); idx += 1
            t += C[idx]; idx += 1
            F += mulhi_trunc(X[a], t)
            peak = max(peak, t, F)
    F += C[idx]
    return F, max(peak, F)


def dense_exact(x, V, D, c):
    xs = list(x) + [Fraction(1)]
    F, idx = Fraction(0), 0
    if D == 3:
        for a in range(V):
            for b in range(a, V):
                for cc in range(b, V):
                    F += Fraction(c[idx]) * xs[a] * xs[b] * xs[cc]; idx += 1
    else:
        for a in range(V):
            for b in range(a, V):
                F += Fraction(c[idx]) * xs[a] * xs[b]; idx += 1
    return F


def dense_size(V, D):
    return V * (V + 1) // 2 if D == 2 else V * (V + 1) * (V + 2) // 6


def test_sector_fixed_horner_bound():
    rng = random.Random(5)
    worst = 0.0
    for trial in range(60):
        V = rng.randint(4, 9)
        D = 3 if trial % 3 else 2
        n = dense_size(V, D)
        c = [rng.random() * (10 ** rng.uniform(-3, 1)) if rng.random() < 0.7 else 0.0
             for _ in range(n)]
        c[-1] = 0.25 + 0.5 * rng.random()                  # constant term
        B = math.fsum(c)
        s = 62 - ilogb(B)
        Cq = [int(round(math.ldexp(v, s))) for v in c]
        X = []
        for k in range(V - 1):
            r = rng.random()
            X.append(0 if r < 0.05 else M64 - 1 if r < 0.1 else rng.getrandbits(64 - rng.randint(0, 40)))
        Fq, peak = dense_fixed(X, V, D, Cq)
        assert peak < 1 << 63
        exact = dense_exact([Fraction(v, M64) for v in X], V, D, c)
        N = n + (dense_size(V, 2) if D == 3 else 0) + V
        err = abs(Fraction(Fq, 1 << s) - exact)
        assert err <= Fraction(45, 10) * N * Fraction(1, 1 << s)
        worst = max(worst, float(err / exact))
        # the staging's guard: relative error <= 2^-42 whenever 4.5 N B <= 2^20 c0
        if 4.5 * N * B <= 2.0 ** 20 * c[-1]:
            assert err / exact <= Fraction(1, 1 << 42)
    assert worst < 2.0 ** -45


# --- complex family: fixed-point Hessian and gradients ------------------------------

def pair(i, j, d):
    return i * d - i * (i - 1) // 2 + (j - i)


def test_complex_fixed_parts_bound():
    rng = np.random.default_rng(9)
    for d in range(3, 7):
        for trial in range(8):
            nU, nF = 1 + d + d * d, 1 + d + d * d + d * d * (d + 1) // 2
            F = rng.standard_normal(nF) * 10.0 ** rng.uniform(-3, 3)
            U = rng.standard_normal(nU)
            F2 = F[1 + d:1 + d + d * d].reshape(d, d)
            F[1 + d:1 + d + d * d] = ((F2 + F2.T) / 2).ravel()
            U2 = U[1 + d:].reshape(d, d)
            U[1 + d:] = ((U2 + U2.T) / 2).ravel()
            bf, bu = float(np.abs(F).sum()), float(np.abs(U).sum())
            sf, su = 61 - ilogb(16 * bf), 61 - ilogb(16 * bu)
            ff = [int(round(math.ldexp(float(v), sf))) for v in F]
            uf = [int(round(math.ldexp(float(v), su))) for v in U]
            X = [int(v) for v in rng.integers(0, 1 << 63, d, dtype=np.uint64) * 2 + 1]
            X[0] = M64 - 1 if trial % 4 == 0 else X[0]
            x = [Fraction(v, M64) for v in X]
            f1, F2q, F3q = ff[1:1 + d], ff[1 + d:1 + d + d * d], ff[1 + d + d * d:]
            u1, U2q = uf[1:1 + d], uf[1 + d:]
            f1e = [Fraction(float(v)) for v in F[1:1 + d]]
            F2e = [Fraction(float(v)) for v in F[1 + d:1 + d + d * d]]
            F3e = [Fraction(float(v)) for v in F[1 + d + d * d:]]
            u1e = [Fraction(float(v)) for v in U[1:1 + d]]
            U2e = [Fraction(float(v)) for v in U[1 + d:]]
            Hq = [[0] * d for _ in range(d)]
            He = [[Fraction(0)] * d for _ in range(d)]
            for i in range(d):
                for j in range(i, d):
                    sq = 2 * F2q[i * d + j]
                    se = 2 * F2e[i * d + j]
                    for k in range(d):
                        sq += smulhi_x(F3q[pair(i, j, d) * d + k], X[k])
                        se += F3e[pair(i, j, d) * d + k] * x[k]
                        assert abs(sq) < 1 << 62
                    Hq[i][j] = Hq[j][i] = sq
                    He[i][j] = He[j][i] = se
            tol_f = Fraction(bf) / (1 << 49)
            tol_u = Fraction(bu) / (1 << 49)
            for i in range(d):
                for j in range(d):
                    assert abs(Fraction(Hq[i][j], 1 << sf) - He[i][j]) <= tol_f
                hx = qx = px = 0
                for j in range(d):
                    hx += smulhi_x(Hq[i][j], X[j])
                    qx += smulhi_x(F2q[i * d + j], X[j])
                    px += smulhi_x(U2q[i * d + j], X[j])
                    assert max(abs(hx), abs(qx)) < 1 << 62 and abs(px) < 1 << 62
                gq = f1[i] + qx + (hx >> 1)
                ge = f1e[i] + sum(F2e[i * d + j] * x[j] for j in range(d)) + \
                    sum(He[i][j] * x[j] for j in range(d)) / 2
                assert abs(Fraction(gq, 1 << sf) - ge) <= tol_f
                gUq = u1[i] + 2 * px
                gUe = u1e[i] + 2 * sum(U2e[i * d + j] * x[j] for j in range(d))
                assert abs(Fraction(gUq, 1 << su) - gUe) <= tol_u


# --- nested (Horner) form slots and the symmetric elimination ------------------------

def test_nested_form_slots_give_the_polynomial():
    rng = np.random.default_rng(3)
    for d in range(1, 7):
        for _ in range(10):
            terms = []
            for _ in range(25):
                deg = int(rng.integers(0, 4))
                e = [0] * d
                for _ in range(deg):
                    e[int(rng.integers(0, d))] += 1
                terms.append((float(rng.standard_normal()), e))
            h = [0.0] * (1 + d + d * (d + 1) // 2 + d * (d + 1) * (d + 2) // 6)
            for c, e in terms:                           # feyn_add_horner's slots
                f = [k for k in range(d) for _ in range(e[k])][:3]
                slot = 0
                if len(f) >= 1:
                    slot = 1 + f[0]
                if len(f) >= 2:
                    slot = 1 + d + pair(f[0], f[1], d)
                if len(f) == 3:
                    off = sum((d - i) * (d - i + 1) // 2 for i in range(f[0])) + \
                        sum(d - j for j in range(f[0], f[1]))
                    slot = 1 + d + d * (d + 1) // 2 + off + (f[2] - f[1])
                h[slot] += c
            x = rng.uniform(0, 1, d)
            c2, c3 = h[1 + d:], h[1 + d + d * (d + 1) // 2:]
            F, p2, p3 = h[0], 0, 0
            for i in range(d):                           # the kernel's nested loop
                tf = h[1 + i]
                for j in range(i, d):
                    tij = c2[p2]
                    for k in range(j, d):
                        tij += c3[p3] * x[k]
                        p3 += 1
                    tf += tij * x[j]
                    p2 += 1
                F += tf * x[i]
            ref = sum(c * np.prod([x[k] ** e[k] for k in range(d)]) for c, e in terms)
            assert abs(F - ref) <= 1e-13 * (1 + sum(abs(c) for c, _ in terms))


def test_symmetric_elimination_gives_det_j():
    rng = np.random.default_rng(5)
    for D in range(1, 7):
        for _ in range(100):
            H = rng.standard_normal((D, D)) * rng.uniform(0.1, 30)
            H = (H + H.T) / 2
            x = rng.uniform(0, 1, D)
            g = rng.standard_normal(D) * 10
            lam = rng.uniform(0.1, 1)
            lx = -lam * x * (1 - x)
            lamb = -lam * (1 - 2 * x) * g
            J = np.eye(D) + 1j * (np.diag(lamb) + lx[:, None] * H)
            Kr, Ki = np.zeros((D, D)), np.zeros((D, D))
            det = complex(1.0, lx[0] * H[0, 0] + lamb[0])
            if D > 1:
                c0 = lx[0] / det
                for r in range(1, D):
                    u = c0 * H[0, r]
                    for q in range(r, D):
                        Kr[r, q] = u.real * H[0, q]
                        Ki[r, q] = u.imag * H[0, q] + H[r, q]
                for c in range(1, D):
                    piv = complex(1 + lx[c] * Kr[c, c], lamb[c] + lx[c] * Ki[c, c])
                    det *= piv
                    if c + 1 == D:
                        break
                    cc = lx[c] / piv
                    for r in range(c + 1, D):
                        w = cc * complex(Kr[c, r], Ki[c, r])
                        for q in range(r, D):
                            k = complex(Kr[r, q], Ki[r, q]) - w * complex(Kr[c, q], Ki[c, q])
                            Kr[r, q], Ki[r, q] = k.real, k.imag
            ref = np.linalg.det(J)
            assert abs(det - ref) <= 1e-12 * abs(ref)


# --- conversions -------------------------------------------------------------------------

def test_fixed_conversions():
    rng = random.Random(11)
    for _ in range(2000):
        x = rng.random() * 2.0 ** -rng.randint(0, 70)
        X = unit_to_fixed64(x)
        assert X == int(Fraction(x) * M64) or (x == 0 and X == 0)
    assert unit_to_fixed64(1.0) == M64 - 1 and unit_to_fixed64(-0.5) == 0
    assert unit_to_fixed64(0.0) == 0
    for _ in range(2000):
        u = rng.getrandbits(rng.randint(1, 64)) | 1
        s = rng.randint(20, 120)
        v = fixed_u64_to_double(u, s)
        exact = Fraction(u, 1 << s)
        assert Fraction(v) <= exact < Fraction(v) + Fraction(v) * Fraction(1, 1 << 52)
        sv = fixed_s64_to_double(-u, s)
        assert sv == -v
    assert fixed_u64_to_double(0, 40) == 0.0
