"""Pins for the oracle's integrands and estimator: closed-form integrals (Genz table,
Sec. 5.2), the minimal example (Sec. 3.2), lattice exactness on trigonometric
polynomials (Eq. (lattice) with the character sum), and the error estimate
(Eq. (lattice-error))."""
import itertools

import mpmath as mp
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import golden
from oracle import closed_forms as CF


@pytest.mark.parametrize("family", [1, 2, 3, 4, 5, 6])
def test_genz_closed_forms_against_quadrature(family):
    """The closed forms themselves, checked by mpmath quadrature in d = 2."""
    c, w = W.genz_params(family, 2, 11)
    f = {1: lambda x, y: mp.cos(2 * mp.pi * w[0] + c[0] * x + c[1] * y),
         2: lambda x, y: 1 / ((c[0] ** -2 + (x - w[0]) ** 2) * (c[1] ** -2 + (y - w[1]) ** 2)),
         3: lambda x, y: (1 + c[0] * x + c[1] * y) ** -3,
         4: lambda x, y: mp.exp(-(c[0] ** 2 * (x - w[0]) ** 2 + c[1] ** 2 * (y - w[1]) ** 2)),
         5: lambda x, y: mp.exp(-(c[0] * abs(x - w[0]) + c[1] * abs(y - w[1]))),
         6: lambda x, y: 0 if (x > w[0] or y > w[1]) else mp.exp(c[0] * x + c[1] * y)}[family]
    mp.mp.dps = 20
    brk = lambda j: sorted({0.0, float(w[j]), 1.0})  # noqa: E731
    q = mp.quad(f, brk(0), brk(1))
    mp.mp.dps = 50
    assert abs(float(q) - CF.genz_exact(family, c, w)) < 1e-10 * max(1.0, abs(float(q)))


@pytest.mark.parametrize("family,d,transform", [
    (1, 6, ("korobov", 3)), (2, 4, ("korobov", 3)), (3, 6, ("korobov", 2)),
    (4, 6, ("korobov", 3)), (1, 8, ("baker",)), (4, 8, ("baker",)), (3, 10, ("korobov", 1)),
    (5, 4, ("baker",)), (6, 3, ("korobov", 1)), (2, 6, ("sidi", 3))])
def test_genz_integrals_agree_with_closed_form(genvec_table, family, d, transform):
    n = 1072187 if d <= 6 else 108863
    c, w = W.genz_params(family, d, 5)
    D = O.shifts(2024 + family, 8, d)
    r = O.integrate(O.genz(family, c, w), transform, n, genvec_table[n], D)
    exact = CF.genz_exact(family, c, w)
    dev = abs(r["value_re"] - exact)
    # within 6 sigma (or a tiny absolute floor when sigma underflows the rule's accuracy)
    assert dev <= 6 * r["error_re"] + 1e-13 * abs(exact), (r["value_re"], r["error_re"], exact)


def test_minimal_example(genvec_table):
    """Sec. 3.2: int x0 x1 x2 = 1/8 with the Korobov weight-3 transform."""
    kv = {}
    for line in open(golden("minimal_example.txt")):
        if not line.startswith("#"):
            k, *v = line.split()
            kv[k] = v
    d = int(kv["d"][0])
    exact = float(kv["exact"][0])
    n = 8191 + 1  # minn default 8191 (App. A.1): the next table size
    n = min(v for v in genvec_table if v >= n)
    D = O.shifts(1, 16, d)
    r = O.integrate(O.monomial(d), ("korobov", int(kv["transform"][1])), n, genvec_table[n], D)
    assert abs(r["value_re"] - exact) <= max(5 * r["error_re"], 1e-14)
    assert r["error_re"] < 1e-9


def test_trig_polynomial_exact_on_lattice(genvec_table):
    """Untransformed lattice sum of prod_j (1 + a_j cos 2 pi (h_j x_j + theta_j)) equals the
    character-sum prediction (1 when no nonzero frequency lies in the dual lattice)."""
    n = 1021
    z = genvec_table[n]
    for d in (2, 4, 6):
        amp, h, th = W.trig_product_params(d, 3 + d)
        D = O.shifts(77 + d, 4, d)
        r = O.shift_sums(O.trig(amp, h, th), ("none",), n, z, D)
        for k in range(4):
            pred = CF.trig_lattice_exact(amp, h, th, n, z[:d], D[k].astype(float) / 2**53)
            got = (r["re"][k, 0] + r["re"][k, 1]) / n
            assert abs(got - pred.real) < 1e-13


def test_trig_polynomial_dual_lattice_frequency(genvec_table):
    """With h in the dual lattice (h . z = 0 mod n) the rule is not exact and the
    deviation is the predicted shift-dependent cosine."""
    n = 1021
    z = genvec_table[n][:2]
    h = np.array([n - z[1], 1])       # h1 + h2 z2 = n = 0 (mod n)
    amp = np.array([0.6, 0.7])
    th = np.array([0.13, 0.71])
    D = O.shifts(5, 6, 2)
    r = O.shift_sums(O.trig(amp, h, th), ("none",), n, z, D)
    for k in range(6):
        pred = CF.trig_lattice_exact(amp, h, th, n, z, D[k].astype(float) / 2**53)
        got = (r["re"][k, 0] + r["re"][k, 1]) / n
        assert abs(pred.real - 1.0) > 1e-3          # genuinely not 1
        # rounding of the points perturbs cos(2 pi h x) by ~ 2 pi h ulp
        assert abs(got - pred.real) < 1e-11


def test_error_estimate_formula():
    """Eq. (lattice-error) on explicit numbers."""
    Q = np.array([1.0, 2.0, 4.0, 7.0])
    qbar, sig = O.shift_reduce(Q)
    assert qbar == 3.5
    assert abs(sig - np.sqrt(((Q - 3.5) ** 2).sum() / 12)) < 1e-15


@pytest.mark.slow
def test_error_estimate_coverage(genvec_table):
    """Over many seeds the true value lies within 3 sigma in most cases (the d = 4 product-peak shape,
    product peak in d = 4, Korobov-3, n = 1021)."""
    n = 1021
    c, w = W.product_peak_params(4, 3)
    exact = CF.genz_exact(2, c, w)
    f = O.genz(2, c, w)
    hits = 0
    N = 60
    for s in range(N):
        D = O.shifts(1000 + s, 16, 4)
        r = O.integrate(f, ("korobov", 3), n, genvec_table[n], D, nthreads=1)
        hits += abs(r["value_re"] - exact) <= 3 * r["error_re"]
    assert hits >= 0.85 * N


def test_shift_sums_independent_of_thread_count(genvec_table):
    n = 108863
    c, w = W.genz_params(1, 5, 1)
    D = O.shifts(3, 4, 5)
    a = O.shift_sums(O.genz(1, c, w), ("korobov", 2), n, genvec_table[n], D, nthreads=1)
    b = O.shift_sums(O.genz(1, c, w), ("korobov", 2), n, genvec_table[n], D, nthreads=4)
    assert np.array_equal(a["re"], b["re"])


def test_index_ranges_add_up(genvec_table):
    """Sums over [0, a) and [a, n) combine to the sum over [0, n)."""
    n = 108863
    c, w = W.genz_params(4, 3, 1)
    D = O.shifts(4, 4, 3)
    f = O.genz(4, c, w)
    full = O.shift_sums(f, ("baker",), n, genvec_table[n], D)
    lo = O.shift_sums(f, ("baker",), n, genvec_table[n], D, i0=0, i1=40000)
    hi = O.shift_sums(f, ("baker",), n, genvec_table[n], D, i0=40000, i1=n)
    tot = lo["re"].sum(axis=1) + hi["re"].sum(axis=1)
    assert np.allclose(tot, full["re"].sum(axis=1), rtol=1e-15, atol=0)


def test_sector_equals_undeformed_feynman_with_positive_coefficients():
    """lambda = 0 leaves z = x and J = 1: the complex family reduces to the real one."""
    fl = W.sector_like(3, 4, 12, 20)
    fr = O.from_feynman(fl)
    fc = O.Integrand("feynman", fl.d, ucoef=fl.U.coef, uexp=fl.U.exps, fcoef=fl.F.coef,
                     fexp=fl.F.exps, pa=fl.a, pb=fl.b, lam=0.0)
    for u in itertools.product([0.1, 0.45, 0.9], repeat=4):
        a = O.eval_g(fr, ("korobov", 3), u)
        b = O.eval_g(fc, ("korobov", 3), u)
        assert abs(a.real - b.real) <= 1e-14 * abs(a.real) and abs(b.imag) <= 1e-14 * abs(a.real)
