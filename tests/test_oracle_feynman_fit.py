"""Pins for the complex Feynman-parameter-like integrand (contour deformation,
Jacobian, determinant, principal branch) and for the variance-reduction fit (Sec. 2.4)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import fit as OF


def _poly(coef, exps, x):
    return sum(c * np.prod([xk ** e for xk, e in zip(x, ee)]) for c, ee in zip(coef, exps))


@pytest.fixture(scope="module")
def fl():
    return W.feynman_like(3)


def test_polynomial_derivatives_by_finite_differences(fl):
    f = O.feynman_complex(fl)
    x = np.array([0.31, 0.62, 0.27, 0.85, 0.44])
    p = O.feynman_parts(f, x)
    assert abs(p["F_real"] - _poly(fl.F.coef, fl.F.exps, x)) < 1e-13
    h = 1e-6
    for k in range(5):
        e = np.zeros(5)
        e[k] = h
        g = (_poly(fl.F.coef, fl.F.exps, x + e) - _poly(fl.F.coef, fl.F.exps, x - e)) / (2 * h)
        assert abs(g - p["grad"][k]) < 1e-7
        for l in range(5):
            e2 = np.zeros(5)
            e2[l] = 1e-4
            gp = (_poly(fl.F.coef, fl.F.exps, x + e + e2) - _poly(fl.F.coef, fl.F.exps, x - e + e2)) / (2 * h)
            gm = (_poly(fl.F.coef, fl.F.exps, x + e - e2) - _poly(fl.F.coef, fl.F.exps, x - e - e2)) / (2 * h)
            assert abs((gp - gm) / 2e-4 - p["hess"][k, l]) < 1e-4
    assert np.allclose(p["hess"], p["hess"].T, atol=1e-12)


def test_deformation_and_jacobian(fl):
    """z_k = x_k - i lam x_k(1-x_k) dF/dx_k, and J = dz/dx by complex finite differences;
    det J against numpy's LU determinant; U(z), F(z) against direct evaluation."""
    f = O.feynman_complex(fl)
    x = np.array([0.21, 0.52, 0.77, 0.35, 0.64])
    p = O.feynman_parts(f, x)

    def zmap(xx):
        return O.feynman_parts(f, xx)["z"]

    z = zmap(x)
    assert np.allclose(z.real, x, atol=0)
    grad = p["grad"]
    assert np.allclose(z.imag, -fl.lam * x * (1 - x) * grad, rtol=1e-14, atol=0)
    h = 1e-6
    Jfd = np.zeros((5, 5), complex)
    for l in range(5):
        e = np.zeros(5)
        e[l] = h
        Jfd[:, l] = (zmap(x + e) - zmap(x - e)) / (2 * h)
    assert np.allclose(p["J"], Jfd, atol=2e-7)
    assert abs(p["det"] - np.linalg.det(p["J"])) < 1e-12 * abs(p["det"])
    assert abs(p["F"] - _poly(fl.F.coef, fl.F.exps, z)) < 1e-12
    assert abs(p["U"] - _poly(fl.U.coef, fl.U.exps, z)) < 1e-12


def test_integrand_value_principal_branch(fl):
    f = O.feynman_complex(fl)
    u = np.array([0.21, 0.52, 0.77, 0.35, 0.64])
    g = O.eval_g(f, ("none",), u)
    p = O.feynman_parts(f, u)
    expect = p["U"] * np.exp(-fl.b * np.log(p["F"])) * p["det"]
    assert abs(g - expect) < 1e-13 * abs(expect)


def test_imaginary_part_of_F_is_nonpositive_near_real_zeros(fl):
    """The deformation realises F - i delta: Im F(z) ~ -lam sum x(1-x)(dF)^2 <= 0 to first
    order; sample points and check the sign where the deformation is small."""
    f = O.Integrand("feynman", 5, ucoef=fl.U.coef, uexp=fl.U.exps, fcoef=fl.F.coef,
                    fexp=fl.F.exps, pa=fl.a, pb=fl.b, lam=0.05)
    rng = np.random.default_rng(0)
    for _ in range(200):
        x = rng.uniform(0, 1, 5)
        p = O.feynman_parts(f, x)
        assert p["F"].imag <= 1e-12


def test_contour_independence(genvec_table):
    """Cauchy: two valid deformations (lam = 0.3, 0.5) give the same integral within the
    combined error."""
    fl = W.feynman_like(3)
    n = 108863
    D = O.shifts(8, 12, 5)
    vals = []
    for lam in (0.3, 0.5):
        f = O.Integrand("feynman", 5, ucoef=fl.U.coef, uexp=fl.U.exps, fcoef=fl.F.coef,
                        fexp=fl.F.exps, pa=fl.a, pb=fl.b, lam=lam)
        r = O.integrate(f, ("korobov", 3), n, genvec_table[n], D)
        vals.append(r)
    dre = abs(vals[0]["value_re"] - vals[1]["value_re"])
    dim = abs(vals[0]["value_im"] - vals[1]["value_im"])
    sre = np.hypot(vals[0]["error_re"], vals[1]["error_re"])
    sim = np.hypot(vals[0]["error_im"], vals[1]["error_im"])
    assert dre < 5 * sre + 1e-10 and dim < 5 * sim + 1e-10


def test_fit_recovers_known_parameters():
    """Data generated from a known PolySingular map is fitted back (inverse CDF lies in
    the ansatz family)."""
    a_true = np.array([1.25, -0.35, 0.18, 0.12, 0.45, 0.03])
    y = np.linspace(0, 1, 101)
    x = OF.polysingular(a_true, y)
    a, cost = OF.fit_polysingular(y, x)
    assert cost < 1e-20
    yy = np.linspace(0, 1, 1001)
    assert np.max(np.abs(OF.polysingular(a, yy) - OF.polysingular(a_true, yy))) < 1e-8


def test_fit_identity_for_uniform_integrand():
    hist = np.ones(1000)
    y, x = OF.cdf_pairs(hist, 10)
    assert np.allclose(y, x)
    a, cost = OF.fit_polysingular(y, x)
    assert cost < 1e-20
    assert np.max(np.abs(OF.polysingular(a, y) - y)) < 1e-10


def test_histogram_totals(genvec_table):
    """Every dimension's histogram sums the same |f| values: row sums agree and equal the
    sum of evaluate()."""
    n = 4691
    c, w = W.genz_params(2, 3, 1)
    f = O.genz(2, c, w)
    D1 = O.shifts(3, 1, 3)[0]
    h = O.histogram(f, n, genvec_table[n], D1, 64)
    vals = O.evaluate(f, n, genvec_table[n], D1)
    assert np.allclose(h.sum(axis=1), np.abs(vals).sum(), rtol=1e-13)
    pts = O.points(n, genvec_table[n], D1[None, :])[:, 0, :]
    for j in range(3):
        b = np.minimum(np.floor(pts[:, j] * 64).astype(int), 63)
        ref = np.bincount(b, weights=np.abs(vals), minlength=64)
        assert np.allclose(ref, h[j], rtol=1e-13)
