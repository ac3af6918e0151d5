"""Seeded synthetic inputs for the lattice-rule integrator.

This module is the only code shared by the CPU oracle, the CUDA parity tests and the
benchmark.  It draws integrand parameters (Genz ``c`` and ``w``, polynomial
coefficients, trigonometric test-function amplitudes) from a seeded NumPy generator
and returns plain arrays.  It holds none of the lattice method's arithmetic: no
lattice points, no transforms, no integrand evaluation, no shift generation.

Workload shapes follow the paper's test suites:

* Genz families 1-6 (Sec. 5.2, table of test functions): ``w_j ~ U(0,1)`` and
  ``c_j > 0`` rescaled so that ``||c||_1`` equals the family's difficulty from the
  paper's difficulty table (6.0, 18.0, 2.2, 15.2, 16.1, 16.4), the same sum for every
  dimension.
* The d=4 product-peak workload uses a fixed ``c_j = 5`` (no rescaling).
* Feynman-parameter-like polynomials ``U`` (all monomials of total degree 2) and
  ``F`` (all monomials of total degree 3) in 5 variables with coefficients
  ``U(-1, 2)``, so that ``F`` changes sign on the unit cube.
* Sector-like real polynomials (positive coefficients) for batches of integrals.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# ||c||_1 per Genz family (Sec. 5.2, difficulty table).
GENZ_DIFFICULTY = {1: 6.0, 2: 18.0, 3: 2.2, 4: 15.2, 5: 16.1, 6: 16.4}

GENZ_NAMES = {1: "oscillatory", 2: "product_peak", 3: "corner_peak", 4: "gaussian",
              5: "c0", 6: "discontinuous"}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed) & ((1 << 63) - 1)))


def genz_params(family: int, d: int, seed: int, c_norm: float | None = None):
    """Draw (c, w) for Genz family ``family`` in ``d`` dimensions.

    ``a_j ~ U(0,1)``, ``c = ||c||_1 * a / sum(a)``, ``w_j ~ U(0,1)``.
    """
    if family not in GENZ_DIFFICULTY:
        raise ValueError(f"unknown Genz family {family}")
    rng = _rng(seed * 1000003 + family * 101 + d)
    a = rng.uniform(0.0, 1.0, d)
    # guard the (measure-zero) all-zero draw
    a = np.maximum(a, 1e-12)
    w = rng.uniform(0.0, 1.0, d)
    norm = GENZ_DIFFICULTY[family] if c_norm is None else float(c_norm)
    c = norm * a / a.sum()
    return c.astype(np.float64), w.astype(np.float64)


def product_peak_params(d: int, seed: int, a: float = 5.0):
    """Fixed-width product peak: ``c_j = a`` for all j, ``w_j ~ U(0,1)``."""
    rng = _rng(seed * 7919 + d)
    w = rng.uniform(0.0, 1.0, d)
    return np.full(d, float(a)), w.astype(np.float64)


def all_monomials(d: int, degree: int) -> np.ndarray:
    """Exponent vectors of every monomial of total degree ``degree`` in ``d`` variables,
    in lexicographic order (deterministic)."""
    out = []
    for combo in itertools.combinations_with_replacement(range(d), degree):
        e = [0] * d
        for v in combo:
            e[v] += 1
        out.append(e)
    out.sort(reverse=True)
    return np.array(out, dtype=np.int32)


@dataclass
class Polynomial:
    """Sum of monomials ``sum_m coef[m] * prod_k x_k**exps[m, k]``."""
    coef: np.ndarray   # (M,) float64
    exps: np.ndarray   # (M, d) int32

    @property
    def nterms(self) -> int:
        return int(self.coef.shape[0])


@dataclass
class FeynmanLike:
    """``U^a / F^b`` with a contour deformation of strength ``lam`` (complex integrand)."""
    U: Polynomial
    F: Polynomial
    a: float = 1.0
    b: float = 2.5
    lam: float = 0.5
    d: int = field(default=5)


def feynman_like(seed: int, d: int = 5, deg_u: int = 2, deg_f: int = 3,
                 lo: float = -1.0, hi: float = 2.0, a: float = 1.0, b: float = 2.5,
                 lam: float = 0.5) -> FeynmanLike:
    """Random U (all monomials of degree ``deg_u``) and F (degree ``deg_f``) with
    coefficients ``U(lo, hi)``."""
    rng = _rng(seed * 31337 + d)
    eu = all_monomials(d, deg_u)
    ef = all_monomials(d, deg_f)
    cu = rng.uniform(lo, hi, eu.shape[0])
    cf = rng.uniform(lo, hi, ef.shape[0])
    return FeynmanLike(Polynomial(cu, eu), Polynomial(cf, ef), a, b, lam, d)


def feynman_regular(seed: int, d: int = 5, beta: float = 0.95, eps: float = 5e-4,
                    a: float = 1.0, b: float = 2.5, lam: float = 0.5) -> FeynmanLike:
    """Feynman-parameter-like integrand whose integral exists: U as in ``feynman_like``
    (all degree-2 monomials, coefficients U(-1, 2)) and
        F = 1 - beta sum_k x_k (1 - x_k) + eps sum_{|m| = 3} c_m x^m,  c_m ~ U(-1, 2),
    which is positive on every face of the cube (for beta < 4/(d-1) and small eps) and
    negative around the centre (beta > 4/d), so F changes sign inside and the contour
    deformation, which vanishes on the faces, keeps F(z) away from zero."""
    rng = _rng(seed * 7907 + d)
    eu = all_monomials(d, 2)
    cu = rng.uniform(-1.0, 2.0, eu.shape[0])
    e3 = all_monomials(d, 3)
    c3 = eps * rng.uniform(-1.0, 2.0, e3.shape[0])
    e0 = np.zeros((1, d), np.int32)
    e1 = np.eye(d, dtype=np.int32)
    e2 = 2 * np.eye(d, dtype=np.int32)
    ef = np.vstack([e0, e1, e2, e3]).astype(np.int32)
    cf = np.concatenate([[1.0], -beta * np.ones(d), beta * np.ones(d), c3])
    return FeynmanLike(Polynomial(cu, eu), Polynomial(cf, ef), a, b, lam, d)


def sector_like(seed: int, d: int, nterms_u: int, nterms_f: int,
                a: float = 1.0, b: float = 2.5) -> FeynmanLike:
    """Real sector-like integrand ``U^a / F^b`` with positive coefficients ``U(0,1)``:
    ``nterms_u`` monomials of degree 2 and ``nterms_f`` of degree 3 picked from all
    monomials in ``d`` variables (with repetition allowed beyond the full set), plus a
    constant term in F so that F > 0 on the closed cube."""
    rng = _rng(seed * 65537 + d * 17 + nterms_u * 3 + nterms_f)
    eu_all = all_monomials(d, 2)
    ef_all = all_monomials(d, 3)
    iu = rng.integers(0, eu_all.shape[0], nterms_u)
    jf = rng.integers(0, ef_all.shape[0], nterms_f - 1)
    eu = eu_all[iu]
    ef = np.vstack([np.zeros((1, d), np.int32), ef_all[jf]])
    cu = rng.uniform(0.0, 1.0, nterms_u)
    cf = rng.uniform(0.0, 1.0, nterms_f)
    cf[0] = 0.25 + 0.5 * cf[0]
    return FeynmanLike(Polynomial(cu, eu), Polynomial(cf, ef), a, b, 0.0, d)


def trig_product_params(d: int, seed: int, hmax: int = 3):
    """Parameters of ``prod_j (1 + a_j cos(2 pi (h_j x_j + theta_j)))``: integer
    frequencies ``h_j`` in ``[1, hmax]``, amplitudes ``a_j ~ U(0.1, 0.9)``, phases
    ``theta_j ~ U(0,1)``."""
    rng = _rng(seed * 104729 + d)
    h = rng.integers(1, hmax + 1, d).astype(np.int64)
    amp = rng.uniform(0.1, 0.9, d)
    theta = rng.uniform(0.0, 1.0, d)
    return amp, h, theta


def fit_params_example(d: int, seed: int):
    """A valid PolySingular parameter set per dimension (a0 >= 1.001, a1 <= -0.001)
    used to test the fit-apply step in isolation: shape (d, 6)."""
    rng = _rng(seed * 4099 + d)
    p = np.empty((d, 6))
    p[:, 0] = 1.001 + rng.uniform(0.05, 1.0, d)
    p[:, 1] = -0.001 - rng.uniform(0.05, 1.0, d)
    p[:, 2] = rng.uniform(0.0, 0.3, d)
    p[:, 3] = rng.uniform(0.0, 0.3, d)
    p[:, 4] = rng.uniform(0.2, 0.6, d)
    p[:, 5] = rng.uniform(-0.1, 0.1, d)
    return p
