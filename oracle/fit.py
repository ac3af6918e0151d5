"""Variance-reduction fit, oracle side -- test infrastructure (see oracle/__init__.py).

Sec. 2.4: per integration variable, fit the PolySingular map p (Eq. (ISfit), with the
|a2|, |a3| form of the fit-function table in App. A.5) to the inverse of
CDF_f(x) = int_0^x |f| / int_0^1 |f| (other variables integrated out).

Reading used here (the paper samples the CDF on a lattice and fits with GSL):
  * the CDF of dimension j is taken at the bin edges x_b = b/B of the per-dimension
    histogram of |f| on one shifted lattice (oracle.histogram);
  * the data pairs are (CDF(x_b), x_b), every ``stepsize``-th pair, plus both ends;
  * p(CDF) ~ x is fitted by nonlinear least squares (SciPy's trust-region reflective
    solver as a library step) with a0 >= 1.001 and a1 <= -0.001 as bounds, starting
    from the identity map (a0 = 1.1, a1 = -0.1, a2 = a3 = 0, a4 = 1, a5 = 0).

Parity unpinned: the paper prints no fitted parameters.  Pins: recovery of known
parameters from exact inverse-CDF data, p(0) = 0, p(1) = 1.
"""
from __future__ import annotations

import numpy as np


def polysingular(a, x):
    a = np.asarray(a, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    a2, a3 = abs(a[2]), abs(a[3])
    a6 = 1.0 - a2 - a3 - a[4] - a[5]
    return (a2 * x * (a[0] - 1.0) / (a[0] - x) + a3 * x * (a[1] - 1.0) / (a[1] - x)
            + x * (a[4] + x * (a[5] + x * a6)))


def cdf_pairs(hist_j, stepsize: int = 10):
    """(y, x): y = CDF at bin edges x = b/B, b = 0..B, subsampled every ``stepsize``."""
    h = np.asarray(hist_j, dtype=np.float64)
    B = h.shape[0]
    cdf = np.concatenate([[0.0], np.cumsum(h)])
    cdf /= cdf[-1]
    x = np.arange(B + 1) / B
    idx = np.arange(0, B + 1, max(1, int(stepsize)))
    if idx[-1] != B:
        idx = np.append(idx, B)
    return cdf[idx], x[idx]


START = np.array([1.1, -0.1, 0.0, 0.0, 1.0, 0.0])


def fit_polysingular(y, x, maxiter: int = 40, xtol: float = 3e-3, gtol: float = 1e-8,
                     ftol: float = 1e-8):
    from scipy.optimize import least_squares

    lb = np.array([1.001, -np.inf, -np.inf, -np.inf, -np.inf, -np.inf])
    ub = np.array([np.inf, -0.001, np.inf, np.inf, np.inf, np.inf])

    def res(a):
        return polysingular(a, y) - x

    r = least_squares(res, START.copy(), bounds=(lb, ub), method="trf",
                      max_nfev=100 * maxiter, xtol=1e-12, gtol=1e-12, ftol=1e-12)
    return r.x, float(np.sum(r.fun ** 2))


def fit_all(hist, stepsize: int = 10):
    """Fit every dimension of a (d, B) histogram; returns (d, 6) parameters."""
    return np.array([fit_polysingular(*cdf_pairs(hj, stepsize))[0] for hj in hist])
