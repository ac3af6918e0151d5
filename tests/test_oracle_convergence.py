"""Error scaling of the randomly shifted lattice rule with periodizing transforms, on the
oracle (CPU): the paper reports (Sec. 5.1, Scaling behaviour, Fig. scalingplot) that the error falls
roughly like 1/n with Korobov-1 and like 1/n^2 with Korobov-3 for its loop integrals; for
the smooth Genz integrands the rates are at least that (observed: about n^-2 and n^-4).
The standard error over 16 shifts, fitted on five CBC lattices from n = 1021 to 256,687,
must fall at least that fast, and the true error (closed forms) must stay within a few
standard errors, i.e. the error estimate of Eq. (lattice-error) is honest."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import ROOT
from oracle import closed_forms as CF

TABLE = O.load_genvec_table(os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt"))
NS = [min(n for n in TABLE if n >= t) for t in (1000, 4000, 16000, 64000, 256000)]


@pytest.mark.parametrize("fam", [1, 2, 4])
@pytest.mark.parametrize("tr,slope_max", [(("korobov", 1), -1.0), (("korobov", 3), -2.0)])
def test_error_falls_at_least_as_fast_as_stated(fam, tr, slope_max):
    d, m = 3, 16
    c, w = W.genz_params(fam, d, 5)
    exact = float(CF.genz_exact(fam, c, w))
    D = O.shifts(3, m, d)
    sig, err = [], []
    for n in NS:
        r = O.integrate(O.genz(fam, c, w), tr, n, TABLE[n][:d], D)
        sig.append(r["error_re"])
        err.append(abs(r["value_re"] - exact))
    slope = np.polyfit(np.log(NS), np.log(sig), 1)[0]
    assert slope <= slope_max, (slope, sig)
    for s, e in zip(sig, err):
        assert e <= 6.0 * s + 1e-14 * abs(exact), (e, s)
