"""Pins for the oracle's periodizing transforms (Sec. 2.3) and the PolySingular map
(Sec. 2.4, Eq. (ISfit))."""
import mpmath as mp
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import closed_forms as CF
from oracle import fit as OF

US = [0.0, 1e-9, 0.013, 0.1, 0.25, 0.3333, 0.5, 0.6, 0.77, 0.9, 0.999, 1.0 - 2**-40, 1.0]


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_korobov_symmetric_matches_hand_integrated_polynomial(r):
    for u in US:
        phi, w = O.transform_eval("korobov", r, r, u)
        assert abs(phi - float(CF.korobov_phi_exact(r, u))) <= 4e-15
        assert abs(w - float(CF.korobov_w_exact(r, u))) <= 1e-13 * max(1.0, abs(w))


@pytest.mark.parametrize("r0,r1", [(1, 1), (2, 5), (5, 3), (0, 2), (3, 0)])
def test_korobov_weight_is_derivative_and_normalised(r0, r1):
    phi0, _ = O.transform_eval("korobov", r0, r1, 0.0)
    phi1, _ = O.transform_eval("korobov", r0, r1, 1.0)
    assert phi0 == 0.0 and abs(phi1 - 1.0) < 1e-15
    integral = mp.quad(lambda t: O.transform_eval("korobov", r0, r1, float(t))[1], [0, 0.5, 1])
    assert abs(integral - 1) < 1e-12
    for u in [0.1, 0.37, 0.5, 0.81]:
        dphi = mp.diff(lambda t: O.transform_eval("korobov", r0, r1, float(t))[0], u, h=1e-4)
        assert abs(dphi - O.transform_eval("korobov", r0, r1, u)[1]) < 1e-6


@pytest.mark.parametrize("r", [1, 2])
def test_sidi_low_orders_closed_form(r):
    for u in US:
        phi, _ = O.transform_eval("sidi", r, r, u)
        assert abs(phi - float(CF.sidi_phi_exact(r, u))) < 1e-15


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
def test_sidi_weight_is_derivative_and_normalised(r):
    assert O.transform_eval("sidi", r, r, 0.0)[0] == 0.0
    assert abs(O.transform_eval("sidi", r, r, 1.0)[0] - 1.0) < 1e-14
    integral = mp.quad(lambda t: O.transform_eval("sidi", r, r, float(t))[1], [0, 0.5, 1])
    assert abs(integral - 1) < 1e-12
    for u in [0.1, 0.37, 0.5, 0.81]:
        dphi = mp.diff(lambda t: O.transform_eval("sidi", r, r, float(t))[0], u, h=1e-4)
        assert abs(dphi - O.transform_eval("sidi", r, r, u)[1]) < 1e-6


def test_baker_tent():
    for u in US:
        phi, w = O.transform_eval("baker", 0, 0, u)
        assert w == 1.0
        assert phi == (2 * u if u <= 0.5 else 2 - 2 * u)
    assert O.transform_eval("none", 0, 0, 0.3) == (0.3, 1.0)


def test_polysingular_endpoints_and_derivative():
    P = W.fit_params_example(6, 1)
    for a in P:
        assert O.polysingular(a, 0.0)[0] == 0.0
        assert abs(O.polysingular(a, 1.0)[0] - 1.0) < 1e-15
        for x in [0.05, 0.3, 0.5, 0.9]:
            p, dp = O.polysingular(a, x)
            num = mp.diff(lambda t: O.polysingular(a, float(t))[0], x, h=1e-4)
            assert abs(num - dp) < 2e-6 * max(1.0, abs(dp))
            assert dp > 0
            # the numpy restatement used by the fit agrees
            assert abs(OF.polysingular(a, x) - p) < 1e-15


def test_polysingular_negative_a2_a3_use_absolute_value():
    """App. A.5 form: |a2|, |a3| enter, so the sign of a2, a3 does not matter."""
    a = np.array([1.3, -0.4, 0.2, 0.1, 0.5, 0.05])
    b = a.copy()
    b[2] *= -1
    b[3] *= -1
    for x in [0.1, 0.6]:
        assert O.polysingular(a, x) == O.polysingular(b, x)
