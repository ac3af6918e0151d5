"""CPU-side checks of the C ABI: the library loads, exports every entry point declared in
include/qmc_gb300.h, validates arguments on the host, and its host-only functions agree
with the oracle (shifts, get_next_n, the Levenberg-Marquardt fit)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "qmc_gb300.h")


@pytest.fixture(scope="module")
def q():
    import paper_1811_11720_gb300 as q
    from paper_1811_11720_gb300 import build
    build.build()
    q.lib()
    return q


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for need in ("qmc_integrate", "qmc_sums", "qmc_points", "qmc_finalize", "qmc_get_next_n",
                 "qmc_make_shifts", "qmc_evaluate", "qmc_histogram", "qmc_fit_polysingular",
                 "qmc_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol(q):
    lib = q.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_1811_11720_gb300 import _capi
    assert set(_capi.PROTOTYPES) == set(declared_functions())


def test_abi_version_and_strerror(q):
    assert q.lib().qmc_abi_version() == 1
    assert q.lib().qmc_strerror(0) == b"ok"
    assert b"coprime" in q.lib().qmc_strerror(-4)


def test_shifts_match_oracle(q):
    import oracle as O
    for seed, m, d in [(0, 4, 3), (12345, 32, 10), (2**63 + 5, 1024, 16), (7, 1, 1)]:
        assert np.array_equal(q.make_shifts(seed, m, d), O.shifts(seed, m, d))


def test_get_next_n(q):
    t = q.GenvecTable.load()
    assert q.get_next_n(t, 100000) == 108863
    assert q.get_next_n(t, 1) == 1021
    assert q.get_next_n(t, 1021) == 1021
    with pytest.raises(q.QMCError) as e:
        q.get_next_n(t, 10**12)
    assert e.value.code == -3


def test_argument_errors_without_device(q):
    """Host-side validation returns error codes before any device call."""
    lib = q.lib()
    assert lib.qmc_make_shifts(1, 0, 3, None) == -1
    D = np.zeros(16, dtype=np.uint64)
    assert lib.qmc_make_shifts(1, 2, 0, D.ctypes.data) == -2
    assert lib.qmc_make_shifts(1, 2000, 2, D.ctypes.data) == -5
    f = q.Integrand.genz(2, [1.0, 2.0], [0.5, 0.5]).host_struct()
    Dd = np.zeros((4, 2), dtype=np.uint64)
    r = q.rule(1021, [1, 374], Dd, ("korobov", 3))
    ws = np.zeros(64, dtype=np.uint8)
    out = np.zeros(16)
    # z not coprime / zero
    r_bad = q.rule(1021, [1, 1021], Dd, ("korobov", 3))
    assert lib.qmc_sums(C.byref(f), C.byref(r_bad), 0, 1021, ws.ctypes.data, 64, out.ctypes.data, None, None) == -4
    # empty range
    assert lib.qmc_sums(C.byref(f), C.byref(r), 5, 5, ws.ctypes.data, 64, out.ctypes.data, None, None) == -12
    # workspace too small
    assert lib.qmc_sums(C.byref(f), C.byref(r), 0, 1021, ws.ctypes.data, 8, out.ctypes.data, None, None) == -10
    # bad transform order
    r_t = q.rule(1021, [1, 374], Dd, ("korobov", 9))
    assert lib.qmc_sums(C.byref(f), C.byref(r_t), 0, 1021, ws.ctypes.data, 1 << 20, out.ctypes.data, None, None) == -8
    # dimension mismatch
    f3 = q.Integrand.genz(2, [1.0, 2.0, 3.0], [0.5, 0.5, 0.5]).host_struct()
    assert lib.qmc_sums(C.byref(f3), C.byref(r), 0, 1021, ws.ctypes.data, 1 << 20, out.ctypes.data, None, None) == -2
    # unknown family
    bad = q.Integrand.genz(2, [1.0, 2.0], [0.5, 0.5]).host_struct()
    bad.family = 99
    assert lib.qmc_sums(C.byref(bad), C.byref(r), 0, 1021, ws.ctypes.data, 1 << 20, out.ctypes.data, None, None) == -7
    # m < 2 for the error estimate
    assert lib.qmc_finalize(out.ctypes.data, 1, 1021, 0, out.ctypes.data, None, None) == -5


def test_workspace_size_depends_on_range_only(q):
    Dd = np.zeros((32, 4), dtype=np.uint64)
    r = q.rule(10560653, [1, 2, 3, 4], Dd, ("baker",))
    a = q.sums_workspace_bytes(r, False, 0, 10560653)
    b = q.sums_workspace_bytes(r, True, 0, 10560653)
    assert a > 0 and b == 2 * a or b >= 2 * a - 512
    Dd2 = np.zeros((1024, 4), dtype=np.uint64)
    r2 = q.rule(10560653, [1, 2, 3, 4], Dd2, ("baker",))
    assert q.sums_workspace_bytes(r2, False, 0, 10560653) > a


def test_tile_count_is_not_monotone_in_n(q):
    """The tile decomposition comes in whole waves, so its tile count is not monotone in
    the range length: at m = 32, n = 886,097 has more tiles than the larger n = 974,707.
    Every reservation of partials for a sequence of lattices (the server's per-request
    pool slice, qmc_integrate's workspace) must therefore take the maximum over the
    lattices, not the largest one; the GPU regression tests exercise exactly this pair."""
    t_small, _ = q.sums_tile_count(886_097, 32)
    t_large, _ = q.sums_tile_count(974_707, 32)
    assert t_small > t_large
    Dd = np.zeros((32, 4), dtype=np.uint64)
    r1 = q.rule(886_097, [1, 2, 3, 4], Dd, ("baker",))
    r2 = q.rule(974_707, [1, 2, 3, 4], Dd, ("baker",))
    assert q.sums_workspace_bytes(r1, False, 0, 886_097) > q.sums_workspace_bytes(r2, False, 0, 974_707)


def test_lm_fit_matches_least_squares_oracle(q):
    """The library's Levenberg-Marquardt and SciPy's trust-region solver, on the same CDF
    data from an oracle histogram, give maps that agree closely (the fit itself is a
    heuristic: its parameters are not unique, the fitted curve is what matters)."""
    import oracle as O
    import workloads as W
    from oracle import fit as OF
    tab = O.load_genvec_table(os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt"))
    n = 108863
    c, w = W.genz_params(2, 3, 4)
    f = O.genz(2, c, w)
    D1 = O.shifts(9, 1, 3)[0]
    hist = O.histogram(f, n, tab[n], D1, 1000)
    opts = q.fit_options(maxiter=200, xtol=1e-10, gtol=1e-12, ftol=1e-14)
    P = q.fit_polysingular(hist, opts)
    yy = np.linspace(0, 1, 501)
    for j in range(3):
        y, x = OF.cdf_pairs(hist[j], 10)
        a_ref, cost_ref = OF.fit_polysingular(y, x)
        cost = float(np.sum((OF.polysingular(P[j], y) - x) ** 2))
        assert cost <= cost_ref * 1.05 + 1e-12
        assert P[j][0] >= 1.001 and P[j][1] <= -0.001
        assert np.max(np.abs(OF.polysingular(P[j], yy) - OF.polysingular(a_ref, yy))) < 2e-3


def test_lm_fit_recovers_known_map(q):
    from oracle import fit as OF
    a_true = np.array([1.25, -0.35, 0.18, 0.12, 0.45, 0.03])
    # a histogram whose CDF at the edges is p^-1: build the density on a fine grid
    bins = 2000
    edges = np.linspace(0, 1, bins + 1)
    yfine = np.linspace(0, 1, 200001)
    xfine = OF.polysingular(a_true, yfine)
    cdf_at_edges = np.interp(edges, xfine, yfine)
    hist = np.diff(cdf_at_edges)[None, :]
    P = q.fit_polysingular(hist, q.fit_options(maxiter=300, xtol=1e-12, gtol=1e-14, ftol=1e-15,
                                               stepsize=5))
    yy = np.linspace(0, 1, 201)
    assert np.max(np.abs(OF.polysingular(P[0], yy) - OF.polysingular(a_true, yy))) < 1e-4


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and raises without its library."""
    pkg = os.path.join(ROOT, "paper_1811_11720_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
    from paper_1811_11720_gb300 import _capi
    with pytest.raises(ImportError):
        _capi.load("/nonexistent/libqmc_gb300.so")


def test_noalloc_argument_codes_match_sums(q):
    """qmc_sums_noalloc validates its arguments exactly as qmc_sums does, in the same order
    and before any device call (m = 0, m above QMC_MAX_SHIFTS, unknown family, dimension
    mismatch, empty range)."""
    lib = q.lib()
    f = q.Integrand.genz(2, [1.0, 2.0], [0.5, 0.5]).host_struct()
    out = np.zeros(16)
    ws = np.zeros(64, dtype=np.uint8)
    Dd = np.zeros((4, 2), dtype=np.uint64)
    f3 = q.Integrand.genz(2, [1.0, 2.0, 3.0], [0.5, 0.5, 0.5]).host_struct()
    bad = q.Integrand.genz(2, [1.0, 2.0], [0.5, 0.5]).host_struct()
    bad.family = 99
    cases = []
    for m in (0, q._capi.QMC_MAX_SHIFTS + 1):
        r = q.rule(1021, [1, 374], Dd, ("korobov", 3))
        r.m = m
        cases.append((f, r, 0, 1021, -5))
    r = q.rule(1021, [1, 374], Dd, ("korobov", 3))
    cases += [(bad, r, 0, 1021, -7), (f3, r, 0, 1021, -2), (f, r, 7, 7, -12)]
    for ff, rr, a, b, code in cases:
        assert lib.qmc_sums_noalloc(C.byref(ff), C.byref(rr), a, b, out.ctypes.data, None, None) == code
        assert lib.qmc_sums(C.byref(ff), C.byref(rr), a, b, ws.ctypes.data, 64, out.ctypes.data,
                            None, None) == code


def test_merge_sums_is_compensated_and_ordered(q):
    """qmc_merge_sums adds double-double per-shift sums in part order: the low words are
    kept (1 + 1e16 - 1e16 survives), the result is the exact sum whenever that fits a
    double-double, and bad sizes are rejected."""
    from fractions import Fraction

    from paper_1811_11720_gb300 import shard
    parts = [np.array([1e16, 0.0]), np.array([1.0, 0.0]), np.array([-1e16, 0.0])]
    out = shard.merge_sums(parts)
    assert out[0] + out[1] == 1.0
    rng = np.random.default_rng(3)
    hi = rng.normal(size=(5, 8)) * 10.0 ** rng.integers(-8, 8, size=(5, 8))
    lo = hi * 2.0 ** -60 * rng.normal(size=(5, 8))
    pairs = np.empty((5, 16))
    pairs[:, 0::2], pairs[:, 1::2] = hi, lo
    got = shard.merge_sums(list(pairs))
    for k in range(8):
        exact = sum(Fraction(float(v)) for v in np.concatenate([hi[:, k], lo[:, k]]))
        err = abs(Fraction(float(got[2 * k])) + Fraction(float(got[2 * k + 1])) - exact)
        assert err <= abs(exact) * Fraction(2) ** -100 + Fraction(2) ** -1070
    lib = q.lib()
    buf = np.zeros(6)
    assert lib.qmc_merge_sums(buf.ctypes.data, 1, 3, buf.ctypes.data) == -1
    assert lib.qmc_merge_sums(buf.ctypes.data, 0, 2, buf.ctypes.data) == -1
    assert lib.qmc_merge_sums(None, 1, 2, buf.ctypes.data) == -1
