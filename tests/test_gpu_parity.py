"""GPU parity: the CUDA path through the C ABI against the CPU oracle on identical seeded
inputs.  Points are compared bit for bit; per-shift sums, the mean and the error within
1e-12 of the mean |g| (the oracle's double-double sum of |g| / n): the kernel's arithmetic
differs from the oracle's by a few ulp per sample (fixed-point forms within ~2^-54
absolutely) and the two-level summation adds at most ~200 ulp of sum |g|, so ~3e-14 is
expected and the bound leaves a factor >= 30."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import closed_forms as CF
from oracle import lattice as L

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1811_11720_gb300 as q
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1811_11720_gb300 import build
    build.build()
    q.lib()
    dev = torch.device("cuda:0")
    return q, torch, dev, q.GenvecTable.load()


def _dev_shifts(torch, D, dev):
    return torch.from_numpy(np.ascontiguousarray(D).astype(np.int64)).to(dev)


def _gpu_sums(env, f, n, z, D, transform, fitp=None, i0=0, i1=None):
    q, torch, dev, _ = env
    Dd = _dev_shifts(torch, D, dev)
    fd = None if fitp is None else torch.from_numpy(np.ascontiguousarray(fitp)).to(dev)
    res, sums, cnt = q.integrate_device(f, n, z, Dd, transform, fd, i0, n if i1 is None else i1)
    torch.cuda.synchronize()
    m = D.shape[0]
    s = sums.cpu().numpy()
    return res.cpu().numpy(), s[: 2 * m].reshape(m, 2), s[2 * m: 4 * m].reshape(m, 2), cnt.cpu().numpy()


def _check_component(Qg, Qo, A, tol):
    """|dQ| <= tol A per shift, and |dQ| <= tol |Q| wherever Q is not cancelled
    (|Q| >= 0.1 A, so the per-sample error cannot be amplified more than tenfold).
    Returns the observed max |dQ| / A."""
    dev = np.abs(Qg - Qo)
    assert np.all(dev <= tol * A), np.max(dev / A)
    big = np.abs(Qo) >= 0.1 * A
    assert np.all(dev[big] <= tol * np.abs(Qo[big])), np.max(dev[big] / np.abs(Qo[big]))
    # an integrand that vanishes identically (A = 0) has dQ = 0 there
    return float(np.max(np.divide(dev, A, out=np.zeros_like(dev), where=A > 0)))


def _compare(gre, gim, o, n, is_complex=False, tol=TOL, label=None):
    A = o["abs"] / n
    Qg = (gre[:, 0] + gre[:, 1]) / n
    Qo = (o["re"][:, 0] + o["re"][:, 1]) / n
    worst = _check_component(Qg, Qo, A, tol)
    if is_complex:
        Qgi = (gim[:, 0] + gim[:, 1]) / n
        Qoi = (o["im"][:, 0] + o["im"][:, 1]) / n
        worst = max(worst, _check_component(Qgi, Qoi, A, tol))
    if label:
        print(f"[parity] {label}: max |dQ|/A = {worst:.2e}")
    return Qg, Qo, A


# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [7, 11, 55, 1021, 108863, 1024565021, 2147483647,
                               1099511627791, 2305843009213693951])
def test_points_bit_exact(env, n):
    q, torch, dev, tab = env
    rng = np.random.default_rng(n % 1000003)
    d = 5
    if n in tab:
        z = [int(v) for v in tab.z_for(n)[:d]]
    else:
        z = []
        while len(z) < d:
            c = int(rng.integers(1, n - 1))
            if np.gcd(c, n) == 1:
                z.append(c)
    m = 3
    D = O.shifts(n & 0xFFFF, m, d)
    D[0, 0] = 0          # a zero shift
    Dd = _dev_shifts(torch, D, dev)
    r = q.rule(n, z, Dd)
    for i0, cnt in [(0, min(n, 300)), (max(0, n - 77), min(n, 77)), (n // 3, min(n - n // 3, 129))]:
        out = torch.empty(cnt * m * d, dtype=torch.float64, device=dev)
        q.points(r, i0, cnt, out)
        got = out.cpu().numpy().view(np.uint64)
        ref = O.points(n, z, D, i0, cnt).reshape(-1).view(np.uint64)
        assert np.array_equal(got, ref), (n, i0)


def test_points_smallest_fractions(env):
    """Points within 2^-64 of an integer take the long-division path: r = 2^-53 mod n and
    D = ceil((n - r) 2^53 / n) give the smallest positive fraction 1/(n 2^53)."""
    q, torch, dev, _ = env
    for n in (108863, 1024565021, 2147483647, 2305843009213693951):
        r = pow(2 ** 53, -1, n)
        D = -(-((n - r) << 53) // n)
        assert D < 2 ** 53
        Dm = np.array([[D]], dtype=np.uint64)
        rr = q.rule(n, [1], _dev_shifts(torch, Dm, dev))
        i0 = max(0, r - 1)
        cnt = min(3, n - i0)
        out = torch.empty(cnt, dtype=torch.float64, device=dev)
        q.points(rr, i0, cnt, out)
        got = out.cpu().numpy()
        ref = O.points(n, [1], Dm, i0, cnt).reshape(-1)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
        assert got[r - i0] == O.point_py(r, n, D) and 0 < got[r - i0] < 2.0 ** -64


def test_points_fig1_lattice(env):
    q, torch, dev, _ = env
    D = np.zeros((1, 2), dtype=np.uint64)
    r = q.rule(55, [1, 34], _dev_shifts(torch, D, dev))
    out = torch.empty(55 * 2, dtype=torch.float64, device=dev)
    q.points(r, 0, 55, out)
    p = out.cpu().numpy().reshape(55, 2)
    assert all(p[i, 0] == i / 55 and p[i, 1] == (34 * i % 55) / 55 for i in range(55))


# ---------------------------------------------------------------------------------------
GENZ_CASES = [(fam, d, tr) for fam in (1, 2, 3, 4) for d in (2, 6, 10)
              for tr in (("korobov", 3), ("baker",))] + \
             [(1, 8, ("korobov", 1)), (4, 8, ("korobov", 2)), (3, 6, ("korobov", 4)),
              (2, 4, ("none",)), (5, 5, ("korobov", 3)), (6, 4, ("baker",)),
              (2, 3, ("sidi", 2)), (1, 3, ("sidi", 3)), (4, 5, ("korobov", 2, 5)),
              (2, 16, ("baker",)), (3, 1, ("korobov", 3)),
              # symmetric r <= 6 runs in integer fixed point; r = 0, r >= 7 and r0 != r1
              # keep the FP64 Horner form
              (1, 10, ("korobov", 4)), (4, 16, ("korobov", 3)), (3, 4, ("korobov", 0)),
              (4, 6, ("korobov", 5)), (3, 7, ("korobov", 6)), (2, 5, ("korobov", 6)),
              (1, 3, ("korobov", 8)), (4, 4, ("korobov", 7)), (3, 5, ("korobov", 3, 1)),
              # families 1 and 3-6 take x in fixed point under none, baker and Korobov r <= 4
              (1, 5, ("none",)), (4, 7, ("none",)), (5, 8, ("baker",)), (6, 6, ("korobov", 2)),
              (3, 10, ("baker",)), (4, 12, ("korobov", 1)),
              # family 2 takes x in fixed point too (product of 1 + q^2 in Fx)
              (2, 8, ("korobov", 1)), (2, 12, ("korobov", 2)), (2, 7, ("korobov", 4)),
              # integer finishes (exp, power and reciprocal) under baker, none, Korobov r <= 2
              (3, 9, ("korobov", 2)), (3, 16, ("korobov", 1)), (3, 3, ("none",)),
              (4, 9, ("korobov", 2)), (5, 11, ("korobov", 1)), (6, 9, ("none",))]


@pytest.mark.parametrize("fam,d,tr", GENZ_CASES)
def test_genz_sums_match_oracle(env, fam, d, tr):
    q, torch, dev, tab = env
    n = 4691
    c, w = W.genz_params(fam, d, 17 + d)
    m = 8
    D = O.shifts(100 + fam * 7 + d, m, d)
    # the table holds s = 10 components; wider rules get their own CBC vector
    z = tab.z_for(n)[:d] if d <= 10 else L.cbc_naive(n, d)[0]
    res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(fam, c, w), n, z, D, tr)
    o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D)
    Qg, Qo, A = _compare(gre, None, o, n)
    qbar, sig = O.shift_reduce(Qo)
    assert abs(res[0] - qbar) <= TOL * A.mean()
    assert abs(res[1] - sig) <= max(1e-9 * sig, 2e-12 * A.mean())
    assert cnt[0] == 0


@pytest.mark.parametrize("fam", [1, 2, 3, 4, 5, 6])
def test_genz_outside_fixed_point_range(env, fam):
    """Parameters outside the Genz ranges (a negative c_j, w_j > 1) take the FP64 form of
    the integrand; results still match the oracle."""
    q, torch, dev, tab = env
    n, d, m = 4691, 4, 8
    c = np.array([1.5, -0.75, 2.0, 0.5])
    w = np.array([0.3, 1.25, 0.6, 0.1])
    z = tab.z_for(n)[:d]
    D = O.shifts(77 + fam, m, d)
    for tr in (("korobov", 3), ("baker",)):
        res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(fam, c, w), n, z, D, tr)
        o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D)
        _compare(gre, None, o, n)


@pytest.mark.parametrize("fam,c", [(5, [300.0, 2.0, 1.0]), (6, [300.0, 2.0, 1.0]),
                                   (4, [1e-3, 2e-3, 5e-4]), (5, [1e-3, 2e-3, 5e-4]),
                                   (6, [1e-3, 2e-3, 5e-4]), (4, [31.0, 0.0, 20.0]),
                                   (5, [0.0, 0.0, 0.0])])
def test_exponential_forms_range(env, fam, c):
    """The integer exponential over its argument range: e^(+-303) (exponent scale 2^54),
    tiny c (scale capped at 2^64, the largest shift), the widest Gaussian and a zero
    argument, under the fixed-point transforms."""
    q, torch, dev, tab = env
    n, m = 4691, 8
    c = np.array(c)
    w = np.array([0.3, 0.85, 0.6])
    d = len(c)
    z = tab.z_for(n)[:d]
    D = O.shifts(57 + fam, m, d)
    for tr in (("korobov", 3), ("baker",), ("none",)):
        res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(fam, c, w), n, z, D, tr)
        o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D)
        _compare(gre, None, o, n)
        assert cnt[0] == 0


@pytest.mark.parametrize("c,w1", [([20.0, 7.0, 13.0], 0.3), ([1e-3, 2e-3, 5e-4], 0.999),
                                  ([0.0, 0.0, 0.0], 0.2), ([6.283185307179586, 3.0, 0.5], 1.0),
                                  ([1000.0, 1.0, 2.0], 0.0)])
def test_oscillatory_turns_range(env, c, w1):
    """Oscillatory cos(2 pi w_1 + sum c_j x_j) with the phase in turns and the integer cos:
    c_j above 2 pi (integer turns per unit x), tiny c, c = 0 (f = cos(2 pi w_1) constant),
    c_1 = 2 pi and w_1 = 1, and c_1 = 1000 (condition number 1000 in the coordinate), under
    baker, none and Korobov-1/2.  (c = 0 with w_1 = 1/4 is left out: there f is 0 exactly
    in turns but 6.1e-17 through the rounded FP64 argument of the oracle's cos.)"""
    q, torch, dev, tab = env
    n, m = 4691, 8
    c = np.array(c)
    d = len(c)
    w = np.array([w1, 0.5, 0.5])
    z = tab.z_for(n)[:d]
    D = O.shifts(13 + int(c[0]), m, d)
    for tr in (("baker",), ("none",), ("korobov", 1), ("korobov", 2)):
        res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(1, c, w), n, z, D, tr)
        o = O.shift_sums(O.genz(1, c, w), tr, n, z, D)
        _compare(gre, None, o, n)
        assert cnt[0] == 0


@pytest.mark.parametrize("c", [[500.0, 300.0, 200.0], [1e-3, 2e-3, 5e-4], [0.0, 0.0, 0.0],
                               [1.0, 0.5, 0.25, 0.125, 2.0, 3.0, 0.75, 1.5, 0.1, 0.2, 0.3,
                                0.4, 0.5, 0.6, 0.7, 0.8]])
def test_corner_peak_power_range(env, c):
    """Corner peak (1 + s)^-(d+1) with the integer power and reciprocal: a large s (the
    result near 1e-11), tiny c (scale capped at 2^64, s below 2^-9), c = 0 (f = 1) and
    d = 16 (the 17th power), under baker, none and Korobov-1/2."""
    q, torch, dev, tab = env
    n, m = 4691, 8
    c = np.array(c)
    d = len(c)
    w = np.full(d, 0.5)
    z = tab.z_for(n)[:d] if d <= 10 else L.cbc_naive(n, d)[0]
    D = O.shifts(31 + d, m, d)
    for tr in (("baker",), ("none",), ("korobov", 1), ("korobov", 2)):
        res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(3, c, w), n, z, D, tr)
        o = O.shift_sums(O.genz(3, c, w), tr, n, z, D)
        _compare(gre, None, o, n)
        assert cnt[0] == 0


@pytest.mark.parametrize("fam", [2, 4])
@pytest.mark.parametrize("c", [[1e3, 3.0, 0.5], [0.01, 0.002, 0.03], [31.0, 1.0, 2.0],
                               [32.0, 1.0, 2.0], [0.0, 2.0, 1.0]])
def test_quadratic_form_scale_limits(env, fam, c):
    """Product peak and Gaussian at the limits of their fixed-point scale: max c = 1000 and
    32 (S < 57, FP64 form), max c = 31 (S = 57, the widest fixed-point case), small c (the
    product peak caps S at 62) and a zero c_j.  Both factors have relative condition number
    up to ~c in the coordinate, so an absolute coordinate difference of 1e-17 between the
    two Korobov forms already moves f by c 1e-17 relatively (c = 2e4 missed the 1e-12
    tolerance by that alone): c stays at 1000 or below."""
    q, torch, dev, tab = env
    n, m = 4691, 8
    c = np.array(c)
    w = np.array([0.3, 0.85, 0.6])
    d = len(c)
    z = tab.z_for(n)[:d]
    D = O.shifts(91 + fam + int(c[0]), m, d)
    for tr in (("korobov", 3), ("baker",)):
        res, gre, _, cnt = _gpu_sums(env, q.Integrand.genz(fam, c, w), n, z, D, tr)
        o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D)
        _compare(gre, None, o, n)
        assert cnt[0] == 0


def test_config1_product_peak_full_size(env):
    """d = 4 product peak, c = 5, Korobov-3, n = 108863, m = 16: whole lattice against the
    oracle and the closed form."""
    q, torch, dev, tab = env
    n, d, m = 108863, 4, 16
    c, w = W.product_peak_params(d, 1)
    D = O.shifts(2024, m, d)
    z = tab.z_for(n)[:d]
    res, gre, _, _ = _gpu_sums(env, q.Integrand.genz(2, c, w), n, z, D, ("korobov", 3))
    o = O.shift_sums(O.genz(2, c, w), ("korobov", 3), n, z, D)
    _compare(gre, None, o, n)
    exact = CF.genz_exact(2, c, w)
    assert abs(res[0] - exact) <= 5 * res[1]


def test_ragged_ranges_and_sharding(env):
    """Arbitrary i-ranges (partial tiles, ragged tails) match the oracle on the same range,
    and ranges that split [0, n) add up to the whole."""
    q, torch, dev, tab = env
    n, d, m = 108863, 6, 5
    c, w = W.genz_params(4, d, 3)
    D = O.shifts(5, m, d)
    z = tab.z_for(n)[:d]
    f = q.Integrand.genz(4, c, w)
    parts = []
    for a, b in [(0, 1), (0, 37), (12345, 12345 + 4097), (n - 1000, n), (0, 50000), (50000, n)]:
        _, gre, _, _ = _gpu_sums(env, f, n, z, D, ("korobov", 3), i0=a, i1=b)
        o = O.shift_sums(O.genz(4, c, w), ("korobov", 3), n, z, D, i0=a, i1=b)
        A = o["abs"]
        Sg = gre[:, 0] + gre[:, 1]
        So = o["re"][:, 0] + o["re"][:, 1]
        assert np.all(np.abs(Sg - So) <= TOL * A)
        parts.append(Sg)
    _, full, _, _ = _gpu_sums(env, f, n, z, D, ("korobov", 3))
    Sfull = full[:, 0] + full[:, 1]
    assert np.allclose(parts[-2] + parts[-1], Sfull, rtol=1e-15, atol=0)


@pytest.mark.parametrize("case", ["real", "complex"])
def test_tile_sharding_is_bit_identical(env, case):
    """Shards cut at tile boundaries, their partials assembled in order and folded by
    qmc_reduce_tiles give qmc_sums bit for bit (the multi-device merge of one rule)."""
    from paper_1811_11720_gb300 import shard
    q, torch, dev, tab = env
    if case == "real":
        n, d, m, i0 = 108863, 6, 32, 17
        c, w = W.genz_params(4, d, 3)
        f = q.Integrand.genz(4, c, w)
    else:
        n, d, m, i0 = 4691, 5, 8, 0
        f = q.Integrand.polynomial(W.feynman_regular(3))
    cplx = f.is_complex
    D = _dev_shifts(torch, O.shifts(9, m, d), dev)
    r = q.rule(n, tab.z_for(n)[:d], D, ("korobov", 3))
    fd = f.device_struct(dev)
    ws = torch.empty(q.sums_workspace_bytes(r, cplx, i0, n), dtype=torch.uint8, device=dev)
    whole = torch.zeros(4 * m, dtype=torch.float64, device=dev)
    q.sums(fd, r, i0, n, ws, whole)
    tiles, _ = q.sums_tile_count(n - i0, m)
    per = 2 * m * (2 if cplx else 1)
    parts = []
    for rank in range(3):
        a, b = shard.shard_tiles(tiles, rank, 3)
        buf = torch.empty((b - a) * per, dtype=torch.float64, device=dev)
        q.sums_tiles(fd, r, i0, n, a, b, buf)
        parts.append(buf.cpu().numpy())
    allp = torch.from_numpy(shard.assemble_tile_partials(parts, m, cplx)).to(dev)
    merged = torch.zeros(4 * m, dtype=torch.float64, device=dev)
    q.reduce_tiles(allp, tiles, m, cplx, merged)
    torch.cuda.synchronize()
    k = (4 if cplx else 2) * m
    assert np.array_equal(merged.cpu().numpy()[:k], whole.cpu().numpy()[:k])


def test_tile_sharding_rejects_bad_ranges(env):
    q, torch, dev, tab = env
    n, d, m = 4691, 3, 8
    c, w = W.genz_params(4, d, 3)
    fd = q.Integrand.genz(4, c, w).device_struct(dev)
    r = q.rule(n, tab.z_for(n)[:d], _dev_shifts(torch, O.shifts(1, m, d), dev), ("baker",))
    tiles, _ = q.sums_tile_count(n, m)
    buf = torch.empty(2 * m * (tiles + 1), dtype=torch.float64, device=dev)
    for a, b in [(0, 0), (3, 2), (0, tiles + 1)]:
        with pytest.raises(q.QMCError) as e:
            q.sums_tiles(fd, r, 0, n, a, b, buf)
        assert e.value.code == -12


def test_deterministic(env):
    q, torch, dev, tab = env
    n, d, m = 108863, 8, 32
    c, w = W.genz_params(1, d, 9)
    D = O.shifts(1, m, d)
    z = tab.z_for(n)[:d]
    f = q.Integrand.genz(1, c, w)
    a = _gpu_sums(env, f, n, z, D, ("baker",))
    b = _gpu_sums(env, f, n, z, D, ("baker",))
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])


@pytest.mark.parametrize("m", [2, 3, 10, 32, 33, 300, 1024])
def test_shift_counts(env, m):
    """m from the minimum (2) past one block (256) to the maximum (1024 = 4 launches)."""
    q, torch, dev, tab = env
    n, d = 1021, 3
    c, w = W.genz_params(2, d, m)
    D = O.shifts(m, m, d)
    z = tab.z_for(n)[:d]
    _, gre, _, _ = _gpu_sums(env, q.Integrand.genz(2, c, w), n, z, D, ("korobov", 2))
    o = O.shift_sums(O.genz(2, c, w), ("korobov", 2), n, z, D)
    _compare(gre, None, o, n)


def test_trig_exactness_on_gpu(env):
    """Lattice exactness: the GPU rule integrates the trigonometric product (no dual-lattice
    frequency) to 1 up to rounding, and reproduces the predicted value when h is in the
    dual lattice."""
    q, torch, dev, tab = env
    n = 1021
    z = [int(v) for v in tab.z_for(n)]
    amp, h, th = W.trig_product_params(4, 7)
    D = O.shifts(3, 4, 4)
    _, gre, _, _ = _gpu_sums(env, q.Integrand.trig(amp, h, th), n, z[:4], D, ("none",))
    Q = (gre[:, 0] + gre[:, 1]) / n
    for k in range(4):
        pred = CF.trig_lattice_exact(amp, h, th, n, z[:4], D[k].astype(float) / 2 ** 53).real
        assert abs(Q[k] - pred) < 1e-13
    h2 = np.array([n - z[1], 1])
    amp2 = np.array([0.6, 0.7])
    th2 = np.array([0.13, 0.71])
    D2 = O.shifts(5, 6, 2)
    _, g2, _, _ = _gpu_sums(env, q.Integrand.trig(amp2, h2, th2), n, z[:2], D2, ("none",))
    Q2 = (g2[:, 0] + g2[:, 1]) / n
    for k in range(6):
        pred = CF.trig_lattice_exact(amp2, h2, th2, n, z[:2], D2[k].astype(float) / 2 ** 53).real
        assert abs(Q2[k] - pred) < 1e-11


def test_minimal_example(env):
    q, torch, dev, tab = env
    out = q.integrate(q.Integrand.monomial(3), tab, 8191, 16, ("korobov", 3), seed=1)
    assert abs(out["value"] - 0.125) <= max(5 * out["err"], 1e-14)
    assert out["n"] == q.get_next_n(tab, 8191)


def test_fit_apply_matches_oracle(env):
    q, torch, dev, tab = env
    n, d, m = 4691, 4, 6
    c, w = W.genz_params(2, d, 2)
    P = W.fit_params_example(d, 3)
    D = O.shifts(8, m, d)
    z = tab.z_for(n)[:d]
    for tr in (("korobov", 3), ("baker",), ("none",)):
        _, gre, _, _ = _gpu_sums(env, q.Integrand.genz(2, c, w), n, z, D, tr, fitp=P)
        o = O.shift_sums(O.genz(2, c, w), tr, n, z, D, fitp=P)
        _compare(gre, None, o, n)


def test_feynman_complex_matches_oracle(env):
    q, torch, dev, tab = env
    fl = W.feynman_like(3)
    n, d, m = 4691, 5, 4
    D = O.shifts(12, m, d)
    z = tab.z_for(n)[:d]
    res, gre, gim, cnt = _gpu_sums(env, q.Integrand.polynomial(fl), n, z, D, ("korobov", 3))
    o = O.shift_sums(O.feynman_complex(fl), ("korobov", 3), n, z, D)
    _compare(gre, gim, o, n, is_complex=True, label="feynman_like d=5 n=4691")
    assert cnt[1] == o["signfail"]


def _quartic_feynman(d):
    """deg F = 4 (forces the factor-list form of the complex family)."""
    base = W.feynman_regular(9, d=d)
    e4 = np.zeros((1, d), np.int32)
    e4[0, 0] = 2
    e4[0, 1] = 2
    F = W.Polynomial(np.concatenate([base.F.coef, [0.3]]), np.vstack([base.F.exps, e4]))
    return W.FeynmanLike(base.U, F, base.a, base.b, base.lam, d)


@pytest.mark.parametrize("case", ["regular_d5", "like_d8", "like_d12", "quartic_d4", "few_terms_d6"])
def test_feynman_forms_match_oracle(env, case):
    """The symmetric-tensor form (deg U <= 2, deg F <= 3, d <= 11, many terms) and the
    factor-list form (higher degree, d > 11, few terms) against the oracle."""
    q, torch, dev, tab = env
    if case == "regular_d5":
        fl = W.feynman_regular(7)
    elif case == "like_d8":
        fl = W.feynman_like(4, d=8)
    elif case == "like_d12":
        fl = W.feynman_like(5, d=12)
    elif case == "quartic_d4":
        fl = _quartic_feynman(4)
    else:
        full = W.feynman_regular(11, d=6)
        keep = np.arange(6)   # constant, the linear terms
        fl = W.FeynmanLike(W.Polynomial(full.U.coef[:3], full.U.exps[:3]),
                           W.Polynomial(full.F.coef[keep], full.F.exps[keep]), 1.0, 2.5, 0.5, 6)
    n, m = 1021, 4
    D = O.shifts(21, m, fl.d)
    z = tab.z_for(n)[:fl.d] if fl.d <= 10 else L.cbc_naive(n, fl.d)[0]
    res, gre, gim, cnt = _gpu_sums(env, q.Integrand.polynomial(fl), n, z, D, ("korobov", 3))
    o = O.shift_sums(O.feynman_complex(fl), ("korobov", 3), n, z, D)
    _compare(gre, gim, o, n, is_complex=True, label=f"feynman {case}")
    assert cnt[1] == o["signfail"]


@pytest.mark.parametrize("d,nu,nf", [(6, 40, 120), (3, 4, 5), (8, 400, 400), (16, 30, 600),
                                     (8, 5, 400), (5, 300, 6)])
def test_sector_real_matches_oracle(env, d, nu, nf):
    """Dense multivariate Horner (many monomials, duplicates merged) and the sparse list
    (few monomials) against the oracle's term-by-term sum."""
    q, torch, dev, tab = env
    nf = min(nf, 512)
    fl = W.sector_like(4 + d, d, nu, nf)
    n, m = 4691, 4
    D = O.shifts(13, m, d)
    z = tab.z_for(n)[:d] if d <= 10 else L.cbc_naive(n, d)[0]
    _, gre, _, _ = _gpu_sums(env, q.Integrand.polynomial(fl), n, z, D, ("korobov", 2))
    o = O.shift_sums(O.from_feynman(fl), ("korobov", 2), n, z, D)
    _compare(gre, None, o, n)


@pytest.mark.parametrize("case", ["negative_term", "small_constant", "no_constant_u_only"])
def test_sector_real_fixed_point_guard(env, case):
    """The dense F takes fixed point only when its relative error bound holds (non-negative
    coefficients, a constant term c0 > 0 and 4.5 N B / c0 <= 2^20); these F fail the
    guard (a negative coefficient, c0 = 1e-5 of B) and take the FP64 form, and the third
    keeps a qualifying F beside a U without constant term.  All match the oracle."""
    q, torch, dev, tab = env
    d = 6
    fl = W.sector_like(40 + len(case), d, 60, 120)
    cf = fl.F.coef.copy()
    if case == "negative_term":
        cf[0] = 2.0 + cf[1:].sum()
        cf[5] = -0.01
    elif case == "small_constant":
        cf[0] = 1e-5 * cf[1:].sum()
    fl = W.FeynmanLike(fl.U, W.Polynomial(cf, fl.F.exps), fl.a, fl.b, 0.0, d)
    n, m = 4691, 4
    D = O.shifts(17, m, d)
    z = tab.z_for(n)[:d]
    _, gre, _, _ = _gpu_sums(env, q.Integrand.polynomial(fl), n, z, D, ("korobov", 3))
    o = O.shift_sums(O.from_feynman(fl), ("korobov", 3), n, z, D)
    _compare(gre, None, o, n, label=f"sector guard {case}")


def test_evaluate_matches_oracle(env):
    q, torch, dev, tab = env
    n, d = 4691, 5
    c, w = W.genz_params(3, d, 1)
    D1 = O.shifts(4, 1, d)[0]
    z = tab.z_for(n)[:d]
    out = torch.empty(1000, dtype=torch.float64, device=dev)
    f = q.Integrand.genz(3, c, w)
    q.evaluate(f.device_struct(dev), n, z, torch.from_numpy(D1.astype(np.int64)).to(dev), 100, 1000, out)
    ref = O.evaluate(O.genz(3, c, w), n, z, D1, 100, 1000)
    got = out.cpu().numpy()
    # per sample: s = 1 + sum c x carries up to ~2d roundings on either side (fused vs
    # separate multiply-add), and t^-(d+1) multiplies its relative error by d + 1:
    # (d + 1) 2d eps = 6.7e-15 for d = 5
    assert np.all(np.abs(got - ref) <= 1e-14 * np.abs(ref))


def test_histogram_matches_oracle(env):
    q, torch, dev, tab = env
    n, d, bins = 108863, 4, 1000
    c, w = W.genz_params(2, d, 5)
    D1 = O.shifts(6, 1, d)[0]
    z = tab.z_for(n)[:d]
    f = q.Integrand.genz(2, c, w)
    hist = torch.empty(d * bins, dtype=torch.float64, device=dev)
    ws = torch.empty(q.histogram_workspace_bytes(n, d, bins), dtype=torch.uint8, device=dev)
    q.histogram(f.device_struct(dev), n, z, torch.from_numpy(D1.astype(np.int64)).to(dev), bins, hist, ws)
    ref = O.histogram(O.genz(2, c, w), n, z, D1, bins)
    got = hist.cpu().numpy().reshape(d, bins)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15 * ref.max())


def test_integrate_with_fit_reduces_error(env):
    """Case with the variance-reduction fit: the fitted integrand integrates to the same
    value (closed form) and the fit runs end to end through qmc_integrate."""
    q, torch, dev, tab = env
    c, w = W.genz_params(2, 3, 8)
    f = q.Integrand.genz(2, c, w)
    exact = CF.genz_exact(2, c, w)
    plain = q.integrate(f, tab, 108863, 16, ("korobov", 1), seed=3)
    fit = q.integrate(f, tab, 108863, 16, ("korobov", 1), fit=q.fit_options(), seed=3)
    assert abs(plain["value"] - exact) <= 6 * plain["err"]
    assert abs(fit["value"] - exact) <= 6 * fit["err"] + 1e-12 * abs(exact)


def test_adaptive_case1_reaches_goal(env):
    q, torch, dev, tab = env
    c, w = W.genz_params(4, 5, 2)
    f = q.Integrand.genz(4, c, w)
    exact = CF.genz_exact(4, c, w)
    out = q.integrate(f, tab, 1021, 16, ("korobov", 3), seed=5,
                      opts=q.options(epsrel=1e-8, epsabs=0.0, maxeval=10**10))
    assert out["err"] <= 1e-8 * abs(out["value"])
    assert out["iterations"] >= 2
    assert abs(out["value"] - exact) <= 10 * out["err"]


def test_adaptive_respects_maxeval(env):
    q, torch, dev, tab = env
    c, w = W.genz_params(1, 8, 2)
    out = q.integrate(q.Integrand.genz(1, c, w), tab, 1021, 8, ("korobov", 1), seed=5,
                      opts=q.options(epsrel=1e-15, epsabs=0.0, maxeval=2_000_000))
    assert out["evaluations"] <= 2_000_000 + out["n"] * out["m"]


def test_nonfinite_counted(env):
    """U/F^2.5 with F = x_1 is infinite at the lattice point x = 0 (zero shift): every such
    sample is counted, once per shift."""
    q, torch, dev, tab = env
    n, m = 1021, 4
    f = q.Integrand("sector", 1, ucoef=np.array([1.0]), uexp=np.zeros((1, 1), np.int32),
                    fcoef=np.array([1.0]), fexp=np.ones((1, 1), np.int32), pa=1.0, pb=2.5)
    D = np.zeros((m, 1), dtype=np.uint64)
    _, _, _, cnt = _gpu_sums(env, f, n, [1], D, ("none",))
    assert cnt[0] == m


@pytest.mark.parametrize("n", [2147483647, 2305843009213693951])
@pytest.mark.parametrize("fam,tr", [(4, ("korobov", 3)), (1, ("korobov", 1)), (3, ("baker",)),
                                    (4, ("none",))])
def test_large_n_fixed_point_paths(env, n, fam, tr):
    """The integer transforms and fixed-point forms on lattices beyond 2^32 points (the
    GPU-built table's 2^31 - 1, and 2^61 - 1 with a Korobov-type vector z_j = 3^j mod n):
    sub-ranges at the start, in the middle and at the end against the oracle."""
    q, torch, dev, tab = env
    d, m = 6, 8
    if n in tab:
        z = [int(v) for v in tab.z_for(n)[:d]]
    else:
        z = [pow(3, j, n) for j in range(d)]
    c, w = W.genz_params(fam, d, 31)
    D = O.shifts(41, m, d)
    f = q.Integrand.genz(fam, c, w)
    for a, b in [(0, 2000), (n // 3, n // 3 + 1500), (n - 1700, n)]:
        _, gre, _, _ = _gpu_sums(env, f, n, z, D, tr, i0=a, i1=b)
        o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D, i0=a, i1=b)
        assert np.all(np.abs((gre[:, 0] + gre[:, 1]) - (o["re"][:, 0] + o["re"][:, 1])) <= TOL * o["abs"])


@pytest.mark.parametrize("fam", [1, 3, 4])
@pytest.mark.parametrize("tr", [("baker",), ("korobov", 1), ("korobov", 2), ("korobov", 3),
                                ("korobov", 4)])
def test_bench_size_sampled_subranges(env, fam, tr):
    """At the benchmark's size (n = 10560653, m = 32, d = 10) and for each of its families
    and maps (integer and FP64 finishes both occur), the full-range GPU result is checked on
    sampled sub-ranges the oracle can afford, and the whole against the closed form."""
    q, torch, dev, tab = env
    n, d, m = 10560653, 10, 32
    c, w = W.genz_params(fam, d, 1)
    D = O.shifts(77, m, d)
    z = tab.z_for(n)[:d]
    f = q.Integrand.genz(fam, c, w)
    res, full, _, _ = _gpu_sums(env, f, n, z, D, tr)
    exact = CF.genz_exact(fam, c, w)
    assert abs(res[0] - exact) <= 6 * res[1] + 1e-13 * abs(exact)
    rng = np.random.default_rng(1)
    for _ in range(3):
        a = int(rng.integers(0, n - 3000))
        b = a + int(rng.integers(1, 3000))
        _, gre, _, _ = _gpu_sums(env, f, n, z, D, tr, i0=a, i1=b)
        o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D, i0=a, i1=b)
        assert np.all(np.abs((gre[:, 0] + gre[:, 1]) - (o["re"][:, 0] + o["re"][:, 1])) <= TOL * o["abs"])
