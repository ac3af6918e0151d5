"""Pins for the oracle's shifts and lattice points (Eq. (lattice), Fig. 1)."""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import golden


def _read_kv(path):
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = [int(t) for t in v]
    return out


def test_point_matches_correctly_rounded_python_division():
    rng = random.Random(7)
    ns = [7, 11, 55, 1021, 108863, 1024565021, 2**31 - 1, (1 << 40) + 15, (1 << 61) - 1,
          (1 << 63) + 29]
    for _ in range(20000):
        n = rng.choice(ns)
        r = rng.randrange(n) if rng.random() > 0.05 else rng.choice([0, 1, n - 1])
        D = rng.randrange(1 << 53) if rng.random() > 0.1 else rng.randrange(8)
        assert O.point(r, n, D) == O.point_py(r, n, D), (r, n, D)


def test_point_is_nearest_double_brute_force():
    """Against exact rationals: the result is within half an ulp and no neighbouring
    double is closer (ties to even)."""
    rng = random.Random(3)
    for _ in range(3000):
        n = rng.choice([7, 11, 55, 1021, 1 << 20 | 1, 999999937])
        r = rng.randrange(n)
        D = rng.randrange(1 << 53)
        exact = Fraction(r, n) + Fraction(D, 1 << 53)
        exact -= int(exact)
        u = O.point(r, n, D)
        err = abs(Fraction(u) - exact)
        for nb in (np.nextafter(u, 0.0), np.nextafter(u, 2.0)):
            assert err <= abs(Fraction(float(nb)) - exact)


def test_fig1_lattice_unshifted():
    """Fig. 1: n = 55, z = (1, 34); with zero shift the points are (i/55, {34 i/55})."""
    kv = _read_kv(golden("fig1_lattice.txt"))
    n, z = kv["n"][0], kv["z"]
    D = np.zeros((1, 2), dtype=np.uint64)
    pts = O.points(n, z, D)[:, 0, :]
    for i in range(n):
        assert pts[i, 0] == i / n
        assert pts[i, 1] == (34 * i % 55) / 55
    # all 55 points distinct and each coordinate visits every multiple of 1/55 once
    assert len({tuple(p) for p in pts}) == n
    assert sorted(np.round(pts[:, 1] * n).astype(int)) == list(range(n))


def test_index_permutation_and_reflection(genvec_table):
    n = 1021
    z = genvec_table[n]
    for zj in z:
        r = [int(O.lib().oracle_index(i, zj, n)) for i in range(n)]
        assert sorted(r) == list(range(n))          # z_j coprime to n: a permutation
        assert all(r[n - i] == (n - r[i]) % n for i in range(1, n))


def test_shift_adds_mod_one():
    """frac(r/n + Delta) wraps: a point plus a shift of 1 - r/n lands on 0."""
    n = 55
    for r in range(1, n):
        # D chosen so that Delta is the double nearest 1 - r/n; exact rational check
        D = int(round((1 - r / n) * 2**53))
        u = O.point(r, n, D)
        exact = (Fraction(r, n) + Fraction(D, 1 << 53)) % 1
        assert abs(Fraction(u) - exact) <= Fraction(1, 1 << 54)


def test_point_can_round_up_to_one():
    """A fraction within half an ulp of 1 rounds to 1.0 (documented reading)."""
    n = 6361                        # divides 2^53 - 1
    r = n - 1
    D = ((1 << 53) - 1) // n        # 1 - (r/n + D 2^-53) = 1/(n 2^53) < 2^-54
    exact = Fraction(r, n) + Fraction(D, 1 << 53)
    assert 1 - exact == Fraction(1, n << 53)
    assert O.point(r, n, D) == 1.0 == O.point_py(r, n, D)


def test_shifts_uniform_and_in_range():
    D = O.shifts(12345, 4096, 8)
    assert D.dtype == np.uint64
    assert int(D.max()) < (1 << 53)
    x = D.astype(np.float64) / 2.0**53
    assert abs(x.mean() - 0.5) < 0.01
    hist, _ = np.histogram(x, bins=16, range=(0, 1))
    expected = x.size / 16
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 50.0            # 15 dof; p ~ 1e-5 threshold
    # different seeds and different (k, j) give different streams
    D2 = O.shifts(12346, 4096, 8)
    assert (D != D2).mean() > 0.99
    assert len(np.unique(D)) == D.size


def test_shifts_row_major_stream():
    """Delta_{k,j} is output number k*d + j of one stream: a (m, d) draw equals the
    first m*d outputs reshaped."""
    D = O.shifts(99, 5, 3)
    flat = [O.splitmix64(99, t) >> 11 for t in range(15)]
    assert D.reshape(-1).tolist() == flat


@pytest.mark.parametrize("n", [7, 11])
def test_custom_genvecs_paper_example(n):
    """App. A.3 custom vectors {7: (1,3), 11: (1,7)}: the rule integrates constants
    exactly and points form a permutation in each coordinate."""
    tab = {}
    for line in open(golden("custom_genvecs.txt")):
        if line.startswith("#"):
            continue
        v = [int(t) for t in line.split()]
        tab[v[0]] = v[1:]
    z = tab[n]
    D = np.zeros((1, 2), dtype=np.uint64)
    pts = O.points(n, z, D)[:, 0, :]
    for j in range(2):
        assert sorted(np.round(pts[:, j] * n).astype(int)) == list(range(n))


def test_splitmix64_published_reference_outputs():
    """The shift generator is SplitMix64 (Steele, Lea, Flood 2014): its first outputs for
    two seeds equal the published reference implementation's test vectors
    (tests/golden/splitmix64_reference.txt), so a mistyped increment or mixing constant
    fails here rather than agreeing with itself on both sides of the parity tests."""
    rows = [line.split() for line in open(golden("splitmix64_reference.txt"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        seed, outs = int(row[0]), [int(v) for v in row[1:]]
        assert [O.splitmix64(seed, t) for t in range(len(outs))] == outs
        # the shift numerators are those outputs >> 11, in row-major [k][j] order
        D = O.shifts(seed, 1, len(outs))
        assert D.reshape(-1).tolist() == [v >> 11 for v in outs]
