"""Pins for lattice sizes and the CBC construction (Sec. 2.2; App. A.1, A.3) and for the
generating-vector table both paths load."""
import math
import os

import numpy as np
import pytest

import oracle as O
from conftest import TABLE, golden
from oracle import lattice as L


def test_sizes_follow_the_paper_rule():
    kv = {}
    for line in open(golden("lattice_sizes.txt")):
        if not line.startswith("#"):
            k, v = line.split()
            kv[k] = int(v)
    sizes = L.lattice_sizes(kv["imax"])
    assert sizes[0] == kv["first"] and sizes[-1] == kv["last"]
    for n in sizes:
        assert L.is_prime(n)
    assert L.get_next_n(sizes, 100000) == 108863
    assert L.get_next_n(sizes, 1021) == 1021
    with pytest.raises(ValueError):
        L.get_next_n(sizes, 2**31)


def test_miller_rabin_against_trial_division():
    def slow(n):
        if n < 2:
            return False
        for p in range(2, int(math.isqrt(n)) + 1):
            if n % p == 0:
                return False
        return True
    for n in range(0, 20000):
        assert L.is_prime(n) == slow(n)
    for n in [2**31 - 1, 2**61 - 1, 1024565021, 1024565023]:
        assert L.is_prime(n) == slow(n) if n < 10**10 else L.is_prime(n)


def test_first_component_closed_form():
    """e^2 of the 1-D lattice z = 1: by the Fourier series omega(x) = sum_{h!=0} e^{2 pi i h x}/h^2,
    only h = multiples of n survive, so e^2 = gamma * 2 zeta(2) / n^2 = gamma pi^2 / (3 n^2)."""
    for n, s in [(7, 2), (11, 3), (1021, 10)]:
        _, e2 = L.cbc_naive(n, s)
        assert abs(e2[0] - (1.0 / s) * math.pi**2 / (3 * n * n)) < 1e-15


def _e2_two_dim_fourier(n, z2, gamma, beta=1.0):
    """1 + e^2 = sum over residues b of S(b) S(-b z2 mod n), where
    S(c) = sum_{h = c (mod n)} r(h), r(0) = beta, r(h != 0) = gamma / h^2, evaluated with
    sum_k 1/(a + k n)^2 = (pi/n)^2 / sin^2(pi a / n).  Independent of the kernel sum."""
    def S(c):
        c %= n
        if c == 0:
            return beta + gamma * math.pi**2 / (3 * n * n)
        return gamma * (math.pi / n) ** 2 / math.sin(math.pi * c / n) ** 2
    return math.fsum(S(b) * S(-b * z2) for b in range(n)) - 1.0


@pytest.mark.parametrize("n", [7, 11, 101, 1021])
def test_two_dim_error_matches_dual_lattice_sum(n):
    s = 2
    z, e2 = L.cbc_naive(n, s)
    assert abs(e2[1] - _e2_two_dim_fourier(n, z[1], 1.0 / s)) < 1e-13
    # and the chosen z2 is a minimiser of that independent formula
    best = min(_e2_two_dim_fourier(n, c, 1.0 / s) for c in range(1, n))
    assert _e2_two_dim_fourier(n, z[1], 1.0 / s) <= best + 1e-14


@pytest.mark.parametrize("n", [7, 11, 13, 101, 1021, 1123, 4099, 7919])
def test_fast_cbc_equals_naive(n):
    s = 2 if n < 20 else 10
    zn, en = L.cbc_naive(n, s)
    zf, ef = L.cbc_fast(n, s)
    assert zn == zf
    assert np.allclose(en, ef, rtol=0, atol=1e-14)


def test_cbc_e2_equals_direct_recomputation():
    n = 4099
    z, e2 = L.cbc_fast(n, 6)
    for j in range(1, 7):
        assert abs(L.worst_case_error_sq(n, z[:j], s_weights=6) - e2[j - 1]) < 1e-14


def test_table_file(genvec_table):
    assert os.path.exists(TABLE)
    sizes = set(L.lattice_sizes())
    for n, z in genvec_table.items():
        assert n in sizes
        assert len(z) == 10 and z[0] == 1
        assert all(0 < v <= (n - 1) // 2 and math.gcd(v, n) == 1 for v in z)
    # the decades used by the workloads are present
    for need in (1021, 108863, 1072187, 10560653):
        assert need in genvec_table


@pytest.mark.parametrize("n", [1021, 1123, 4691, 108863])
def test_table_entries_reproduce(genvec_table, n):
    z = (L.cbc_naive if n <= 5000 else L.cbc_fast)(n, 10)[0]
    assert z == genvec_table[n]


def test_rank1_lattice_integrates_trig_exactly_for_table(genvec_table):
    """e^2 of a table vector is small and decreasing in n (better lattices for larger n)."""
    prev = None
    for n in sorted(genvec_table)[:12]:
        e = L.worst_case_error_sq(n, genvec_table[n][:4], s_weights=10)
        assert e > 0
        if prev is not None:
            assert e < prev * 1.5
        prev = e


def test_extension_table_file():
    """The GPU-built rows beyond the CPU table: the paper's remaining sizes up to 2^31 - 1,
    well-formed vectors, and the whole size rule covered by the two files together."""
    ext = os.path.join(os.path.dirname(TABLE), "cbc_korobov_a2_s10_gpu.txt")
    rows = O.load_genvec_table(ext)
    main = O.load_genvec_table(TABLE)
    sizes = L.lattice_sizes()
    assert sorted(set(rows) | set(main)) == sorted(sizes)
    assert min(rows) > max(main)
    for n, z in rows.items():
        assert L.is_prime(n)
        assert len(z) == 10 and z[0] == 1
        assert all(0 < v <= (n - 1) // 2 for v in z)


def test_extension_size_rule_matches_oracle():
    """The package's own size rule (used to extend the table) equals the oracle's."""
    from paper_1811_11720_gb300.extend_table import table_sizes
    assert table_sizes() == L.lattice_sizes()


def test_loader_roundtrip(tmp_path):
    p = tmp_path / "t.txt"
    p.write_text("# x\n7 1 3\n11 1 7\n")
    assert O.load_genvec_table(str(p)) == {7: [1, 3], 11: [1, 7]}
