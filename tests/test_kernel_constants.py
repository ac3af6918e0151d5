"""Pins of the numerical constants the CUDA kernels carry as literals, against the
mathematics they stand for, recomputed here in 300-bit arithmetic (mpmath): the
table-driven exponential's 2^(j/64) table and its scalar constants, the quarter-wave cosine
table of the integer cos, its Taylor coefficients and 2 pi, and the double-double 1/(2 pi)
split.  Each literal must be the correctly rounded value at its stated scale; a wrong
digit in any of them fails here, on the CPU, before any GPU run.  (The kernels' use of
these constants is covered by the GPU parity tests.)"""
from __future__ import annotations

import os
import re

import pytest

mp = pytest.importorskip("mpmath")
mp.mp.prec = 300

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1811_11720_gb300", "csrc")


def _read(name: str) -> str:
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _table(src: str, name: str) -> list[int]:
    m = re.search(name + r"\[\d+\]\s*=\s*\{(.*?)\};", src, re.S)
    assert m, name
    return [int(v, 16) for v in re.findall(r"0x([0-9a-fA-F]+)ull", m.group(1))]


def _const(src: str, name: str) -> int:
    m = re.search(r"constexpr uint64_t " + name + r"\s*=\s*0x([0-9a-fA-F]+)ull", src)
    assert m, name
    return int(m.group(1), 16)


def _nint(x) -> int:
    return int(mp.nint(x))


def test_exp2_fixed_table():
    t = _table(_read("qmc_exp.cuh"), "kExp2Fixed")
    assert len(t) == 64
    for j, v in enumerate(t):
        assert v == _nint(mp.power(2, mp.mpf(j) / 64) * mp.mpf(2) ** 63), j


def test_exp2_fixed_table_rounds_to_the_double_table():
    """The FP64 form's 2^(j/32) (even entries rounded to 53 bits) are the correctly
    rounded doubles."""
    t = _table(_read("qmc_exp.cuh"), "kExp2Fixed")
    for j in range(32):
        v = t[2 * j]
        mant, rest = v >> 11, v & 0x7FF
        if rest > 0x400 or (rest == 0x400 and mant & 1):
            mant += 1
        assert mant * 2.0 ** -52 == float(mp.power(2, mp.mpf(j) / 32)), j


def test_exp_fixed_scalars():
    src = _read("qmc_exp.cuh")
    two = mp.mpf(2)
    assert _const(src, "kLog2e") == _nint(two ** 63 / mp.log(2))
    assert _const(src, "kLn2") == _nint(mp.log(2) * two ** 64)
    for k in range(2, 7):
        assert _const(src, f"kD{k}") == _nint(two ** (64 - 6 * (k - 1)) / mp.factorial(k)), k


def test_cos_table_and_scalars():
    src = _read("qmc_cos.cuh")
    t = _table(src, "kCos256")
    assert len(t) == 65
    for i, v in enumerate(t):
        assert v == _nint(mp.cos(2 * mp.pi * i / 256) * mp.mpf(2) ** 62), i
    two = mp.mpf(2)
    assert _const(src, "k2Pi") == _nint(2 * mp.pi * two ** 61)
    assert _const(src, "kC6") == _nint(two ** 64 / 6)
    assert _const(src, "kC24") == _nint(two ** 64 / 24)
    assert _const(src, "kK120") == _nint(two ** 54 / 120)
    assert _const(src, "kK720") == _nint(two ** 54 / 720)


def test_inverse_two_pi_split():
    src = _read("qmc_integrands.cuh")
    hi = float.fromhex(re.search(r"kInv2PiHi = (-?0x[0-9a-fA-Fp.+-]+);", src).group(1))
    lo = float.fromhex(re.search(r"kInv2PiLo = (-?0x[0-9a-fA-Fp.+-]+);", src).group(1))
    x = 1 / (2 * mp.pi)
    assert hi == float(x)
    assert lo == float(x - mp.mpf(hi))


def test_exp_table_reduction_constants():
    """The FP64 exp's 32/ln2 and the two-part ln2/32 of its argument reduction."""
    src = _read("qmc_exp.cuh")

    def dbl(name):
        return float.fromhex(re.search(name + r" = (0x[0-9a-fA-Fp.+-]+);", src).group(1))

    assert dbl("kInvL") == float(32 / mp.log(2))
    l1 = dbl("kL1")
    assert l1 == float(mp.log(2) / 32)
    assert dbl("kL2") == float(mp.log(2) / 32 - mp.mpf(l1))
