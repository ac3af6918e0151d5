"""CPU oracle for the randomly shifted rank-1 lattice rule (arXiv:1811.11720).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  It shares no code
with the CUDA path in ``paper_1811_11720_gb300/`` and imports nothing from it; the only
module both sides use is ``workloads`` (seeded parameter draws, no method arithmetic).

Layout:
  qmc_oracle.c      plain C: shifts (SplitMix64), exact lattice points, transforms,
                    PolySingular map, integrands, double-double per-shift sums,
                    evaluate() and the per-dimension |f| histogram
  lattice.py        lattice sizes, get_next_n, naive and FFT CBC, e^2(z)
  closed_forms.py   exact integrals (mpmath) and the lattice character-sum prediction
  fit.py            CDF pairs from the histogram and the PolySingular least-squares fit
  make_genvec_table.py   writes tables/cbc_korobov_a2_s10.txt with lattice.py

Parity status: every function is pinned by tests/test_oracle_*.py except the fit
(``fit.fit_polysingular``), whose output the paper does not print: parity unpinned
(pinned only by recovery of known parameters and by invariants).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

TRANSFORMS = {"none": 0, "baker": 1, "korobov": 2, "sidi": 3}

FAMILY = {"osc": 1, "product_peak": 2, "corner_peak": 3, "gaussian": 4, "c0": 5,
          "discontinuous": 6, "monomial": 10, "trig": 11, "feynman": 20, "sector": 21}


class _Integrand(C.Structure):
    _fields_ = [("family", C.c_int), ("d", C.c_int),
                ("c", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
                ("h", C.POINTER(C.c_int64)),
                ("nu", C.c_int), ("nf", C.c_int),
                ("ucoef", C.POINTER(C.c_double)), ("fcoef", C.POINTER(C.c_double)),
                ("uexp", C.POINTER(C.c_int32)), ("fexp", C.POINTER(C.c_int32)),
                ("pa", C.c_double), ("pb", C.c_double), ("lam", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u64, dbl, i32 = C.c_uint64, C.c_double, C.c_int
        P = C.POINTER
        L.oracle_splitmix64.argtypes = [u64, u64]
        L.oracle_splitmix64.restype = u64
        L.oracle_shifts.argtypes = [u64, i32, i32, P(u64)]
        L.oracle_index.argtypes = [u64, u64, u64]
        L.oracle_index.restype = u64
        L.oracle_point.argtypes = [u64, u64, u64]
        L.oracle_point.restype = dbl
        L.oracle_points.argtypes = [u64, P(u64), i32, P(u64), i32, u64, u64, P(dbl)]
        L.oracle_transform_eval.argtypes = [i32, i32, i32, dbl, P(dbl), P(dbl)]
        L.oracle_polysingular.argtypes = [P(dbl), dbl, P(dbl), P(dbl)]
        L.oracle_eval_g.argtypes = [P(_Integrand), i32, i32, i32, P(dbl), P(dbl), P(dbl), P(dbl)]
        L.oracle_shift_sums.argtypes = [P(_Integrand), i32, i32, i32, P(dbl), u64, P(u64), P(u64),
                                        i32, u64, u64, P(dbl), P(dbl), P(dbl), i32]
        L.oracle_shift_sums.restype = C.c_long
        L.oracle_evaluate.argtypes = [P(_Integrand), u64, P(u64), P(u64), u64, u64, P(dbl), P(dbl)]
        L.oracle_histogram.argtypes = [P(_Integrand), u64, P(u64), P(u64), i32, P(dbl)]
        L.oracle_feynman_parts.argtypes = [P(_Integrand), P(dbl), P(dbl), P(dbl), P(dbl), P(dbl),
                                           P(dbl), P(dbl), P(dbl), P(dbl)]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _u64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------------------
# shifts and points
# ----------------------------------------------------------------------------------------
def splitmix64(seed: int, t: int) -> int:
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), t))


def shifts(seed: int, m: int, d: int) -> np.ndarray:
    """53-bit integer shift numerators D[k, j]; Delta = D * 2^-53."""
    D = np.zeros((m, d), dtype=np.uint64)
    lib().oracle_shifts(seed & (2**64 - 1), m, d, _p(D, C.c_uint64))
    return D


def point(r: int, n: int, D: int) -> float:
    return float(lib().oracle_point(r, n, D))


def point_py(r: int, n: int, D: int) -> float:
    """The lattice point by its definition with Python integers: RN of the exact rational
    ((r 2^53 + D n) mod (n 2^53)) / (n 2^53).  CPython's int/int true division is
    correctly rounded (round half to even), so this is an implementation independent of
    the C long division."""
    M = n << 53
    return ((r << 53) + D * n) % M / M


def points(n: int, z, D, i0: int = 0, count: int | None = None) -> np.ndarray:
    """u[i - i0, k, j] for i0 <= i < i0 + count."""
    z = _u64(z)
    D = _u64(D)
    m, d = D.shape
    count = n - i0 if count is None else count
    out = np.empty((count, m, d))
    lib().oracle_points(n, _p(z, C.c_uint64), d, _p(D, C.c_uint64), m, i0, count, _p(out, C.c_double))
    return out


def transform_eval(kind: str, r0: int, r1: int, u: float):
    phi, w = C.c_double(), C.c_double()
    lib().oracle_transform_eval(TRANSFORMS[kind], r0, r1, u, C.byref(phi), C.byref(w))
    return phi.value, w.value


def polysingular(a, x: float):
    a = _f64(a)
    p, dp = C.c_double(), C.c_double()
    lib().oracle_polysingular(_p(a, C.c_double), x, C.byref(p), C.byref(dp))
    return p.value, dp.value


# ----------------------------------------------------------------------------------------
# integrands
# ----------------------------------------------------------------------------------------
@dataclass
class Integrand:
    """Oracle-side description of an integrand (keeps its arrays alive)."""
    family: str
    d: int
    c: np.ndarray | None = None
    w: np.ndarray | None = None
    h: np.ndarray | None = None
    ucoef: np.ndarray | None = None
    uexp: np.ndarray | None = None
    fcoef: np.ndarray | None = None
    fexp: np.ndarray | None = None
    pa: float = 1.0
    pb: float = 2.5
    lam: float = 0.0

    @property
    def is_complex(self) -> bool:
        return self.family == "feynman"

    def struct(self) -> _Integrand:
        s = _Integrand()
        s.family = FAMILY[self.family]
        s.d = self.d
        keep = []

        def arr(x, dt, ct):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            keep.append(a)
            return _p(a, ct)

        s.c = arr(self.c, np.float64, C.c_double)
        s.w = arr(self.w, np.float64, C.c_double)
        s.h = arr(self.h, np.int64, C.c_int64)
        s.nu = 0 if self.ucoef is None else len(self.ucoef)
        s.nf = 0 if self.fcoef is None else len(self.fcoef)
        s.ucoef = arr(self.ucoef, np.float64, C.c_double)
        s.fcoef = arr(self.fcoef, np.float64, C.c_double)
        s.uexp = arr(self.uexp, np.int32, C.c_int32)
        s.fexp = arr(self.fexp, np.int32, C.c_int32)
        s.pa, s.pb, s.lam = self.pa, self.pb, self.lam
        s._keep = keep
        return s


def genz(family: int, c, w) -> Integrand:
    name = {1: "osc", 2: "product_peak", 3: "corner_peak", 4: "gaussian", 5: "c0",
            6: "discontinuous"}[family]
    return Integrand(name, len(c), c=_f64(c), w=_f64(w))


def monomial(d: int) -> Integrand:
    return Integrand("monomial", d)


def trig(amp, h, theta) -> Integrand:
    return Integrand("trig", len(amp), c=_f64(amp), w=_f64(theta), h=np.asarray(h, np.int64))


def from_feynman(fl) -> Integrand:
    """Build from a ``workloads.FeynmanLike`` (complex when lam != 0 or ``complex``)."""
    fam = "feynman" if fl.lam != 0.0 else "sector"
    return Integrand(fam, fl.d, ucoef=fl.U.coef, uexp=fl.U.exps, fcoef=fl.F.coef,
                     fexp=fl.F.exps, pa=fl.a, pb=fl.b, lam=fl.lam)


def feynman_complex(fl) -> Integrand:
    return Integrand("feynman", fl.d, ucoef=fl.U.coef, uexp=fl.U.exps, fcoef=fl.F.coef,
                     fexp=fl.F.exps, pa=fl.a, pb=fl.b, lam=fl.lam)


def _tr(transform):
    kind = transform[0]
    r0 = transform[1] if len(transform) > 1 else 0
    r1 = transform[2] if len(transform) > 2 else r0
    return TRANSFORMS[kind], int(r0), int(r1)


def eval_g(f: Integrand, transform, u, fitp=None) -> complex:
    s = f.struct()
    u = _f64(u)
    fp = None if fitp is None else _f64(fitp)
    re, im = C.c_double(), C.c_double()
    k, r0, r1 = _tr(transform)
    lib().oracle_eval_g(C.byref(s), k, r0, r1, None if fp is None else _p(fp, C.c_double),
                        _p(u, C.c_double), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def shift_sums(f: Integrand, transform, n: int, z, D, fitp=None, i0: int = 0,
               i1: int | None = None, nthreads: int | None = None):
    """Per-shift sums over i0 <= i < i1 as double-double: returns dict with
    ``re`` (m, 2) [hi, lo], ``im`` (m, 2) or None, ``abs`` (m,) sum of |g| and the
    ``signfail`` count."""
    s = f.struct()
    z = _u64(z)
    D = _u64(D)
    m, d = D.shape
    assert d == f.d and len(z) >= d
    i1 = n if i1 is None else i1
    nthreads = os.cpu_count() if nthreads is None else nthreads
    fp = None if fitp is None else _f64(fitp)
    re = np.zeros((m, 2))
    im = np.zeros((m, 2)) if f.is_complex else None
    ab = np.zeros(m)
    k, r0, r1 = _tr(transform)
    fails = lib().oracle_shift_sums(C.byref(s), k, r0, r1,
                                    None if fp is None else _p(fp, C.c_double), n,
                                    _p(z, C.c_uint64), _p(D, C.c_uint64), m, i0, i1,
                                    _p(re, C.c_double),
                                    None if im is None else _p(im, C.c_double),
                                    _p(ab, C.c_double), nthreads)
    return {"re": re, "im": im, "abs": ab, "signfail": int(fails)}


def shift_reduce(Q) -> tuple:
    """Eq. (lattice) and Eq. (lattice-error): Qbar = mean_k Q^(k) and
    sigma = sqrt(sum_k (Q^(k) - Qbar)^2 / (m (m - 1))), per real component."""
    Q = np.asarray(Q, dtype=np.float64)
    m = Q.shape[0]
    qbar = Q.sum() / m
    var = ((Q - qbar) ** 2).sum() / (m * (m - 1))
    return float(qbar), float(np.sqrt(var))


def integrate(f: Integrand, transform, n: int, z, D, fitp=None, nthreads=None):
    """Fixed-lattice estimate: per-shift Q^(k) = S_k / n, their mean and standard error."""
    r = shift_sums(f, transform, n, z, D, fitp=fitp, nthreads=nthreads)
    Qre = (r["re"][:, 0] + r["re"][:, 1]) / n
    out = {"Q_re": Qre, "sums_re": r["re"], "signfail": r["signfail"], "A": r["abs"] / n}
    out["value_re"], out["error_re"] = shift_reduce(Qre)
    if r["im"] is not None:
        Qim = (r["im"][:, 0] + r["im"][:, 1]) / n
        out["Q_im"] = Qim
        out["sums_im"] = r["im"]
        out["value_im"], out["error_im"] = shift_reduce(Qim)
    return out


def evaluate(f: Integrand, n: int, z, D1, i0: int = 0, count: int | None = None):
    """Raw samples f(x_i) on one shifted lattice (the paper's evaluate(), App. A.2)."""
    s = f.struct()
    z = _u64(z)
    D1 = _u64(D1).reshape(-1)
    count = n - i0 if count is None else count
    re = np.empty(count)
    im = np.empty(count) if f.is_complex else None
    lib().oracle_evaluate(C.byref(s), n, _p(z, C.c_uint64), _p(D1, C.c_uint64), i0, count,
                          _p(re, C.c_double), None if im is None else _p(im, C.c_double))
    return re if im is None else re + 1j * im


def histogram(f: Integrand, n: int, z, D1, bins: int) -> np.ndarray:
    """hist[j, b] = sum of |f(x_i)| over lattice points with floor(x_ij * bins) == b."""
    s = f.struct()
    z = _u64(z)
    D1 = _u64(D1).reshape(-1)
    h = np.zeros((f.d, bins))
    lib().oracle_histogram(C.byref(s), n, _p(z, C.c_uint64), _p(D1, C.c_uint64), bins,
                           _p(h, C.c_double))
    return h


def feynman_parts(f: Integrand, x):
    """Deformed point z, Jacobian J, U(z), F(z), det J and real F, grad F, Hessian at x."""
    s = f.struct()
    d = f.d
    x = _f64(x)
    z = np.zeros(2 * d)
    J = np.zeros(2 * d * d)
    U = np.zeros(2)
    F = np.zeros(2)
    det = np.zeros(2)
    Fr = C.c_double()
    g = np.zeros(d)
    H = np.zeros(d * d)
    pd = lambda a: _p(a, C.c_double)  # noqa: E731
    lib().oracle_feynman_parts(C.byref(s), pd(x), pd(z), pd(J), pd(U), pd(F), pd(det),
                               C.byref(Fr), pd(g), pd(H))
    return {"z": z[0::2] + 1j * z[1::2], "J": (J[0::2] + 1j * J[1::2]).reshape(d, d),
            "U": complex(*U), "F": complex(*F), "det": complex(*det), "F_real": Fr.value,
            "grad": g, "hess": H.reshape(d, d)}


def load_genvec_table(path: str) -> dict:
    """Read 'n z_1 .. z_s' lines into {n: [z...]}."""
    tab = {}
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = [int(t) for t in line.split()]
                tab[v[0]] = v[1:]
    return tab
