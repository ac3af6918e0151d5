"""GB300 randomly shifted rank-1 lattice quadrature (arXiv:1811.11720) -- Python binding.

Thin marshalling over the C ABI in include/qmc_gb300.h (libqmc_gb300.so, built by
``paper_1811_11720_gb300.build``).  Every step of the quadrature runs in the library's
CUDA kernels; PyTorch only provides device memory and streams for the device entry
points.  Importing works without a GPU; calling an entry point without the built library
raises ImportError (there is no CPU fallback).

Functions keep the C names without the ``qmc_`` prefix:
  get_next_n, make_shifts, points, sums_workspace_bytes, sums, finalize, evaluate,
  histogram_workspace_bytes, histogram, fit_polysingular, integrate
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import _capi
from ._capi import (FAMILY, QMC_MAX_DIM, STATUS, TRANSFORM, qmc_batch_config, qmc_batch_item,
                    qmc_fit_opts, qmc_genvec_table, qmc_integrand, qmc_options, qmc_result,
                    qmc_rule, qmc_server_config, qmc_transform)

__all__ = ["QMCError", "lib", "GenvecTable", "Integrand", "make_transform", "get_next_n",
           "make_shifts", "rule", "points", "sums_workspace_bytes", "sums", "sums_noalloc",
           "sums_tile_count", "sums_tiles", "reduce_tiles",
           "finalize", "probe_units",
           "evaluate", "histogram_workspace_bytes", "histogram", "fit_polysingular",
           "integrate", "integrate_device", "Batch", "Server", "cbc_korobov", "DEFAULT_TABLE",
           "EXTENSION_TABLE"]

_TABLES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tables")
DEFAULT_TABLE = os.path.join(_TABLES, "cbc_korobov_a2_s10.txt")
# sizes past the CPU-built table, computed with qmc_cbc_korobov (extend_table.py)
EXTENSION_TABLE = os.path.join(_TABLES, "cbc_korobov_a2_s10_gpu.txt")

_lib = None


class QMCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.qmc_strerror(code).decode() if _lib is not None else STATUS.get(code, "?")
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = _capi.load()
    return _lib


def _check(code: int, where: str, allow=()):
    if code != 0 and code not in allow:
        raise QMCError(code, where)
    return code


def _ptr(x) -> int | None:
    """Raw address of a numpy array or torch tensor (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------------------------------
class GenvecTable:
    """Generating-vector table: ascending sizes n[c] and rows z[c, :s_max]."""

    def __init__(self, n, z):
        self.n = np.ascontiguousarray(np.asarray(n, dtype=np.uint64))
        self.z = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
        order = np.argsort(self.n)
        self.n = np.ascontiguousarray(self.n[order])
        self.z = np.ascontiguousarray(self.z[order])
        self.struct = qmc_genvec_table(self.n.ctypes.data, self.z.ctypes.data,
                                       int(self.z.shape[1]), int(self.n.shape[0]))

    @classmethod
    def load(cls, path: str | None = None, extension: bool = True) -> "GenvecTable":
        """Rows "n z_1 .. z_s" ('#' comments).  Default: the shipped table plus, when
        present, its extension to larger n; a size in both keeps the first file's row."""
        paths = [path or DEFAULT_TABLE]
        if path is None and extension and os.path.exists(EXTENSION_TABLE):
            paths.append(EXTENSION_TABLE)
        rows, seen = [], set()
        for pth in paths:
            with open(pth) as fh:
                for line in fh:
                    if line.strip() and not line.startswith("#"):
                        r = [int(t) for t in line.split()]
                        if r[0] not in seen:
                            seen.add(r[0])
                            rows.append(r)
        s = min(len(r) - 1 for r in rows)
        return cls([r[0] for r in rows], [r[1:1 + s] for r in rows])

    def z_for(self, n: int) -> np.ndarray:
        idx = np.nonzero(self.n == np.uint64(n))[0]
        if idx.size == 0:
            raise KeyError(n)
        return self.z[idx[0]]

    def __contains__(self, n) -> bool:
        return bool(np.any(self.n == np.uint64(n)))


def make_transform(spec) -> qmc_transform:
    """('korobov', r) | ('korobov', r0, r1) | ('sidi', r) | ('baker',) | ('none',)."""
    if isinstance(spec, qmc_transform):
        return spec
    if isinstance(spec, str):
        spec = (spec,)
    kind = spec[0]
    r0 = int(spec[1]) if len(spec) > 1 else 0
    r1 = int(spec[2]) if len(spec) > 2 else r0
    return qmc_transform(TRANSFORM[kind], r0, r1)


@dataclass
class Integrand:
    """Integrand description; arrays are host numpy arrays (see ``to_device``)."""
    family: str
    dim: int
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
    _dev: dict = field(default_factory=dict, repr=False)

    @property
    def is_complex(self) -> bool:
        return self.family == "feynman"

    @staticmethod
    def genz(family: int, c, w) -> "Integrand":
        name = {1: "oscillatory", 2: "product_peak", 3: "corner_peak", 4: "gaussian", 5: "c0",
                6: "discontinuous"}[family]
        c = np.ascontiguousarray(c, dtype=np.float64)
        return Integrand(name, len(c), c=c, w=np.ascontiguousarray(w, dtype=np.float64))

    @staticmethod
    def monomial(d: int) -> "Integrand":
        return Integrand("monomial", d)

    @staticmethod
    def trig(amp, h, theta) -> "Integrand":
        return Integrand("trig", len(amp), c=np.ascontiguousarray(amp, np.float64),
                         w=np.ascontiguousarray(theta, np.float64),
                         h=np.ascontiguousarray(h, np.int64))

    @staticmethod
    def polynomial(fl, complex_: bool | None = None) -> "Integrand":
        """From a workloads.FeynmanLike: complex deformed family when lam != 0 (or when
        ``complex_`` is True), real sector family otherwise."""
        cplx = (fl.lam != 0.0) if complex_ is None else complex_
        return Integrand("feynman" if cplx else "sector", fl.d,
                         ucoef=np.ascontiguousarray(fl.U.coef, np.float64),
                         uexp=np.ascontiguousarray(fl.U.exps, np.int32),
                         fcoef=np.ascontiguousarray(fl.F.coef, np.float64),
                         fexp=np.ascontiguousarray(fl.F.exps, np.int32),
                         pa=float(fl.a), pb=float(fl.b), lam=float(fl.lam))

    def _struct(self, arrs) -> qmc_integrand:
        s = qmc_integrand()
        s.family = FAMILY[self.family]
        s.dim = self.dim
        s.c, s.w, s.h = _ptr(arrs["c"]), _ptr(arrs["w"]), _ptr(arrs["h"])
        s.nu = 0 if self.ucoef is None else len(self.ucoef)
        s.nf = 0 if self.fcoef is None else len(self.fcoef)
        s.ucoef, s.fcoef = _ptr(arrs["ucoef"]), _ptr(arrs["fcoef"])
        s.uexp, s.fexp = _ptr(arrs["uexp"]), _ptr(arrs["fexp"])
        s.pa, s.pb, s.lambda_ = self.pa, self.pb, self.lam
        s._keep = arrs   # the struct holds raw addresses: keep the arrays alive with it
        return s

    def _arrays(self) -> dict:
        return {k: getattr(self, k) for k in ("c", "w", "h", "ucoef", "uexp", "fcoef", "fexp")}

    def host_struct(self) -> qmc_integrand:
        return self._struct(self._arrays())

    def device_struct(self, device="cuda") -> qmc_integrand:
        """Copies the arrays to ``device`` (cached) and returns a struct of device pointers."""
        import torch
        key = str(device)
        if key not in self._dev:
            arrs = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).to(device))
                    for k, v in self._arrays().items()}
            self._dev[key] = arrs
        return self._struct(self._dev[key])


# ----------------------------------------------------------------------------------------
def get_next_n(table: GenvecTable, preferred: int) -> int:
    out = C.c_uint64()
    _check(lib().qmc_get_next_n(C.byref(table.struct), int(preferred), C.byref(out)), "get_next_n")
    return int(out.value)


def cbc_korobov(n: int, s: int, gamma: float | None = None, beta: float = 1.0, stream=None):
    """Fast CBC generating vector on the device (qmc_cbc_korobov): returns (z, e2), the
    s components and the squared worst-case error after each.  gamma defaults to 1/s."""
    z = np.zeros(s, dtype=np.uint64)
    e2 = np.zeros(s)
    g = float(gamma) if gamma is not None else (1.0 / s if s > 0 else 0.0)
    _check(lib().qmc_cbc_korobov(int(n), int(s), g, float(beta),
                                 z.ctypes.data_as(C.POINTER(C.c_uint64)),
                                 e2.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)),
           "cbc_korobov")
    return z, e2


def make_shifts(seed: int, m: int, d: int) -> np.ndarray:
    D = np.zeros((m, d), dtype=np.uint64)
    _check(lib().qmc_make_shifts(int(seed) & (2**64 - 1), m, d, D.ctypes.data), "make_shifts")
    return D


def rule(n: int, z, shifts_dev, transform=("none",), fit_dev=None) -> qmc_rule:
    """A qmc_rule over device shifts ``shifts_dev`` (m x d uint64 tensor)."""
    r = qmc_rule()
    r.n = int(n)
    z = [int(v) for v in z]
    m, d = int(shifts_dev.shape[0]), int(shifts_dev.shape[1])
    r.dim = d
    for j in range(d):
        r.z[j] = z[j]
    r.m = m
    r.shifts = _ptr(shifts_dev)
    r.transform = make_transform(transform)
    r.fit = _ptr(fit_dev)
    r._keep = (shifts_dev, fit_dev)
    return r


def points(r: qmc_rule, i_begin: int, count: int, out, stream=None):
    _check(lib().qmc_points(C.byref(r), int(i_begin), int(count), _ptr(out), _stream(stream)), "points")
    return out


def sums_workspace_bytes(r: qmc_rule, is_complex: bool, i_begin: int, i_end: int) -> int:
    return int(lib().qmc_sums_workspace_bytes(C.byref(r), int(bool(is_complex)), int(i_begin), int(i_end)))


def sums(f: qmc_integrand, r: qmc_rule, i_begin: int, i_end: int, workspace, out, counters=None,
         stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().qmc_sums(C.byref(f), C.byref(r), int(i_begin), int(i_end), _ptr(workspace), nbytes,
                          _ptr(out), _ptr(counters), _stream(stream)), "sums")
    return out


def sums_tile_count(range_len: int, m: int) -> tuple[int, int]:
    """qmc_sums_tile_count: (tiles, points per tile) of qmc_sums' decomposition."""
    t, ppt = C.c_uint64(), C.c_uint64()
    _check(lib().qmc_sums_tile_count(int(range_len), int(m), C.byref(t), C.byref(ppt)),
           "sums_tile_count")
    return int(t.value), int(ppt.value)


def sums_tiles(f: qmc_integrand, r: qmc_rule, i_begin: int, i_end: int, tile_begin: int,
               tile_end: int, partials, counters=None, stream=None):
    """qmc_sums_tiles: partials of tiles [tile_begin, tile_end) of [i_begin, i_end)
    (device tensor of 2 m T doubles, 4 m T complex)."""
    _check(lib().qmc_sums_tiles(C.byref(f), C.byref(r), int(i_begin), int(i_end), int(tile_begin),
                                int(tile_end), _ptr(partials), _ptr(counters), _stream(stream)),
           "sums_tiles")
    return partials


def reduce_tiles(partials, tiles: int, m: int, is_complex: bool, out, stream=None):
    """qmc_reduce_tiles: the fixed-order fold of tile partials into per-shift sums."""
    _check(lib().qmc_reduce_tiles(_ptr(partials), int(tiles), int(m), int(bool(is_complex)),
                                  _ptr(out), _stream(stream)), "reduce_tiles")
    return out


def sums_noalloc(f: qmc_integrand, r: qmc_rule, i_begin: int, i_end: int, out, counters=None,
                 stream=None):
    """qmc_sums_noalloc: the per-shift sums with the library's fixed device scratch instead
    of a caller workspace, for callers that cannot allocate (graph capture, preallocated
    deployments).  Raises QMCError(QMC_ERR_WORKSPACE) when the problem needs more than
    QMC_NOALLOC_SCRATCH_BYTES of partials; calls on one device must not overlap."""
    _check(lib().qmc_sums_noalloc(C.byref(f), C.byref(r), int(i_begin), int(i_end), _ptr(out),
                                  _ptr(counters), _stream(stream)), "sums_noalloc")
    return out


PROBE_UNITS = {"fp64_fma": 1, "int_mulhi": 2}


def probe_units(unit: str, trips: int, sink, stream=None) -> float:
    """qmc_probe_units: enqueue one throughput probe of ``unit`` ("fp64_fma" or "int_mulhi")
    and return the operations it executes (time it with events on ``stream``)."""
    ops = C.c_double()
    _check(lib().qmc_probe_units(PROBE_UNITS[unit], int(trips), _ptr(sink), C.byref(ops),
                                 _stream(stream)), "probe_units")
    return float(ops.value)


def finalize(sums_dev, m: int, n: int, is_complex: bool, result, Q=None, stream=None):
    _check(lib().qmc_finalize(_ptr(sums_dev), int(m), int(n), int(bool(is_complex)), _ptr(result),
                              _ptr(Q), _stream(stream)), "finalize")
    return result


def evaluate(f: qmc_integrand, n: int, z, shift_dev, i_begin: int, count: int, out, stream=None):
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    _check(lib().qmc_evaluate(C.byref(f), int(n), zz.ctypes.data, int(f.dim), _ptr(shift_dev),
                              int(i_begin), int(count), _ptr(out), _stream(stream)), "evaluate")
    return out


def histogram_workspace_bytes(n: int, dim: int, bins: int) -> int:
    return int(lib().qmc_histogram_workspace_bytes(int(n), int(dim), int(bins)))


def histogram(f: qmc_integrand, n: int, z, shift_dev, bins: int, hist, workspace, stream=None):
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.uint64))
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().qmc_histogram(C.byref(f), int(n), zz.ctypes.data, int(f.dim), _ptr(shift_dev),
                               int(bins), _ptr(hist), _ptr(workspace), nbytes, _stream(stream)),
           "histogram")
    return hist


def fit_options(enabled=True, evaluateminn=100000, bins=1000, maxiter=40, xtol=3e-3, gtol=1e-8,
                ftol=1e-8, stepsize=10) -> qmc_fit_opts:
    return qmc_fit_opts(int(enabled), int(evaluateminn), int(bins), int(maxiter), float(xtol),
                        float(gtol), float(ftol), int(stepsize))


def fit_polysingular(hist: np.ndarray, opts: qmc_fit_opts | None = None) -> np.ndarray:
    h = np.ascontiguousarray(np.asarray(hist, dtype=np.float64))
    d, bins = h.shape
    out = np.zeros((d, 6))
    _check(lib().qmc_fit_polysingular(h.ctypes.data, d, bins, None if opts is None else C.byref(opts),
                                      out.ctypes.data), "fit_polysingular")
    return out


def options(epsrel=0.01, epsabs=1e-7, maxeval=1_000_000, errormode="all") -> qmc_options:
    """Defaults of App. A.1 (epsrel 0.01, epsabs 1e-7, maxeval 1e6, errormode all)."""
    return qmc_options(float(epsrel), float(epsabs), int(maxeval), _capi.ERRORMODE[errormode])


def integrate(f: Integrand, table: GenvecTable, n: int, m: int, transform, fit=None, seed: int = 0,
              opts: qmc_options | None = None, stream=None) -> dict:
    """Host-buffer integrate (qmc_integrate).  ``opts`` None: fixed lattice of size
    get_next_n(n); otherwise adaptive from get_next_n(n)."""
    res = qmc_result()
    fs = f.host_struct()
    code = lib().qmc_integrate(C.byref(fs), C.byref(table.struct), int(n), int(m),
                               make_transform(transform), None if fit is None else C.byref(fit),
                               int(seed) & (2**64 - 1), None if opts is None else C.byref(opts),
                               _stream(stream), C.byref(res))
    _check(code, "integrate", allow=(_capi.QMC_ERR_NONFINITE,))
    return {"integral": complex(res.integral.re, res.integral.im),
            "error": complex(res.error.re, res.error.im),
            "value": res.integral.re, "err": res.error.re,
            "n": res.n, "m": res.m, "iterations": res.iterations, "evaluations": res.evaluations,
            "nonfinite": res.nonfinite, "signfail": res.signfail, "status": code}


def integrate_device(f: Integrand, n: int, z, shifts_dev, transform, fit_dev=None, i_begin=0,
                     i_end=None, workspace=None, stream=None):
    """Device-resident pass: qmc_sums over [i_begin, i_end) then qmc_finalize.  Returns
    (result[4], sums[2m or 4m], counters[2]) as device tensors; allocations go through
    torch (pass ``workspace`` to reuse one)."""
    import torch
    dev = shifts_dev.device
    r = rule(n, z, shifts_dev, transform, fit_dev)
    i_end = n if i_end is None else i_end
    need = sums_workspace_bytes(r, f.is_complex, i_begin, i_end)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 8), dtype=torch.uint8, device=dev)
    m = int(shifts_dev.shape[0])
    out = torch.empty(4 * m, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    res = torch.empty(4, dtype=torch.float64, device=dev)
    fd = f.device_struct(dev)
    sums(fd, r, i_begin, i_end, workspace, out, cnt, stream)
    finalize(out, m, n, f.is_complex, res, None, stream)
    return res, out, cnt


# ----------------------------------------------------------------------------------------
class Batch:
    """Many integrals of one family and one m in a single launch (qmc_batch_sums).

    ``entries``: list of (qmc_integrand with device arrays, qmc_rule, i_begin, i_end).
    The structs (and the tensors they point to) are kept alive by this object."""

    def __init__(self, entries):
        self.count = len(entries)
        self.arr = (qmc_batch_item * self.count)()
        for i, (fs, r, a, b) in enumerate(entries):
            self.arr[i].f = fs
            self.arr[i].rule = r
            self.arr[i].i_begin = int(a)
            self.arr[i].i_end = int(b)
        self._keep = entries
        self.m = int(entries[0][1].m)

    def workspace_bytes(self, cfg: qmc_batch_config | None = None) -> int:
        return int(lib().qmc_batch_workspace_bytes(self.arr, self.count,
                                                   None if cfg is None else C.byref(cfg)))

    def sums(self, workspace, sums, results=None, counters=None, cfg=None, stream=None):
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().qmc_batch_sums(self.arr, self.count, None if cfg is None else C.byref(cfg),
                                    _ptr(workspace), nbytes, _ptr(sums), _ptr(results),
                                    _ptr(counters), _stream(stream)), "batch_sums")
        return sums

    def autotune(self, workspace, sums, stream=None) -> qmc_batch_config:
        best = qmc_batch_config()
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().qmc_batch_autotune(self.arr, self.count, _ptr(workspace), nbytes, _ptr(sums),
                                        _stream(stream), C.byref(best)), "batch_autotune")
        return best

    def plan(self, workspace, cfg=None, stream=None) -> "BatchPlan":
        h = C.c_void_p()
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().qmc_batch_plan_create(self.arr, self.count, None if cfg is None else C.byref(cfg),
                                           _ptr(workspace), nbytes, _stream(stream), C.byref(h)),
               "batch_plan_create")
        return BatchPlan(h, self, workspace)


class BatchPlan:
    """Uploaded batch descriptors; run() enqueues kernels only (graph-capturable)."""

    def __init__(self, handle, batch, workspace):
        self.handle = handle
        self._keep = (batch, workspace)

    def run(self, sums, results=None, counters=None, stream=None):
        _check(lib().qmc_batch_plan_run(self.handle, _ptr(sums), _ptr(results), _ptr(counters),
                                        _stream(stream)), "batch_plan_run")
        return sums

    def close(self):
        if self.handle:
            lib().qmc_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------------
def _result_dict(res: qmc_result) -> dict:
    return {"integral": complex(res.integral.re, res.integral.im),
            "error": complex(res.error.re, res.error.im),
            "value": res.integral.re, "err": res.error.re,
            "n": res.n, "m": res.m, "iterations": res.iterations, "evaluations": res.evaluations,
            "nonfinite": res.nonfinite, "signfail": res.signfail}


class Server:
    """Continuous-batching request loop (qmc_server_*)."""

    PENDING, ACTIVE, DONE = 0, 1, 2

    def __init__(self, table: GenvecTable, memory_budget: int, max_slots: int, m: int,
                 transform=("korobov", 3), stream=None, step_evaluations: int = 0):
        cfg = qmc_server_config(int(memory_budget), int(max_slots), int(m), make_transform(transform),
                                int(step_evaluations))
        h = C.c_void_p()
        _check(lib().qmc_server_create(C.byref(table.struct), C.byref(cfg), _stream(stream),
                                       C.byref(h)), "server_create")
        self.handle = h
        self._table = table

    def submit(self, f: Integrand, epsrel: float, epsabs: float = 0.0, minn: int = 1021,
               maxeval: int = 10**8, seed: int = 0) -> int:
        fs = f.host_struct()
        rid = C.c_uint64()
        _check(lib().qmc_server_submit(self.handle, C.byref(fs), float(epsrel), float(epsabs),
                                       int(minn), int(maxeval), int(seed) & (2**64 - 1),
                                       C.byref(rid)), "server_submit")
        return int(rid.value)

    def step(self) -> int:
        done = C.c_int()
        _check(lib().qmc_server_step(self.handle, C.byref(done)), "server_step")
        return int(done.value)

    def status(self, rid: int):
        st, res, lat = C.c_int(), qmc_result(), C.c_double()
        code = lib().qmc_server_status(self.handle, int(rid), C.byref(st), C.byref(res), C.byref(lat))
        if code not in (0, _capi.QMC_ERR_NONFINITE):
            raise QMCError(code, "server_status")
        out = _result_dict(res)
        out.update({"state": int(st.value), "latency_s": float(lat.value), "status": int(code)})
        return out

    def counts(self):
        p, a, f = C.c_int(), C.c_int(), C.c_size_t()
        _check(lib().qmc_server_counts(self.handle, C.byref(p), C.byref(a), C.byref(f)), "server_counts")
        return int(p.value), int(a.value), int(f.value)

    def completed(self, cap: int = 4096) -> list[int]:
        """Identifiers of the requests finished since the previous call (qmc_server_completed)."""
        out = []
        buf = (C.c_uint64 * cap)()
        while True:
            k = C.c_int()
            _check(lib().qmc_server_completed(self.handle, buf, cap, C.byref(k)), "server_completed")
            out.extend(int(buf[i]) for i in range(k.value))
            if k.value < cap:
                return out

    def close(self):
        if self.handle:
            lib().qmc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
