"""Benchmark: FP64 integrand evaluations per second of randomly shifted rank-1 lattice
quadrature on GB300 (one JSON line on stdout).

Workload (one step = the whole hot path over one batch): Genz oscillatory, corner peak
and Gaussian (Sec. 5.2 test functions, ||c||_1 = 6.0, 2.2, 15.2) in d = 6, 8, 10, each
with the baker and Korobov r = 1..4 maps (3 x 3 x 5 = 45 integrals), each on the CBC lattice
n = 10,560,653 (the first table size >= 1e7) with m = 32 random shifts; seeded synthetic
parameters (workloads.genz_params).  Per integral the step runs the lattice-sum kernel,
the fixed-order tile reduction and the shift reduction (mean and standard error).

  value      evaluations/s with inputs resident in HBM (device entry points)
  e2e        the same through qmc_integrate() with host buffers: host->device copies of
             coefficients and shifts and the device->host result read inside the timed
             region
  roofline   the lattice-sum kernel against the unit that bounds it: for the Genz
             workload the integer multiply pipe (its fixed-point transforms and forms),
             achieved = algorithmic 32-bit multiplies per evaluation (int_mul_per_eval)
             x evaluations per launch / CUDA-event launch time, peak = the same
             operation's rate measured on the device by qmc_probe_units; for the complex
             workload the FP64 pipe (counted FP64 flops against the measured FP64 FMA
             rate), likewise for --workload sector (four real sector integrands U/F^2.5,
             d = 8, 200 + 200 monomials: the batching configuration's kernel), each with
             the integer pipe's share beside it.  The method's FP64 work rate against the FP64 peak is reported beside
             it as fp64_equivalent (it can exceed 1: the kernel does much of that work
             exactly on the integer pipe)
  latency, feynman, batch, serve   bounded runs of the other configurations (the d = 4
             integral's latency, the complex family's rate, a batch with n log-uniform
             in [1e4, 1e8] against one launch per integral, Poisson-arrival serving)
  cpu_baseline   the CPU oracle on a bounded sample of the same workload

--impl reference times the oracle alone (the reference arm for this build).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FAMILIES = (1, 3, 4)          # oscillatory, corner peak, Gaussian
DIMS = (6, 8, 10)
TRANSFORMS = (("baker",), ("korobov", 1), ("korobov", 2), ("korobov", 3), ("korobov", 4))
N_LATTICE = 10560653
M_SHIFTS = 32
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) of one lattice-sum launch from an ncu capture of the current
# kernel, or None when the kernel has changed since the capture: sums_kernel<Gaussian,
# integer Korobov>, d = 10, Korobov-3, n = 1,072,187, m = 32 (2272 tiles): 98,560 bytes
# read, 0 written (the partials stay in L2).  The inputs are kilobytes and the partials
# grow only with the tile count (at most six waves of 760), so the figure stands for the
# benchmark's launches.
TRAFFIC_BYTES_PER_LAUNCH = 98_560

# 32-bit integer multiplies of the fixed-point primitives (qmc_fixed.cuh):
MUL_HI = 3        # truncated 64-bit high product: one 32x32->64, two 32-bit high multiplies
SQ_HI = 2         # its square form: one 32x32->64, one 32-bit high multiply
MUL64_HI = 4      # full 64-bit high product: four 32-bit multiplies
MUL64_LO = 3      # 64-bit low product: one 32x32->64, two 32-bit low multiplies
RECIP = 2 * (MUL64_LO + 2 * MUL64_HI)                      # two Newton steps (fx_recip)
EXP_FIXED = MUL64_LO + MUL64_HI + MUL_HI + 6 * MUL_HI + MUL_HI   # Tang's exp (exp_fixed)
COS_TURNS = MUL_HI + SQ_HI + 8 * MUL_HI                   # cos of a phase in turns
# highest Korobov order whose final function runs on the integer pipe (FamilyAcc)
INT_FINISH_MAX_R = {1: 4, 2: 6, 3: 1, 4: 3, 5: 3, 6: 3}


def korobov_map_muls(r: int) -> int:
    """Per dimension, the fixed-point Korobov<r,r> map: v^2, P(w) in Estrin's form, v^(r+1),
    phi = v^(r+1) P, and the weight factor t = v - v^2 into the running product."""
    P = {1: 0, 2: MUL_HI, 3: MUL_HI, 4: MUL_HI + SQ_HI + MUL_HI, 5: MUL_HI + SQ_HI + MUL_HI,
         6: 3 * MUL_HI + SQ_HI + 2 * MUL_HI}[r]
    pw = {1: 0, 2: MUL_HI, 3: SQ_HI, 4: SQ_HI + MUL_HI, 5: MUL_HI + SQ_HI,
          6: MUL_HI + SQ_HI + MUL_HI}[r]
    return SQ_HI + P + pw + MUL_HI + MUL_HI


def korobov_weight_muls(r: int) -> int:
    """Per evaluation: (prod_j t_j)^r by binary powering, times C^d."""
    return (r.bit_length() - 1) * SQ_HI + (bin(r).count("1") - 1) * MUL_HI + MUL_HI


def int_mul_per_eval(family: int, transform, d: int, c=None) -> int:
    """Algorithmic integer-multiply work of one evaluation in the kernel's fixed-point form
    (32-bit multiplies; the unit the Genz lattice sums are bound by), for families 1-6
    under baker, none and Korobov<r,r> r <= 6 with parameters in the Genz ranges:
      map: Korobov-r korobov_map_muls(r) per dimension + korobov_weight_muls(r); baker 0;
      form per dimension: oscillatory, corner, C0, discontinuous one high product (the
        oscillatory adds a 64-bit low product when some c_j >= 2 pi), Gaussian and
        product peak one high product and one square (the product peak also its running
        product);
      final function on the integer pipe (below the family's crossover order): cos in
        turns, Tang's exp, or the (d+1)-th power and Newton reciprocal.
    The lattice points themselves are additions (one step per point and coordinate,
    shared by the warp's 32 shifts) and cost no multiplies."""
    kind = transform[0]
    r = transform[1] if kind == "korobov" else 0
    if kind == "korobov" and (len(transform) > 2 and transform[2] != r or not 1 <= r <= 6):
        return 0
    if kind not in ("baker", "none", "korobov"):
        return 0
    per_dim, per_eval = 0, 0
    if kind == "korobov":
        per_dim += korobov_map_muls(r)
        per_eval += korobov_weight_muls(r)
    int_finish = kind != "korobov" or r <= INT_FINISH_MAX_R[family]
    if family in (1, 3, 5, 6):
        per_dim += MUL_HI
        if family == 1 and c is not None and max(c) >= 2 * math.pi:
            per_dim += MUL64_LO
    elif family in (2, 4):
        per_dim += MUL_HI + SQ_HI + (MUL_HI if family == 2 else 0)
    if int_finish:
        if family == 1:
            per_eval += COS_TURNS
        elif family in (4, 5, 6):
            per_eval += EXP_FIXED
        elif family == 3:
            p = d + 1
            per_eval += (p.bit_length() - 1) * SQ_HI + (bin(p).count("1") - 1) * MUL_HI + RECIP
        elif family == 2:
            per_eval += MUL_HI + RECIP
    return per_dim * d + per_eval


def fp64_flops_per_eval(family: int, transform, d: int) -> int:
    """Algorithmic FP64 work of one evaluation (add/mul = 1, fma = 2, each library call or
    division = 1 "special" flop), per family and transform:
      Korobov-r: (2r+1) fma for phi, (r+2) mul for w, 1 mul into the product, per dim
      baker: 2 per dim;  oscillatory: d fma + cos;  corner: d fma + ceil(log2(d+1)) mul + div;
      Gaussian: d (sub + fma) + exp;  accumulation: weight multiply + add;
      point: 1 add + 1 compare per dimension (u = x + Delta, u -= 1 if u >= 1; the
      division x = r/n is per point, shared by the m shifts, and is not counted)."""
    kind = transform[0]
    if kind == "korobov":
        r = transform[1]
        tr = d * (2 * (2 * r + 1) + (r + 2) + 1)
    elif kind == "baker":
        tr = 2 * d
    else:
        tr = 0
    if family == 1:
        fam = 2 * d + 1
    elif family == 3:
        fam = 2 * d + math.ceil(math.log2(d + 1)) + 1
    elif family == 4:
        fam = 3 * d + 1
    elif family == 2:
        fam = 5 * d
    else:
        fam = 2 * d
    return tr + fam + 2 + 2 * d


def feynman_flops_per_eval(fl) -> int:
    """Algorithmic FP64 work of one evaluation of the complex deformed integrand U^a F^-b
    det J (d = 5 Feynman-parameter workload), with the rules of fp64_flops_per_eval
    (add/mul = 1, fma = 2, each library call = 1): value, gradient and Hessian of F (one fused multiply-add per term and
    derivative, nf (1 + d + d(d+1)/2) of them), U and F at the complex point (a complex
    multiply-add per factor: 8 flops), the deformation and the Jacobian entries (3d + 2d^2),
    complex LU of the d x d Jacobian (8 d^3 / 3), two complex powers (hypot, atan2, log, exp,
    sincos: 5 calls + 4 flops each), two complex products and the weighted accumulation."""
    d = fl.d
    nf, nu = fl.F.nterms, fl.U.nterms
    factors = int(fl.U.exps.sum() + fl.F.exps.sum())
    derivs = 2 * nf * (1 + d + d * (d + 1) // 2)
    complex_vals = 8 * factors + 2 * 2 * (nu + nf)
    deform = 3 * d + 2 * d * d
    lu = (8 * d ** 3) // 3
    return derivs + complex_vals + deform + lu + 2 * 9 + 12 + 4


def sector_flops_per_eval(fl, transform) -> int:
    """Algorithmic FP64 work of one evaluation of the real sector integrand U^a F^-b in the
    paper's term-by-term form (rules of fp64_flops_per_eval): per monomial of degree q,
    q - 1 multiplies and one fused multiply-add; the power F^-b (a = 1, half-integer b:
    two multiplies, a square root and a reciprocal) and the product with U; the Korobov-r
    map per dimension, the weight and the accumulation as for the Genz families."""
    terms = fl.U.nterms + fl.F.nterms
    factors = int(fl.U.exps.sum() + fl.F.exps.sum())
    d = fl.d
    r = transform[1] if transform[0] == "korobov" else 0
    tr = d * (2 * (2 * r + 1) + (r + 2) + 1) if r else 0
    return (factors - terms) + 2 * terms + 5 + tr + 2 + 2 * d


def sector_kernel_flops_per_eval(d: int) -> int:
    """FP64 work of one evaluation in the form the kernel runs for the sector benchmark
    workload (both polynomials dense, F in fixed point, d compiled in; qmc_poly.cuh): U's
    dense quadratic in V = d + 1 variables with the x_d = 1 iterations as additions
    (V (V - 1) / 2 + V - 1 fma, V + 1 adds), the power U (F^-1/2)^5 (a reciprocal square
    root, 4 mul), the weight (2 mul) and the accumulation (2 adds).  F's Horner form and the
    Korobov map run on the integer pipe (sector_int_mul_per_eval)."""
    V = d + 1
    fma = V * (V - 1) // 2 + V - 1
    return 2 * fma + (V + 1) + 5 + 2 + 2


def sector_int_mul_per_eval(transform, d: int) -> int:
    """32-bit multiplies of one sector evaluation on the integer pipe: F's dense cubic in
    fixed point with the x_d = 1 iterations as additions (C(V+1, 3) + V (V - 1) / 2 + V - 1
    truncated high products, V = d + 1) and the integer Korobov<r,r> map and weight."""
    V = d + 1
    prods = math.comb(V + 1, 3) + V * (V - 1) // 2 + (V - 1)
    per = MUL_HI * prods
    kind = transform[0]
    r = transform[1] if kind == "korobov" else 0
    if kind == "korobov" and 1 <= r <= 6 and (len(transform) < 3 or transform[2] == r):
        per += korobov_map_muls(r) * d + korobov_weight_muls(r)
    return per


FEYN_FIXED_DIMS = range(3, 7)      # dimensions whose contractions run in fixed point


def feynman_fixed_int_mul_per_eval(d: int) -> int:
    """32-bit multiplies of the fixed-point part of one complex evaluation (d = 3..6): the
    Hessian 2 F2 + 6 F3 x (d per entry of the upper triangle) and the contractions H x, F2 x,
    U2 x (d^2 each), one truncated 64-bit high product (MUL_HI) apiece."""
    if d not in FEYN_FIXED_DIMS:
        return 0
    return MUL_HI * (d * d * (d + 1) // 2 + 3 * d * d)


def feynman_int_mul_per_eval(transform, d: int) -> int:
    """32-bit multiplies of one complex evaluation: the integer Korobov<r,r> map and weight
    (as int_mul_per_eval counts them) and the fixed-point contractions."""
    kind = transform[0]
    r = transform[1] if kind == "korobov" else 0
    per = feynman_fixed_int_mul_per_eval(d)
    if kind == "korobov" and 1 <= r <= 6 and (len(transform) < 3 or transform[2] == r):
        per += korobov_map_muls(r) * d + korobov_weight_muls(r)
    return per


def feynman_tensor_flops_per_eval(d: int) -> int:
    """FP64 work of one evaluation of the complex deformed integrand in the symmetric-tensor
    form the kernel evaluates for deg U <= 2, deg F <= 3 (qmc_poly.cuh), with fma = 2 and
    add/mul/div/sqrt = 1, for a = 1 and a half-integer b (b = 2.5): the Hessian 2 F2 + 6 F3 x,
    gradient and grad U (in fixed point for d = 3..6, so no FP64 work there; FP64 otherwise),
    F(x) and U(x) (the nested form in FP64 for d = 3..6), the deformation
    y = -lam x (1 - x) g, F(z) and U(z) by the exact Taylor series (for d = 3..6 y.H y over
    the upper triangle and the cubic and quadratic parts at y by nested forms), det J by elimination
    without pivoting (the first column on purely imaginary entries; for d = 3..6 the
    symmetric elimination of diag(1 + i Lambda) + diag(lx) i H), 1 / (F^2 sqrt F) by the
    principal root, the products with U and det J, the weight and the accumulation.  It does
    not grow with the number of monomials."""
    P = d * (d + 1) // 2
    fma, mul, add, special = 0, 0, 0, 0
    if d in FEYN_FIXED_DIMS:
        fma += d * (d + 1) * (d + 2) // 6 + P + d        # F(x), nested form
        fma += P + d                                     # U(x), nested form
    else:
        fma += P * (d + 1)                               # Hessian entries
        fma += d * (3 * d + 6)                           # gradient, F(x), U(x), grad U
        add += 2 * d + 2
    add += d                                             # 1 - x
    mul += 3 * d                                         # -lam x (1 - x), y = xo g
    if d in FEYN_FIXED_DIMS:
        fma += (P - d) + 2 * d + 2 * d                   # y.H y (upper triangle), g.y, gradU.y
        mul += d
        fma += d * (d + 1) * (d + 2) // 6 + 2 * P + 2 * d   # F3[y,y,y], y.U2 y nested
        fma += 1
        add += 2                                         # F(z), U(z)
    else:
        fma += d * (2 * d + 4) + P * (d + 1)             # y.H y, y.U2 y, g.y, gradU.y, F3[y,y,y]
        mul += 2 * P
        fma += 2
        add += 1                                         # F(z), U(z)
    if d in FEYN_FIXED_DIMS:
        # symmetric elimination of J = diag(1 + i Lambda) + diag(lx) i H (upper triangle)
        fma += d
        mul += 2 * d                                     # Lambda
        fma += 1 + 1                                     # first pivot, its reciprocal
        mul += 3 + 2 + 2 * (d - 1)
        special += 1
        fma += (d - 1) * d // 2                          # first step: K' = i H + u H_0q
        mul += (d - 1) * d // 2
        for c in range(1, d):                            # pivots c >= 1
            fma += 2 + 2                                 # pivot, det product
            mul += 2
            if c + 1 < d:
                fma += 1
                mul += 3 + 2
                special += 1
                rows = d - c - 1
                fma += rows * 2 + 4 * rows * (rows + 1) // 2
                mul += rows * 2
    else:
        mul += d * d + d                                 # Jacobian entries
        fma += 2 * d
        fma += 1 + (d - 1) * 2 * (d - 1)                 # first column
        mul += 3 + (d - 1) * 2
        special += 1
        for c in range(1, d):                            # pivots c >= 1
            fma += 2
            mul += 2
            if c + 1 < d:
                fma += 1
                mul += 3
                special += 1
                rows = d - c - 1
                fma += rows * (2 + 4 * rows)
                mul += rows * 2
    fma += 1                                             # principal sqrt, F^2 sqrt F, 1/den
    mul += 1 + 1 + 1
    add += 1
    special += 3
    fma += 2 * 2 + 1 + 2 * 2
    mul += 2 * 2 + 3 + 2 * 2
    special += 1
    mul += 2 + 1                                         # weight (x2), C^d weight factor
    add += 2                                             # accumulation
    return 2 * fma + mul + add + special


def parse_transform(tok: str):
    if tok == "baker":
        return ("baker",)
    if tok.startswith("korobov"):
        return ("korobov", int(tok[len("korobov"):]))
    raise ValueError(tok)


FEYNMAN_FAMILY = 20
FEYNMAN_INTEGRALS = 4
SECTOR_FAMILY = 21
SECTOR_INTEGRALS = 4
SECTOR_D, SECTOR_TERMS = 8, 200


def workload_items(rank: int = 0, only: str | None = None, workload: str = "genz"):
    """The 45 (family, d, transform, c, w) Genz integrals, or the single one named by
    ``only`` ("FAMILY:D:TRANSFORM", e.g. "4:10:korobov3") for profiling a small case.
    workload "feynman": four d = 5 complex deformed Feynman-parameter integrands
    (workloads.feynman_regular) with Korobov-3, as (20, 5, transform, FeynmanLike, None)."""
    if workload == "feynman":
        return [(FEYNMAN_FAMILY, 5, ("korobov", 3), W.feynman_regular(1000 + 17 * rank + k), None)
                for k in range(FEYNMAN_INTEGRALS)]
    if workload == "sector":
        # real sector integrands U / F^2.5, d = 8, 200 + 200 monomials (both forms dense,
        # F in fixed point): the lattice-sum kernel of the batching configuration
        return [(SECTOR_FAMILY, SECTOR_D, ("korobov", 3),
                 W.sector_like(1000 + 17 * rank + k, SECTOR_D, SECTOR_TERMS, SECTOR_TERMS), None)
                for k in range(SECTOR_INTEGRALS)]
    if workload == "feynman_like":
        # the configuration's literal polynomials (all 15 + 35 monomials, coefficients
        # U(-1, 2), lam = 0.5): the same kernel cost; U F^-2.5 is not integrable where F
        # vanishes on the cube's faces, so its values are a throughput check only
        return [(FEYNMAN_FAMILY, 5, ("korobov", 3), W.feynman_like(1000 + 17 * rank + k), None)
                for k in range(FEYNMAN_INTEGRALS)]
    items = []
    for fam in FAMILIES:
        for d in DIMS:
            c, w = W.genz_params(fam, d, 1000 + 17 * rank + d)
            for tr in TRANSFORMS:
                items.append((fam, d, tr, c, w))
    if only:
        f, d, t = only.split(":")
        key = (int(f), int(d), parse_transform(t))
        items = [it for it in items if (it[0], it[1], it[2]) == key]
        if not items:
            raise ValueError(f"--only {only} names no workload item")
    return items


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
def measure_unit_peaks(q, torch, dev, stream, local: int = 0, kernel_mhz: float | None = None,
                       target_ms: float = 50.0, launches: int = 10) -> dict:
    """The roofline's denominators on this device: the FP64 fused multiply-add rate and
    the rate of the kernel's truncated 64-bit high product (in 32-bit multiplies).  Each
    unit runs `launches` qmc_probe_units launches of ~target_ms back to back, timed with
    CUDA events on the launching stream after a sizing launch, with the SM clock sampled
    meanwhile.  A full-occupancy FMA loop can draw the GPU to its power cap and lower the
    clock; the rate is therefore also stated per SM clock and, as `peak`, scaled to the
    median SM clock of the benchmark's timed region (kernel_mhz)."""
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {}
    for unit in ("fp64_fma", "int_mulhi"):
        trips = 256
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):                                  # warm-up and sizing
            e0.record(stream)
            q.probe_units(unit, trips, sink, stream)
            e1.record(stream)
            e1.synchronize()
            trips = max(1, int(trips * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.25)
        ops = 0.0
        e0.record(stream)
        for _ in range(launches):
            ops += q.probe_units(unit, trips, sink, stream)
        e1.record(stream)
        e1.synchronize()
        time.sleep(0.25)
        clk = sampler.stop()
        rate = ops / (e0.elapsed_time(e1) * 1e-3)
        mhz = clk.get("sm_mhz")
        scale = (kernel_mhz / mhz) if (mhz and kernel_mhz) else 1.0
        out[unit] = {"rate": rate, "probe_sm_mhz": mhz, "at_kernel_clock": rate * scale,
                     "per_sm_clock": rate / (SM_COUNT * mhz * 1e6) if mhz else None,
                     "reasons": clk.get("reasons")}
    f, m = out["fp64_fma"], out["int_mulhi"]
    return {"fp64_gflops": 2.0 * f["at_kernel_clock"] / 1e9,
            "int_mul_gops": m["at_kernel_clock"] / 1e9,
            "fp64_gflops_measured": 2.0 * f["rate"] / 1e9, "int_mul_gops_measured": m["rate"] / 1e9,
            "fp64_fma_per_sm_clock": f["per_sm_clock"], "int_mul_per_sm_clock": m["per_sm_clock"],
            "probe_sm_mhz": {"fp64": f["probe_sm_mhz"], "int": m["probe_sm_mhz"]},
            "probe_reasons": {"fp64": f["reasons"], "int": m["reasons"]},
            "kernel_sm_mhz": kernel_mhz,
            "how": f"qmc_probe_units: chains of FP64 FMA / of the truncated 64-bit high product "
                   f"(3 32-bit multiplies) on a full-occupancy grid, {launches} launches of "
                   f"~{target_ms:.0f} ms timed with CUDA events, SM clock sampled meanwhile; "
                   f"peak = rate scaled to the benchmark's median SM clock"}


def run_gpu(args, rank: int, world: int):
    import torch

    import paper_1811_11720_gb300 as q

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    table = q.GenvecTable.load()
    n = args.n
    zfull = table.z_for(n)
    items = workload_items(rank, args.only, args.workload)
    stream = torch.cuda.current_stream(dev)
    cplx = args.workload in ("feynman", "feynman_like")

    # resident inputs: coefficients, shifts, workspace, outputs
    prepared = []
    max_ws = 0
    for idx, (fam, d, tr, c, w) in enumerate(items):
        f = (q.Integrand.polynomial(c) if fam in (FEYNMAN_FAMILY, SECTOR_FAMILY)
             else q.Integrand.genz(fam, c, w))
        D = q.make_shifts(args.seed + 7919 * rank + idx, M_SHIFTS, d)
        Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
        r = q.rule(n, zfull[:d], Dd, tr)
        fd = f.device_struct(dev)
        max_ws = max(max_ws, q.sums_workspace_bytes(r, cplx, 0, n))
        prepared.append((fam, d, tr, f, fd, r, Dd, D))
    ws = torch.empty(max_ws, dtype=torch.uint8, device=dev)
    sums = torch.empty(len(items), 4 * M_SHIFTS, dtype=torch.float64, device=dev)
    res = torch.empty(len(items), 4, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    evals_per_step = len(items) * n * M_SHIFTS
    flops_per_step = sum(feynman_flops_per_eval(c) if fam == FEYNMAN_FAMILY else
                         sector_flops_per_eval(c, tr) if fam == SECTOR_FAMILY else
                         fp64_flops_per_eval(fam, tr, d) for fam, d, tr, c, _ in items) * n * M_SHIFTS
    muls_per_step = sum(feynman_int_mul_per_eval(tr, d) if fam == FEYNMAN_FAMILY else
                        sector_int_mul_per_eval(tr, d) if fam == SECTOR_FAMILY else
                        int_mul_per_eval(fam, tr, d, c) for fam, d, tr, c, _ in items) * n * M_SHIFTS
    # FP64 work of the form the kernel runs (polynomial families)
    tensor_flops_per_step = sum(feynman_tensor_flops_per_eval(d) if fam == FEYNMAN_FAMILY else
                                sector_kernel_flops_per_eval(d) if fam == SECTOR_FAMILY else 0
                                for fam, d, tr, c, _ in items) * n * M_SHIFTS

    ev_k = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in items]

    def step(time_kernels: bool, s=stream):
        kt = 0.0
        for i, (fam, d, tr, f, fd, r, Dd, D) in enumerate(prepared):
            if time_kernels:
                ev_k[i][0].record(s)
            q.sums(fd, r, 0, n, ws, sums[i], cnt, s)
            if time_kernels:
                ev_k[i][1].record(s)
            q.finalize(sums[i], M_SHIFTS, n, cplx, res[i], None, s)
        if time_kernels:
            torch.cuda.synchronize(dev)
            per = [a.elapsed_time(b) for a, b in ev_k]
            for i, v in enumerate(per):
                item_ms[i] += v
            kt = sum(per)
        return kt

    item_ms = [0.0] * len(prepared)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize(dev)
    graph = None
    if getattr(args, "graph", False):
        # the whole step (2 launches per integral) captured once and replayed: the host's
        # argument checks and launch calls leave the timed region
        graph = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream(dev)          # capture needs a stream other than the default
        with torch.cuda.graph(graph, stream=gs):
            step(False, gs)
        graph.replay()
        torch.cuda.synchronize(dev)

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms = []
    kernel_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()                      # L2 flushed between steps, outside the timing
        torch.cuda.synchronize(dev)
        e0.record(stream)
        if graph is not None:
            graph.replay()
        elif args.kernel_events:
            kernel_ms += step(True)
        else:
            step(False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()

    # correctness spot check of the last step (cheap): closed forms within 8 sigma
    from_host = res.cpu().numpy()
    nonfinite = int(cnt[0].item())

    # e2e through qmc_integrate with host buffers
    e2e_ms = []
    h2d = 0
    for it in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for (fam, d, tr, f, fd, r, Dd, D), (_, _, _, c, w) in zip(prepared, items):
            out = q.integrate(f, table, n, M_SHIFTS, tr, seed=args.seed + 7919 * rank, stream=stream)
            if it == 0:
                h2d += M_SHIFTS * d * 8 + (c.nbytes + w.nbytes if fam not in (FEYNMAN_FAMILY, SECTOR_FAMILY) else
                                           sum(a.nbytes for a in (c.U.coef, c.U.exps, c.F.coef, c.F.exps)))
        torch.cuda.synchronize(dev)
        if it > 0:                         # first pass warms the library's arena
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = float(sum(e2e_ms))
    if world > 1:
        t = torch.tensor([e2e_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())

    k_per_launch_ms = (kernel_ms / (args.steps * len(items))
                       if args.kernel_events and graph is None else None)
    peaks = (measure_unit_peaks(q, torch, dev, stream, local, clocks.get("sm_mhz"))
             if rank == 0 and not getattr(args, "skip_peaks", False) else None)
    out = {
        "total_ms": total_ms, "step_ms": step_ms, "evals_per_step": evals_per_step,
        "flops_per_step": flops_per_step, "muls_per_step": muls_per_step,
        "tensor_flops_per_step": tensor_flops_per_step,
        "kernel_ms_per_item": ({f"{fam}:{d}:{tr[0]}{tr[1] if len(tr) > 1 else ''}": ms / args.steps
                                for (fam, d, tr, _, _), ms in zip(items, item_ms)}
                               if args.kernel_events and graph is None else None),
        "kernel_ms_per_launch": k_per_launch_ms, "unit_peaks": peaks,
        "clocks": clocks, "e2e_total_ms": e2e_total, "e2e_steps": args.e2e_steps,
        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(items) * ((8 if cplx else 4) * 8 + 2 * 8),
        "nonfinite": nonfinite, "results": from_host, "items": items,
        "launches_per_step": len(items) * 3,
    }
    return out


def run_batch_workload(args):
    """Batching (many sector integrals in one launch) against one launch per integral.

    Workload: `--batch-count` sector integrands U/F^2.5 with positive coefficients,
    d ~ U{3..8}, U and F of 10..400 monomials each, m = 32, Korobov-3, the
    variance-reduction fit (histogram + Levenberg-Marquardt) on every second integral, and
    n log-uniform in [1e4, --batch-nmax] snapped to the table.  Every integral is
    evaluated twice per step-pair: once inside one batched launch (autotuned shape, replayed
    from a CUDA graph) and once as separate qmc_sums + qmc_finalize launches (also replayed
    from a CUDA graph); both reach the same error (same lattices and shifts)."""
    import torch

    import paper_1811_11720_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    table = q.GenvecTable.load()
    rng = np.random.default_rng(args.seed)
    count = args.batch_count
    m = M_SHIFTS
    entries, keep = [], []
    fit_s = 0.0
    n_fit = q.get_next_n(table, 100000)
    z_fit = table.z_for(n_fit)
    evals = 0
    for i in range(count):
        d = int(rng.integers(3, 9))
        fl = W.sector_like(args.seed + i, d, int(rng.integers(10, 401)), int(rng.integers(10, 401)))
        f = q.Integrand.polynomial(fl)
        fs = f.device_struct(dev)
        n = q.get_next_n(table, int(np.exp(rng.uniform(np.log(1e4), np.log(args.batch_nmax)))))
        D = q.make_shifts(args.seed + 31 * i, m, d)
        Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
        fitd = None
        if i % 2 == 1:
            t0 = time.perf_counter()
            sh = torch.from_numpy(q.make_shifts(args.seed + 31 * i + 1, 1, d)[0].astype(np.int64)).to(dev)
            hist = torch.empty(d * 1000, dtype=torch.float64, device=dev)
            hws = torch.empty(q.histogram_workspace_bytes(n_fit, d, 1000), dtype=torch.uint8, device=dev)
            q.histogram(fs, n_fit, z_fit[:d], sh, 1000, hist, hws)
            params = q.fit_polysingular(hist.cpu().numpy().reshape(d, 1000))
            fitd = torch.from_numpy(params).to(dev)
            fit_s += time.perf_counter() - t0
        r = q.rule(n, table.z_for(n)[:d], Dd, ("korobov", 3), fitd)
        entries.append((fs, r, 0, n))
        keep.append((f, Dd, fitd))
        evals += n * m
    b = q.Batch(entries)
    sums = torch.zeros(count, 4 * m, dtype=torch.float64, device=dev)
    res = torch.zeros(count, 4, dtype=torch.float64, device=dev)
    ws0 = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    cfg = b.autotune(ws0, sums)
    ws = torch.empty(b.workspace_bytes(cfg), dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream()
    plan = b.plan(ws, cfg, stream=s)
    # single-integral path: one workspace per integral, captured in one graph
    singles = []
    for (fs, r, a, bnd) in entries:
        wsi = torch.empty(max(8, q.sums_workspace_bytes(r, False, a, bnd)), dtype=torch.uint8, device=dev)
        singles.append((fs, r, a, bnd, wsi))
    sums1 = torch.zeros(count, 4 * m, dtype=torch.float64, device=dev)
    res1 = torch.zeros(count, 4, dtype=torch.float64, device=dev)

    def single_pass(stream):
        for i, (fs, r, a, bnd, wsi) in enumerate(singles):
            q.sums(fs, r, a, bnd, wsi, sums1[i], None, stream)
            q.finalize(sums1[i], m, int(r.n), False, res1[i], None, stream)

    with torch.cuda.stream(s):
        for _ in range(max(1, getattr(args, "batch_warm", 2))):
            plan.run(sums, res, stream=s)
            single_pass(s)
    torch.cuda.synchronize()
    g_b, g_s = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_b, stream=s):
        plan.run(sums, res, stream=s)
    with torch.cuda.graph(g_s, stream=s):
        single_pass(s)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    tb, ts = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        with torch.cuda.stream(s):          # replay and events on the same stream
            ev[0].record(s)
            g_b.replay()
            ev[1].record(s)
            ev[2].record(s)
            g_s.replay()
            ev[3].record(s)
        torch.cuda.synchronize()
        tb.append(ev[0].elapsed_time(ev[1]))
        ts.append(ev[2].elapsed_time(ev[3]))
    same = bool(torch.allclose(res[:, 0], res1[:, 0], rtol=1e-12, atol=0))
    err_rel = (res[:, 1].abs() / res[:, 0].abs()).median().item()
    line = {"metric": "batched integrals/s", "unit": "integrals/s",
            "value": count / (float(np.median(tb)) / 1e3), "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sector_batch_{count}_d3-8_terms10-400_n1e4-{args.batch_nmax:.0e}_m32_korobov3_fit_half",
                       "evaluations": evals, "launch_shape": {"streams_per_block": cfg.streams_per_block,
                                                              "points_per_stream": cfg.points_per_stream}},
            "batched_ms": float(np.median(tb)), "per_integral_ms": float(np.median(ts)),
            "per_integral_integrals_per_s": count / (float(np.median(ts)) / 1e3),
            "speedup": float(np.median(ts) / np.median(tb)),
            "evals_per_s_batched": evals / (float(np.median(tb)) / 1e3),
            "same_results": same, "median_rel_error": err_rel, "fit_setup_s": fit_s,
            "gpu_launches_batched": 3, "gpu_launches_per_integral": 3 * count}
    plan.close()
    return line


SERVE_EPSABS = 1e-7   # the library's default absolute goal (App. A.1)


def run_latency_workload(args):
    """Latency of one small integral: the d = 4 product peak (c_j = 5, Korobov-3,
    n = 108863, m = 16; 1.74e6 evaluations per integral) integrated repeatedly.  Three
    paths: qmc_integrate with host buffers (coefficients and shifts copied in, the result
    read back: what a caller waits for), the device entry points qmc_sums + qmc_finalize
    on resident inputs (CUDA events), and the same pair replayed from a CUDA graph.
    Reports median and 99th-percentile latency per integral in microseconds."""
    import torch

    import paper_1811_11720_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    table = q.GenvecTable.load()
    n, d, m, tr = 108863, 4, 16, ("korobov", 3)
    c, w = W.product_peak_params(d, args.seed)
    f = q.Integrand.genz(2, c, w)
    reps = max(20, args.steps * 40)
    # host-buffer path
    for _ in range(5):
        q.integrate(f, table, n, m, tr, seed=args.seed)
    torch.cuda.synchronize()
    host = []
    for _ in range(reps):
        t0 = time.perf_counter()
        q.integrate(f, table, n, m, tr, seed=args.seed)
        host.append((time.perf_counter() - t0) * 1e6)
    # device path on resident inputs
    D = torch.from_numpy(q.make_shifts(args.seed, m, d).astype(np.int64)).to(dev)
    r = q.rule(n, table.z_for(n)[:d], D, tr)
    fd = f.device_struct(dev)
    ws = torch.empty(q.sums_workspace_bytes(r, False, 0, n), dtype=torch.uint8, device=dev)
    sums = torch.zeros(4 * m, dtype=torch.float64, device=dev)
    res = torch.zeros(4, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()

    def once():
        q.sums(fd, r, 0, n, ws, sums, None, s)
        q.finalize(sums, m, n, False, res, None, s)

    with torch.cuda.stream(s):
        for _ in range(5):
            once()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        once()
    dev_us, graph_us = [], []
    for lst, fn in ((dev_us, once), (graph_us, g.replay)):
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                e0.record(s)
                fn()
                e1.record(s)
            e1.synchronize()
            lst.append(e0.elapsed_time(e1) * 1e3)

    def pct(v):
        return {"p50_us": float(np.percentile(v, 50)), "p99_us": float(np.percentile(v, 99))}

    out = {"metric": "product-peak d=4 integral latency", "unit": "us", "higher_is_better": False,
           "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "product_peak_d4_c5_korobov3_n108863_m16", "repetitions": reps,
                      "evaluations": n * m},
           "value": float(np.percentile(host, 50)),
           "host_buffers": pct(host), "device_entry_points": pct(dev_us),
           "cuda_graph": pct(graph_us),
           "device_evals_per_s": n * m / (float(np.percentile(graph_us, 50)) * 1e-6)}
    return out


def goal_met(res, epsrel: float, epsabs: float = SERVE_EPSABS) -> bool:
    """The adaptive mode's goal per component (errormode all):
    |error| <= max(epsabs, epsrel |integral|) for the real and the imaginary part."""
    I, E = res["integral"], res["error"]
    return (abs(E.real) <= max(epsabs, epsrel * abs(I.real)) and
            abs(E.imag) <= max(epsabs, epsrel * abs(I.imag)))


def run_serve_workload(args):
    """Serving: Poisson arrivals of integrals with error targets, served by continuous
    batching (qmc_server) and, for the same arrival stream, one integral at a time
    (qmc_integrate, adaptive).  Reports p50/p99 latency (arrival to completion),
    integrals/s and the number of goals met for both.  Profiles:
      feynman  64 Feynman-parameter-like integrals (complex, d = 5, contour deformation
               with lam = 1, Korobov-3, m = 32; half with F > 0 on the cube, half with F
               changing sign inside), relative targets log-uniform in [1e-8, 1e-3], the
               default absolute target 1e-7 and an evaluation budget: GPU-bound requests;
      small    512 Genz integrals in d = 4 (product peak and Gaussian alternately,
               Korobov-3, m = 32), relative targets log-uniform in [1e-6, 1e-3], budget
               4e6 evaluations: requests of 3e4 to 1e6 evaluations (microseconds of GPU
               time), bound by launches and host round trips."""
    import torch

    import paper_1811_11720_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    table = q.GenvecTable.load()
    rng = np.random.default_rng(args.seed)
    small = args.serve_profile == "small"
    N = args.requests if not small or args.requests != 64 else 512
    rates = args.rates if args.rates else ([1000.0, 4000.0, 16000.0] if small else [2.0, 8.0, 32.0])
    maxeval = 4e6 if small and args.serve_maxeval == 3.2e7 else args.serve_maxeval
    reqs = []
    for i in range(N):
        if small:
            # alternately a d = 4 product peak (c_j = 5) and a d = 4 Gaussian from the Genz
            # ranges, relative targets log-uniform in [1e-6, 1e-3]: n from 1021 to ~3e4
            if i % 2 == 0:
                c, w = W.product_peak_params(4, args.seed + i)
                f = q.Integrand.genz(2, c, w)
            else:
                c, w = W.genz_params(4, 4, args.seed + i)
                f = q.Integrand.genz(4, c, w)
            eps = float(10 ** rng.uniform(-6, -3))
        else:
            # alternately Euclidean-like (F > 0 on the cube, beta = 0.6) and with F changing
            # sign inside (beta = 0.95); lam = 1 keeps F(z) away from zero
            beta = 0.6 if i % 2 == 0 else 0.95
            f = q.Integrand.polynomial(W.feynman_regular(args.seed + i, beta=beta, lam=1.0))
            eps = float(10 ** rng.uniform(-8, -3))
        reqs.append((f, eps))
    workload = ("genz_product_peak|gaussian_d4_korobov3_m32_eps1e-6..1e-3_poisson" if small else
                "feynman_regular_d5_beta0.6|0.95_lam1_korobov3_m32_eps1e-8..1e-3_poisson")
    out = {"metric": "served integrals/s", "unit": "integrals/s", "higher_is_better": True,
           "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload,
                      "requests": N, "maxeval": maxeval,
                      "step_evaluations": int(args.serve_step_evals)}, "rates": []}

    def arrivals(rate):
        r = np.random.default_rng(args.seed + int(rate * 1000))
        return np.cumsum(r.exponential(1.0 / rate, N))

    for rate in rates:
        t_arr = arrivals(rate)
        # continuous batching
        srv = q.Server(table, memory_budget=int(args.serve_budget), max_slots=256, m=M_SHIFTS,
                       step_evaluations=int(args.serve_step_evals))
        ids = [None] * N
        done_t = [None] * N
        t0 = time.perf_counter()
        nxt = 0
        open_ids = {}
        while nxt < N or open_ids:
            now = time.perf_counter() - t0
            while nxt < N and t_arr[nxt] <= now:
                f, eps = reqs[nxt]
                ids[nxt] = srv.submit(f, epsrel=eps, epsabs=SERVE_EPSABS, minn=1021,
                                      maxeval=int(maxeval), seed=nxt)
                open_ids[ids[nxt]] = nxt
                nxt += 1
            if open_ids:
                srv.step()
                tnow = time.perf_counter() - t0
                for rid in srv.completed():
                    done_t[open_ids.pop(rid)] = tnow
            elif nxt < N:
                time.sleep(max(0.0, t_arr[nxt] - (time.perf_counter() - t0)))
        span_b = max(done_t) - t_arr[0]
        lat_b = np.array(done_t) - t_arr
        res_b = [srv.status(ids[i]) for i in range(N)]
        met_b = sum(goal_met(res_b[i], reqs[i][1]) for i in range(N))
        srv.close()
        # one integral at a time, FIFO, same arrivals
        done_s = [None] * N
        t0 = time.perf_counter()
        res_s = []
        for i in range(N):
            now = time.perf_counter() - t0
            if t_arr[i] > now:
                time.sleep(t_arr[i] - now)
            f, eps = reqs[i]
            r = q.integrate(f, table, 1021, M_SHIFTS, ("korobov", 3), seed=i,
                            opts=q.options(epsrel=eps, epsabs=SERVE_EPSABS, maxeval=int(maxeval)))
            done_s[i] = time.perf_counter() - t0
            res_s.append(r)
        span_s = max(done_s) - t_arr[0]
        lat_s = np.array(done_s) - t_arr
        same = all(rb["integral"] == rs["integral"] for rb, rs in zip(res_b, res_s))
        diffs = [{"request": i, "n": [int(res_b[i]["n"]), int(res_s[i]["n"])],
                  "evaluations": [int(res_b[i]["evaluations"]), int(res_s[i]["evaluations"])],
                  "rel_diff": float(abs(res_b[i]["integral"] - res_s[i]["integral"]) /
                                    max(abs(res_s[i]["integral"]), 1e-300))}
                 for i in range(N) if res_b[i]["integral"] != res_s[i]["integral"]]
        met_s = sum(goal_met(res_s[i], reqs[i][1]) for i in range(N))
        ok_b = np.array([goal_met(res_b[i], reqs[i][1]) for i in range(N)], dtype=bool)
        ok_s = np.array([goal_met(res_s[i], reqs[i][1]) for i in range(N)], dtype=bool)

        def pcts(lat, ok):
            # latency over all requests, and over those that reached their error goal
            d = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))}
            if ok.any():
                d["goal_met_p50_s"] = float(np.percentile(lat[ok], 50))
                d["goal_met_p99_s"] = float(np.percentile(lat[ok], 99))
            return d

        out["rates"].append({
            "rate_per_s": rate,
            "batched": {"integrals_per_s": N / span_b, **pcts(lat_b, ok_b), "goal_met": int(met_b)},
            "one_at_a_time": {"integrals_per_s": N / span_s, **pcts(lat_s, ok_s),
                              "goal_met": int(met_s)},
            "same_results": bool(same),
            **({"mismatches": len(diffs), "mismatch_examples": diffs[:4]} if diffs else {})})
    best = out["rates"][-1]
    out["value"] = best["batched"]["integrals_per_s"]
    out["p50_s"] = best["batched"]["p50_s"]
    out["p99_s"] = best["batched"]["p99_s"]
    return out


def cpu_baseline(budget_s: float, items, nthreads: int | None = None):
    """The oracle as it stands on the host cores: per-shift sums over a bounded prefix of
    the same lattices, scaled to evaluations per second."""
    import oracle as O
    from oracle import load_genvec_table
    tab = load_genvec_table(os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt"))
    z = tab[N_LATTICE]
    nthreads = nthreads or os.cpu_count()
    # calibrate the prefix length on the first item, then give every item the same share
    def integrand(fam, c, w):
        if fam == SECTOR_FAMILY:
            return O.from_feynman(c)
        return O.feynman_complex(c) if fam == FEYNMAN_FAMILY else O.genz(fam, c, w)

    fam, d, tr, c, w = items[0]
    D = O.shifts(1, M_SHIFTS, d)
    t0 = time.perf_counter()
    O.shift_sums(integrand(fam, c, w), tr, N_LATTICE, z, D, i0=0, i1=2048, nthreads=nthreads)
    dt = time.perf_counter() - t0
    rate = 2048 * M_SHIFTS / max(dt, 1e-6)
    per_item = max(1024, int(budget_s / len(items) * rate / M_SHIFTS))
    per_item = min(per_item, N_LATTICE)
    evals = 0
    t0 = time.perf_counter()
    for (fam, d, tr, c, w) in items:
        D = O.shifts(1, M_SHIFTS, d)
        O.shift_sums(integrand(fam, c, w), tr, N_LATTICE, z, D, i0=0, i1=per_item, nthreads=nthreads)
        evals += per_item * M_SHIFTS
    el = time.perf_counter() - t0
    return {"value": evals / el, "unit": "evals/s", "cores": nthreads, "kind": "oracle",
            "sample": f"first {per_item} lattice points x {M_SHIFTS} shifts of each of the "
                      f"{len(items)} integrals ({evals} evaluations, {el:.1f} s)"}


def roofline(r, workload: str):
    """The dominant kernel's roofline (see the module docstring) from the live per-launch
    CUDA-event time and the unit peaks measured in the same process."""
    pk = r["unit_peaks"]
    if not r["kernel_ms_per_launch"] or not pk:
        return None
    launches = len(r["items"])
    sec = r["kernel_ms_per_launch"] / 1e3
    flops = r["flops_per_step"] / launches / sec / 1e9          # GFLOP/s of counted FP64 work
    fp64 = {"achieved": round(flops, 1), "peak": round(pk["fp64_gflops"], 1), "unit": "GFLOP/s",
            "frac": round(flops / pk["fp64_gflops"], 4),
            "note": "the method's FP64 work (fp64_flops_per_eval, Sec. 2.3 maps + Sec. 5.2 "
                    "forms) per second against the measured FP64 FMA rate"}
    common = {"traffic": TRAFFIC_BYTES_PER_LAUNCH if workload == "genz" else None,
              "kernel": "sums_kernel (+ tile reduction, <0.1%)",
              "per_launch_ms": round(r["kernel_ms_per_launch"], 4), "peaks": pk}
    if workload == "sector":
        # F's Horner form runs on the integer pipe; U, the power, weight and accumulation
        # keep the FP64 pipe the busier unit
        kf = r["tensor_flops_per_step"] / launches / sec / 1e9
        fp64["note"] = ("term-by-term FP64 work of U and F (sector_flops_per_eval) against "
                        "the measured FP64 FMA rate")
        muls = r["muls_per_step"] / launches / sec / 1e9
        int_pipe = {"achieved": round(muls, 1), "peak": round(pk["int_mul_gops"], 1),
                    "unit": "G int32 mul/s", "frac": round(muls / pk["int_mul_gops"], 4),
                    "work": "sector_int_mul_per_eval: F's fixed-point Horner form, integer "
                            "Korobov map and weight"}
        return {"bound": "alu", "unit": "GFLOP/s", "achieved": round(kf, 1),
                "peak": round(pk["fp64_gflops"], 1), "frac": round(kf / pk["fp64_gflops"], 4),
                "peak_source": "measured FP64 FMA rate (qmc_probe_units), 2 flops per FMA",
                "work": "sector_kernel_flops_per_eval: the FP64 part of the kernel's form",
                "int_pipe": int_pipe, "fp64_equivalent": fp64, **common}
    if workload == "feynman":
        # the FP64 pipe bounds the complex family: the symmetric-tensor form's FP64 work
        # against the measured FMA rate; the term-by-term count of the polynomials is the
        # FP64-equivalent rate
        kf = r["tensor_flops_per_step"] / launches / sec / 1e9
        fp64["note"] = ("term-by-term FP64 work of U, F and their derivatives "
                        "(feynman_flops_per_eval) against the measured FP64 FMA rate")
        muls = r["muls_per_step"] / launches / sec / 1e9
        int_pipe = {"achieved": round(muls, 1), "peak": round(pk["int_mul_gops"], 1),
                    "unit": "G int32 mul/s", "frac": round(muls / pk["int_mul_gops"], 4),
                    "work": "feynman_int_mul_per_eval: integer Korobov map and weight, "
                            "fixed-point Hessian and contractions"}
        return {"bound": "alu", "unit": "GFLOP/s", "achieved": round(kf, 1),
                "peak": round(pk["fp64_gflops"], 1), "frac": round(kf / pk["fp64_gflops"], 4),
                "peak_source": "measured FP64 FMA rate (qmc_probe_units), 2 flops per FMA",
                "work": "feynman_tensor_flops_per_eval: the symmetric-tensor form's FP64 part",
                "int_pipe": int_pipe, "fp64_equivalent": fp64, **common}
    muls = r["muls_per_step"] / launches / sec / 1e9            # G 32-bit multiplies/s
    return {"bound": "alu", "unit": "G int32 mul/s", "achieved": round(muls, 1),
            "peak": round(pk["int_mul_gops"], 1), "frac": round(muls / pk["int_mul_gops"], 4),
            "peak_source": "measured rate of the kernel's truncated 64-bit high product "
                           "(qmc_probe_units), in 32-bit multiplies",
            "work": "int_mul_per_eval: the fixed-point map, forms and finishes",
            "fp64_equivalent": fp64, **common}


EXTRA_BATCH_COUNT = 48
EXTRA_SERVE_REQUESTS = 32
EXTRA_SERVE_RATE = 16.0
# evaluations per request: ~0.45 s of GPU time for the hardest requests (F changing sign,
# goals near 1e-8 need ~3e9, which does not fit a bounded run: those stop at the budget)
EXTRA_SERVE_MAXEVAL = 3.2e8


def run_extras(args) -> dict:
    """Bounded runs of the other configurations, each with its own config, after the main
    timed region (none of them enters `value`): the d = 4 product-peak integral's latency,
    the d = 5 complex Feynman-parameter family's evaluation rate on n = 10,560,653, a batch
    of EXTRA_BATCH_COUNT sector integrals with n log-uniform in [1e4, 1e8] (batched vs one
    launch per integral) and Poisson-arrival serving of EXTRA_SERVE_REQUESTS complex
    integrals at EXTRA_SERVE_RATE per second.  A failure is reported in its object."""
    out = {}

    def ns(**kw):
        d = dict(vars(args))
        d.update(kw)
        return argparse.Namespace(**d)

    def guarded(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:          # keep the main line; report the failure
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)

    def latency():
        r = run_latency_workload(ns(steps=1))
        return {k: r[k] for k in ("metric", "unit", "config", "value", "host_buffers",
                                  "device_entry_points", "cuda_graph", "device_evals_per_s")}

    def feynman():
        a = ns(workload="feynman", steps=2, warmup=1, e2e_steps=0, kernel_events=True, only=None)
        r = run_gpu(a, 0, 1)
        items = workload_items(0, None, "feynman")
        return {"metric": "FP64 integrand evals/sec", "unit": "evals/s",
                "value": r["evals_per_step"] * a.steps / (r["total_ms"] / 1e3),
                "config": {"workload": f"feynman_regular_d5_complex_korobov3_n{args.n}_m32",
                           "integrals_per_step": len(items), "steps": a.steps},
                "roofline": roofline(r, "feynman"), "nonfinite": r["nonfinite"]}

    def batch():
        return run_batch_workload(ns(batch_count=EXTRA_BATCH_COUNT, batch_nmax=1e8, steps=1,
                                     batch_warm=1))

    def serve():
        r = run_serve_workload(ns(requests=EXTRA_SERVE_REQUESTS, rates=[EXTRA_SERVE_RATE],
                                  serve_profile="feynman", serve_maxeval=EXTRA_SERVE_MAXEVAL))
        return r

    def serve_small():
        # launch-bound requests: 512 small d = 4 Genz integrals at 16,000 arrivals/s
        return run_serve_workload(ns(requests=64, rates=[16000.0], serve_profile="small",
                                     serve_maxeval=3.2e7))

    def small_lattice():
        # the 45 Genz integrals on the table size just above 1e5 (launch-bound regime):
        # the step as the main line runs it, and the same step replayed from a CUDA graph
        n = 108863
        plain = run_gpu(ns(n=n, steps=5, warmup=3, e2e_steps=0, kernel_events=True), 0, 1)
        graphed = run_gpu(ns(n=n, steps=5, warmup=3, e2e_steps=0, kernel_events=False,
                             graph=True, skip_peaks=True), 0, 1)
        ev = plain["evals_per_step"] * 5
        return {"metric": "FP64 integrand evals/sec", "unit": "evals/s",
                "config": {"workload": f"genz_osc_corner_gauss_d6_8_10_baker_korobov1-4_n{n}_m32",
                           "integrals_per_step": 45, "steps": 5},
                "value": ev / (plain["total_ms"] / 1e3),
                "cuda_graph_value": ev / (graphed["total_ms"] / 1e3),
                "kernel_only_value": plain["evals_per_step"] / (plain["kernel_ms_per_launch"] * 45 / 1e3),
                "roofline": roofline(plain, "genz")}

    guarded("latency", latency)
    guarded("small_lattice", small_lattice)
    guarded("feynman", feynman)
    guarded("batch", batch)
    guarded("serve", serve)
    guarded("serve_small", serve_small)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=20181128)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-kernel-events", dest="kernel_events", action="store_false")
    ap.add_argument("--only", default=None, help="FAMILY:D:TRANSFORM, e.g. 4:10:korobov3")
    ap.add_argument("--n", type=int, default=N_LATTICE, help="lattice size (a table size)")
    ap.add_argument("--workload", default="genz",
                    choices=["genz", "feynman", "feynman_like", "sector", "batch", "serve",
                             "latency"])
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rates", type=float, nargs="*", default=None,
                    help="arrival rates per second (default: 2 8 32 for the Feynman profile, "
                         "500 2000 8000 for the small profile)")
    ap.add_argument("--serve-profile", default="feynman", choices=["feynman", "small"],
                    help="serve workload: Feynman-parameter integrals (GPU-bound requests) or "
                         "small Genz integrals (launch-bound requests)")
    ap.add_argument("--serve-maxeval", type=float, default=3.2e7)
    ap.add_argument("--serve-budget", type=float, default=4e9)
    ap.add_argument("--serve-step-evals", type=float, default=2.0 ** 25,
                    help="server step budget in evaluations (0: all running requests each step)")
    ap.add_argument("--batch-count", type=int, default=2000)
    ap.add_argument("--batch-nmax", type=float, default=1e8)
    ap.add_argument("--per-item", action="store_true",
                    help="add each integral's mean lattice-sum launch time (ms) to the line")
    ap.add_argument("--graph", action="store_true",
                    help="replay each timed step from a CUDA graph (host launch work out of "
                         "the timed region; no per-launch kernel events)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the bounded latency/feynman/batch/serve runs after the main line")
    args = ap.parse_args()
    if args.workload == "batch":
        print(json.dumps(run_batch_workload(args)))
        return
    if args.workload == "serve":
        print(json.dumps(run_serve_workload(args)))
        return
    if args.workload == "latency":
        print(json.dumps(run_latency_workload(args)))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    base = {"metric": "FP64 integrand evals/sec", "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"{'feynman_regular' if args.workload == 'feynman' else 'feynman_like'}"
                                    f"_d5_complex_korobov3_n{args.n}_m32"
                                    if args.workload in ("feynman", "feynman_like") else
                                    f"sector_like_d{SECTOR_D}_terms{SECTOR_TERMS}_korobov3_n{args.n}_m32"
                                    if args.workload == "sector" else
                                    f"genz_osc_corner_gauss_d6_8_10_baker_korobov1-4_n{args.n}_m32"
                                    if not args.only else f"genz_{args.only}_n{args.n}_m32"),
                       "integrals_per_step": len(workload_items(0, args.only, args.workload)),
                       "n": args.n, "m": M_SHIFTS, "l2": "flushed between steps",
                       "parallelism": f"replicas x{args.gpus} (independent integrals per rank)"}}

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo", init_method="env://")
            if rank != 0:
                dist.destroy_process_group()
                return
        items = workload_items(0, args.only, args.workload)
        per_step = []
        samples = []
        for _ in range(args.warmup):
            cpu_baseline(min(2.0, args.cpu_budget), items)
        for _ in range(args.steps):
            cb = cpu_baseline(args.cpu_budget / max(1, args.steps) * 2, items)
            per_step.append(cb["value"])
            samples.append(cb["sample"])
        v = float(np.mean(per_step))
        line = dict(base)
        line.update({"impl": "reference", "value": v, "ms_per_step": None,
                     "cpu_baseline": {"value": v, "unit": "evals/s", "cores": os.cpu_count(),
                                      "kind": "oracle", "sample": samples[-1]},
                     "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                             "d2h_bytes_per_step": 0}})
        print(json.dumps(line))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    r = run_gpu(args, rank, world)
    evals_total = r["evals_per_step"] * args.steps * world
    value = evals_total / (r["total_ms"] / 1e3)
    e2e_value = (r["evals_per_step"] * r["e2e_steps"] * world / (r["e2e_total_ms"] / 1e3)
                 if r["e2e_total_ms"] > 0 else None)
    clk = r["clocks"]
    roof = (roofline(r, "feynman" if args.workload == "feynman_like" else args.workload)
            if rank == 0 else None)
    if rank == 0:
        line = dict(base)
        line.update({
            "value": value, "ms_per_step": r["total_ms"] / args.steps,
            "e2e": {"value": e2e_value, "unit": "evals/s",
                    "h2d_bytes_per_step": r["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": r["d2h_bytes_per_step"]},
            "gpu_launches": r["launches_per_step"] * args.steps,
            "roofline": roof,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons")},
            "nonfinite": r["nonfinite"],
            **({"kernel_ms_per_item": r["kernel_ms_per_item"]} if args.per_item else {}),
        })
        if world == 1 and args.cpu_budget > 0:
            line["cpu_baseline"] = cpu_baseline(args.cpu_budget, workload_items(0, args.only, args.workload))
        if world == 1 and args.extras and args.workload == "genz" and not args.only:
            line.update(run_extras(args))
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
