"""The benchmark's workload definition and its FP64 work count, on the CPU: the 45 Genz
integrals (families 1, 3, 4 x d = 6, 8, 10 x baker and Korobov-1..4) with seeded
parameters in the paper's difficulty ranges (Sec. 5.2), the single-integral selection used
for profiling, the per-evaluation FP64 count behind the roofline's `fp64_equivalent` (the
method's FP64 work: Korobov-r costs (2r+1) fma + (r+2) mul + 1 mul per dimension, baker 2,
the point's add and compare per dimension, the family's form and its final function, and
the weighted accumulation), and the integer-multiply count behind its `achieved` (the
fixed-point form's 32-bit multiplies, restated here from the primitives' definitions)."""
from __future__ import annotations

import pytest

import bench
import workloads as W


def test_default_workload_is_45_integrals():
    items = bench.workload_items()
    assert len(items) == 45
    keys = {(f, d, tr) for f, d, tr, _, _ in items}
    assert len(keys) == 45
    assert {f for f, *_ in items} == {1, 3, 4}
    assert {d for _, d, *_ in items} == {6, 8, 10}
    assert {tr for _, _, tr, _, _ in items} == set(bench.TRANSFORMS)
    for f, d, tr, c, w in items:
        assert len(c) == d and len(w) == d
        assert abs(c.sum() - W.GENZ_DIFFICULTY[f]) < 1e-12 * W.GENZ_DIFFICULTY[f]
        assert (c > 0).all() and (w >= 0).all() and (w <= 1).all()


def test_replica_ranks_draw_distinct_parameters():
    a, b = bench.workload_items(0), bench.workload_items(1)
    assert [it[:3] for it in a] == [it[:3] for it in b]
    assert any((x[3] != y[3]).any() for x, y in zip(a, b))


def test_only_selects_one_integral():
    (it,) = bench.workload_items(only="4:10:korobov3")
    assert it[:3] == (4, 10, ("korobov", 3))
    with pytest.raises(ValueError):
        bench.workload_items(only="2:10:korobov3")


@pytest.mark.parametrize("fam,tr,d,expect", [
    (4, ("korobov", 3), 10, 10 * (2 * 7 + 5 + 1) + 3 * 10 + 1 + 2 + 2 * 10),
    (1, ("baker",), 6, 2 * 6 + 2 * 6 + 1 + 2 + 2 * 6),
    (3, ("korobov", 1), 8, 8 * (2 * 3 + 3 + 1) + 2 * 8 + 4 + 1 + 2 + 2 * 8),
])
def test_fp64_work_count(fam, tr, d, expect):
    assert bench.fp64_flops_per_eval(fam, tr, d) == expect


def test_feynman_workload_shape():
    items = bench.workload_items(workload="feynman")
    assert len(items) == bench.FEYNMAN_INTEGRALS
    for fam, d, tr, fl, _ in items:
        assert fam == bench.FEYNMAN_FAMILY and d == 5 and tr == ("korobov", 3)
        assert bench.feynman_flops_per_eval(fl) > 500


# 32-bit multiplies of the fixed-point primitives: a truncated 64-bit high product takes
# three (32x32->64 of the high halves, two 32-bit high cross products), its square two.
@pytest.mark.parametrize("r,expect", [
    # v^2 (2) + P(w): r=1 none, r=2,3 one product (3), r=4 product + square + product (8)
    # + v^(r+1): r=1 none (v^2), r=2 v^2 v (3), r=3 (v^2)^2 (2), r=4 (v^2)^2 v (5)
    # + phi = v^(r+1) P (3) + the weight factor into the running product (3)
    (1, 2 + 0 + 0 + 3 + 3), (2, 2 + 3 + 3 + 3 + 3), (3, 2 + 3 + 2 + 3 + 3),
    (4, 2 + 8 + 5 + 3 + 3)])
def test_korobov_map_multiplies(r, expect):
    assert bench.korobov_map_muls(r) == expect


@pytest.mark.parametrize("fam,tr,d,expect", [
    # Gaussian, Korobov-3, d = 10: map 13 + form (product 3 + square 2) per dimension,
    # weight^3 (square 2 + product 3) times C^d (3), integer exp (Tang: 31)
    (4, ("korobov", 3), 10, 10 * (13 + 5) + (2 + 3 + 3) + 31),
    # Gaussian, Korobov-4: the exp is in FP64 above r = 3
    (4, ("korobov", 4), 10, 10 * (21 + 5) + (2 + 2 + 3)),
    # oscillatory, baker, d = 6: one product per dimension and the cos in turns (29)
    (1, ("baker",), 6, 6 * 3 + 29),
    # corner peak, Korobov-1, d = 8: the 9th power (3 squares, 1 product) and reciprocal (22)
    (3, ("korobov", 1), 8, 8 * (8 + 3) + 3 + (3 * 2 + 3) + 22),
    # corner peak, Korobov-2: FP64 power and division above r = 1
    (3, ("korobov", 2), 8, 8 * (14 + 3) + (2 + 3)),
])
def test_int_multiply_work_count(fam, tr, d, expect):
    assert bench.int_mul_per_eval(fam, tr, d) == expect


def test_int_multiply_work_is_positive_for_the_benchmark():
    for fam, d, tr, c, _ in bench.workload_items():
        assert bench.int_mul_per_eval(fam, tr, d, c) > 0



def test_complex_family_work_split():
    """d = 3..6 evaluate the Hessian and the contractions in fixed point: 150 truncated
    high products for d = 5 (75 Hessian terms, 25 each for H x, F2 x, U2 x) on top of the
    Korobov-3 map and weight; the FP64 count keeps the nested-form values F(x) (55 fused
    multiply-adds) and U(x) (20) of that part, and the Taylor terms at y take the upper
    triangle and the nested forms, det J the symmetric elimination.  d = 7 keeps the
    all-FP64 form."""
    assert bench.feynman_fixed_int_mul_per_eval(5) == bench.MUL_HI * 150
    assert bench.feynman_int_mul_per_eval(("korobov", 3), 5) == (
        bench.MUL_HI * 150 + 5 * bench.korobov_map_muls(3) + bench.korobov_weight_muls(3))
    assert bench.feynman_fixed_int_mul_per_eval(7) == 0
    # FP64 form for d = 5: Hessian 15 * 6 and gradient/values 5 * 21 fma, 12 adds; Taylor
    # terms 5 * 14 + 15 * 6 + 2 fma, 30 mul, 1 add
    fp64_form = 2 * (15 * 6 + 5 * 21) + 12 + 2 * (70 + 90 + 2) + 30 + 1
    # values 55 + 20 fma; Taylor terms 10 + 10 + 10 fma and 5 mul (y.H y, g.y, grad U.y),
    # 35 + 30 + 10 fma (nested cubic and quadratic at y), 1 fma, 2 adds
    fixed_form = 2 * (55 + 20) + 2 * (30 + 75 + 1) + 5 + 2
    # det J: general elimination of the formed J (122 fma, 70 mul, 4 reciprocals) against
    # the symmetric elimination of diag(1 + i Lambda) + diag(lx) i H (88 fma, 68 mul, 4)
    fp64_form += 2 * 122 + 70 + 4
    fixed_form += 2 * 88 + 68 + 4
    assert bench.feynman_tensor_flops_per_eval(5) == 1139 - fp64_form + fixed_form
    assert bench.feynman_tensor_flops_per_eval(7) > bench.feynman_tensor_flops_per_eval(6)


def test_sector_work_counts():
    """The sector kernel's integer work equals the products of the fixed-point Horner loop
    (x_d = 1 iterations taken as additions), counted here by walking that loop, plus the
    Korobov-3 map and weight; its FP64 work is U's dense quadratic walked the same way,
    the power, weight and accumulation."""
    for d in range(3, 9):
        V = d + 1
        prods = 0
        for a in range(V - 1):
            for b in range(a, V - 1):
                prods += (V - 1) - b          # c = b .. V - 2
                prods += 1                    # sa += X_b t
            prods += 1                        # F += X_a sa
        assert bench.sector_int_mul_per_eval(("korobov", 3), d) == (
            bench.MUL_HI * prods + d * bench.korobov_map_muls(3) + bench.korobov_weight_muls(3))
        fma = adds = 0
        for a in range(V):
            fma += (V - 1) - a                # b = a .. V - 2
            adds += 1                         # t + C (b = V - 1)
            if a < V - 1:
                fma += 1
            else:
                adds += 1
        assert bench.sector_kernel_flops_per_eval(d) == 2 * fma + adds + 5 + 2 + 2
    assert len(bench.workload_items(0, None, "sector")) == bench.SECTOR_INTEGRALS


def test_roofline_fractions_follow_from_the_counts():
    """roofline() turns the per-step counts and the per-launch time into achieved rates
    and fractions of the measured peaks, per workload (binding unit first)."""
    pk = {"fp64_gflops": 1000.0, "int_mul_gops": 8000.0}
    evals = 1e9                                   # per launch
    for workload, key, per_eval in (("genz", "muls_per_step", 200),
                                    ("feynman", "tensor_flops_per_step", 700),
                                    ("sector", "tensor_flops_per_step", 100)):
        r = {"unit_peaks": pk, "kernel_ms_per_launch": 500.0, "items": [0, 1],
             "flops_per_step": 2 * evals * 50, "muls_per_step": 2 * evals * 300,
             "tensor_flops_per_step": 2 * evals * per_eval}
        if key == "muls_per_step":
            r["muls_per_step"] = 2 * evals * per_eval
        roof = bench.roofline(r, workload)
        assert roof["bound"] == "alu"
        rate = evals * per_eval / 0.5 / 1e9        # per second, G units
        peak = pk["int_mul_gops"] if workload == "genz" else pk["fp64_gflops"]
        assert roof["achieved"] == pytest.approx(rate, rel=1e-3)
        assert roof["frac"] == pytest.approx(rate / peak, rel=1e-3)
        assert roof["fp64_equivalent"]["frac"] == pytest.approx(evals * 50 / 0.5 / 1e9 / 1000.0, rel=1e-3)
        if workload != "genz":
            assert roof["int_pipe"]["frac"] == pytest.approx(evals * 300 / 0.5 / 1e9 / 8000.0, rel=1e-3)
        assert (roof["traffic"] is not None) == (workload == "genz")
