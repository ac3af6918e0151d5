"""The benchmark's workload definition and its FP64 work count, on the CPU: the 45 Genz
integrals (families 1, 3, 4 x d = 6, 8, 10 x baker and Korobov-1..4) with seeded
parameters in the paper's difficulty ranges (Sec. 5.2), the single-integral selection used
for profiling, and the per-evaluation FP64 count behind the roofline's `achieved` (the
method's FP64 work: Korobov-r costs (2r+1) fma + (r+2) mul + 1 mul per dimension, baker 2,
the family's form and its final function, and the weighted accumulation)."""
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
    (4, ("korobov", 3), 10, 10 * (2 * 7 + 5 + 1) + 3 * 10 + 1 + 2),
    (1, ("baker",), 6, 2 * 6 + 2 * 6 + 1 + 2),
    (3, ("korobov", 1), 8, 8 * (2 * 3 + 3 + 1) + 2 * 8 + 4 + 1 + 2),
])
def test_fp64_work_count(fam, tr, d, expect):
    assert bench.fp64_flops_per_eval(fam, tr, d) == expect


def test_feynman_workload_shape():
    items = bench.workload_items(workload="feynman")
    assert len(items) == bench.FEYNMAN_INTEGRALS
    for fam, d, tr, fl, _ in items:
        assert fam == bench.FEYNMAN_FAMILY and d == 5 and tr == ("korobov", 3)
        assert bench.feynman_flops_per_eval(fl) > 500
