"""Batches (many integrals in one launch) against one launch per integral and the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1811_11720_gb300 as q
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1811_11720_gb300 import build
    build.build()
    q.lib()
    return q, torch, torch.device("cuda:0"), q.GenvecTable.load()


def _entry(env, f, n, d, m, seed, tr, fitp=None, i0=0, i1=None):
    q, torch, dev, tab = env
    D = q.make_shifts(seed, m, d)
    Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
    fd = None if fitp is None else torch.from_numpy(np.ascontiguousarray(fitp)).to(dev)
    r = q.rule(n, tab.z_for(n)[:d], Dd, tr, fd)
    return (f.device_struct(dev), r, i0, n if i1 is None else i1), D


def _single(env, entry):
    q, torch, dev, _ = env
    fs, r, a, b = entry
    ws = torch.empty(max(8, q.sums_workspace_bytes(r, fs.family == 20, a, b)), dtype=torch.uint8, device=dev)
    out = torch.zeros(4 * r.m, dtype=torch.float64, device=dev)
    q.sums(fs, r, a, b, ws, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _genz_batch(env, count, seed0=0):
    q = env[0]
    rng = np.random.default_rng(seed0)
    entries, meta = [], []
    sizes = [1021, 4691, 108863, 1072187]
    for i in range(count):
        fam = 4
        d = int(rng.integers(2, 11))
        n = int(sizes[rng.integers(0, len(sizes))])
        tr = [("korobov", 3), ("baker",), ("korobov", 1), ("none",)][i % 4]
        c, w = W.genz_params(fam, d, 100 + i)
        fitp = W.fit_params_example(d, i) if i % 2 else None
        f = q.Integrand.genz(fam, c, w)
        e, D = _entry(env, f, n, d, 16, 500 + i, tr, fitp)
        entries.append(e)
        meta.append((fam, d, n, tr, c, w, fitp, D, f))
    return entries, meta


def test_batch_default_shape_is_bit_identical_to_single_launches(env):
    q, torch, dev, tab = env
    entries, meta = _genz_batch(env, 24)
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    sums = torch.zeros(b.count, 4 * b.m, dtype=torch.float64, device=dev)
    res = torch.zeros(b.count, 4, dtype=torch.float64, device=dev)
    cnt = torch.zeros(b.count, 2, dtype=torch.int64, device=dev)
    b.sums(ws, sums, res, cnt)
    torch.cuda.synchronize()
    S = sums.cpu().numpy()
    for i, e in enumerate(entries):
        ref = _single(env, e)
        assert np.array_equal(S[i, : 2 * b.m], ref[: 2 * b.m]), i
    R = res.cpu().numpy()
    checked = 0
    for i, (fam, d, n, tr, c, w, fitp, D, f) in enumerate(meta):
        if n > 200000 or checked >= 6:
            continue
        checked += 1
        o = O.shift_sums(O.genz(fam, c, w), tr, n, [int(v) for v in tab.z_for(n)[:d]], D, fitp=fitp)
        Qo = (o["re"][:, 0] + o["re"][:, 1]) / n
        A = o["abs"] / n
        assert abs(R[i, 0] - Qo.mean()) <= 1e-12 * A.mean()
    assert not cnt.any().item()


def test_batch_tuned_shape_matches_oracle(env):
    q, torch, dev, tab = env
    entries, meta = _genz_batch(env, 40, seed0=3)
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    sums = torch.zeros(b.count, 4 * b.m, dtype=torch.float64, device=dev)
    cfg = b.autotune(ws, sums)
    assert cfg.points_per_stream in (16, 32, 64, 128, 256, 512)
    ws2 = torch.empty(b.workspace_bytes(cfg), dtype=torch.uint8, device=dev)
    sums.zero_()
    b.sums(ws2, sums, cfg=cfg)
    torch.cuda.synchronize()
    S = sums.cpu().numpy()
    for i, (fam, d, n, tr, c, w, fitp, D, f) in enumerate(meta):
        if n > 200000:
            continue   # the oracle is slow at n = 1e6; the default-shape test covers those
        o = O.shift_sums(O.genz(fam, c, w), tr, n, [int(v) for v in tab.z_for(n)[:d]], D, fitp=fitp)
        Sg = S[i, 0:2 * b.m:2] + S[i, 1:2 * b.m:2]
        So = o["re"][:, 0] + o["re"][:, 1]
        assert np.all(np.abs(Sg - So) <= 1e-12 * o["abs"]), i


def test_sector_batch_workload_shape(env):
    """The sector batch workload's shape at small n: sector integrands, d 3..8, 10..400
    monomials, fit on half, against single launches."""
    q, torch, dev, tab = env
    rng = np.random.default_rng(4)
    entries = []
    for i in range(12):
        d = int(rng.integers(3, 9))
        fl = W.sector_like(i, d, int(rng.integers(10, 400)), int(rng.integers(10, 400)))
        f = q.Integrand.polynomial(fl)
        fitp = W.fit_params_example(d, i) if i % 2 else None
        e, _ = _entry(env, f, 4691, d, 32, 700 + i, ("korobov", 3), fitp)
        entries.append(e)
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    sums = torch.zeros(b.count, 4 * b.m, dtype=torch.float64, device=dev)
    b.sums(ws, sums)
    torch.cuda.synchronize()
    S = sums.cpu().numpy()
    for i, e in enumerate(entries):
        assert np.array_equal(S[i, : 2 * b.m], _single(env, e)[: 2 * b.m])


def test_complex_batch(env):
    q, torch, dev, tab = env
    entries = []
    for i in range(3):
        fl = W.feynman_like(10 + i)
        e, _ = _entry(env, q.Integrand.polynomial(fl), 1021, 5, 8, 800 + i, ("korobov", 3))
        entries.append(e)
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    sums = torch.zeros(b.count, 4 * b.m, dtype=torch.float64, device=dev)
    cnt = torch.zeros(b.count, 2, dtype=torch.int64, device=dev)
    b.sums(ws, sums, counters=cnt)
    torch.cuda.synchronize()
    S = sums.cpu().numpy()
    for i, e in enumerate(entries):
        assert np.array_equal(S[i], _single(env, e))


def test_batch_plan_replays_in_a_cuda_graph(env):
    q, torch, dev, tab = env
    entries, _ = _genz_batch(env, 8, seed0=9)
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    sums = torch.zeros(b.count, 4 * b.m, dtype=torch.float64, device=dev)
    res = torch.zeros(b.count, 4, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    plan = b.plan(ws, stream=s)
    with torch.cuda.stream(s):
        plan.run(sums, res, stream=s)
    torch.cuda.synchronize()
    ref = sums.clone()
    sums.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(sums, res, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sums, ref)
    plan.close()


def test_batch_rejects_mixed_families_and_m(env):
    q, torch, dev, tab = env
    c, w = W.genz_params(4, 3, 1)
    e1, _ = _entry(env, q.Integrand.genz(4, c, w), 1021, 3, 8, 1, ("baker",))
    e2, _ = _entry(env, q.Integrand.genz(2, c, w), 1021, 3, 8, 2, ("baker",))
    e3, _ = _entry(env, q.Integrand.genz(4, c, w), 1021, 3, 16, 3, ("baker",))
    for bad in ([e1, e2], [e1, e3]):
        b = q.Batch(bad)
        assert b.workspace_bytes() == 0
        ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
        sums = torch.zeros(2, 64, dtype=torch.float64, device=dev)
        with pytest.raises(q.QMCError) as e:
            b.sums(ws, sums)
        assert e.value.code == -1
