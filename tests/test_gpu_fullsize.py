"""GPU parity at the benchmark's full sizes (Sec. 2.1, Eq. (lattice)).

The benchmark integrates 45 Genz integrals (families 1, 3, 4 in d = 6, 8, 10 under baker
and Korobov-1..4) on n = 10,560,653 points with m = 32 shifts; the paper's sweep reaches
n ~ 1e9.  At those sizes the oracle cannot afford whole lattices, so the CUDA path is
checked tile by tile: qmc_sums leaves the per-tile partial sums of its decomposition in
the caller's workspace, and randomly chosen tiles (always including the ragged last one)
are recomputed by the oracle over exactly the tile's i-range.  These launches use the
streams of the sizes the benchmark times: 290 points per stream at n = 1.06e7 and 8192 at
n = 1.02e9, so the 64-sample inner blocks are flushed 4 and 128 times per stream, and
hundreds to thousands of consecutive lattice steps run from each stream start.  One
whole-lattice comparison with more than 64 points per stream closes the fold over tiles.

Tolerance: |S_gpu - S_oracle| <= 1e-12 * sum |g| over the same points, per shift, and
relative 1e-12 of S itself wherever S is not cancelled (|S| >= 0.1 sum |g|)."""
import numpy as np
import pytest

import bench
import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
M = 32
D_BENCH = 10
SEED = 20181128           # bench.py's default seed


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


def _bench_item(fam, tr):
    """The benchmark's own integral for (family, d = 10, transform) and its shift seed."""
    for idx, it in enumerate(bench.workload_items(0)):
        if it[0] == fam and it[1] == D_BENCH and it[2] == tr:
            return it, SEED + idx
    raise KeyError((fam, tr))


def _check_sums(S_gpu, S_or, A, what):
    dev = np.abs(S_gpu - S_or)
    assert np.all(dev <= TOL * A), (what, float(np.max(dev / A)))
    big = np.abs(S_or) >= 0.1 * A
    assert np.all(dev[big] <= TOL * np.abs(S_or[big])), (what, float(np.max(dev[big] / np.abs(S_or[big]))))
    return float(np.max(dev / A))


def _full_launch(env, fam, tr, n):
    """qmc_sums over [0, n) with the benchmark's inputs; returns everything a tile check needs."""
    q, torch, dev, tab = env
    (f_, d, t_, c, w), seed = _bench_item(fam, tr)
    D = O.shifts(seed, M, d)
    z = tab.z_for(n)[:d]
    Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
    r = q.rule(n, z, Dd, tr)
    fd = q.Integrand.genz(fam, c, w).device_struct(dev)
    ws = torch.empty(q.sums_workspace_bytes(r, False, 0, n), dtype=torch.uint8, device=dev)
    sums = torch.zeros(4 * M, dtype=torch.float64, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    q.sums(fd, r, 0, n, ws, sums, cnt)
    torch.cuda.synchronize()
    tiles, ppt = q.sums_tile_count(n, M)
    part = ws[: tiles * M * 16].view(torch.float64).cpu().numpy().reshape(tiles, M, 2)
    return dict(q=q, torch=torch, dev=dev, fd=fd, r=r, c=c, w=w, D=D, z=z, d=d, tiles=tiles,
                ppt=ppt, part=part, sums=sums.cpu().numpy(), cnt=cnt.cpu().numpy())


def _tiles_against_oracle(L, fam, tr, n, picks):
    q, torch, dev = L["q"], L["torch"], L["dev"]
    worst = 0.0
    for t in picks:
        a = t * L["ppt"]
        b = min(a + L["ppt"], n)
        o = O.shift_sums(O.genz(fam, L["c"], L["w"]), tr, n, L["z"], L["D"], i0=a, i1=b)
        S_gpu = L["part"][t, :, 0] + L["part"][t, :, 1]
        S_or = o["re"][:, 0] + o["re"][:, 1]
        worst = max(worst, _check_sums(S_gpu, S_or, o["abs"], (fam, tr, n, t)))
        # the single-tile entry point reproduces the full launch's tile bit for bit
        one = torch.empty(2 * M, dtype=torch.float64, device=dev)
        q.sums_tiles(L["fd"], L["r"], 0, n, t, t + 1, one)
        torch.cuda.synchronize()
        assert np.array_equal(one.cpu().numpy().reshape(M, 2), L["part"][t]), (fam, tr, n, t)
    return worst


def _picks(tiles, k, seed):
    rng = np.random.default_rng(seed)
    inner = rng.choice(tiles - 1, size=k - 1, replace=False)
    return sorted(int(t) for t in inner) + [tiles - 1]


@pytest.mark.parametrize("fam", bench.FAMILIES)
@pytest.mark.parametrize("tr", bench.TRANSFORMS)
def test_bench_size_tiles_match_oracle(env, fam, tr):
    """n = 10,560,653 (the benchmark's lattice), m = 32, d = 10: five tiles of the full
    launch (290 points per stream) against the oracle."""
    n = bench.N_LATTICE
    L = _full_launch(env, fam, tr, n)
    assert L["ppt"] == 8 * 290 and L["tiles"] == 4553
    worst = _tiles_against_oracle(L, fam, tr, n, _picks(L["tiles"], 5, fam * 10 + len(tr[0])))
    print(f"[parity] tiles n={n} fam={fam} {tr}: max |dS|/A = {worst:.2e}")
    assert L["cnt"][0] == 0


@pytest.mark.parametrize("fam", bench.FAMILIES)
@pytest.mark.parametrize("tr", bench.TRANSFORMS)
def test_largest_cpu_table_size_tiles_match_oracle(env, fam, tr):
    """n = 1,024,565,021 (the paper's sweep end), m = 32, d = 10: two tiles of the full
    launch (8192 points per stream, 65,536 points per tile) against the oracle."""
    n = 1024565021
    L = _full_launch(env, fam, tr, n)
    assert L["ppt"] == 8 * 8192
    worst = _tiles_against_oracle(L, fam, tr, n, _picks(L["tiles"], 2, fam * 100 + len(tr)))
    print(f"[parity] tiles n={n} fam={fam} {tr}: max |dS|/A = {worst:.2e}")
    assert L["cnt"][0] == 0


@pytest.mark.parametrize("fam,tr", [(4, ("korobov", 3)), (1, ("baker",))])
def test_whole_lattice_with_long_streams(env, fam, tr):
    """The whole lattice n = 2,528,147 (70 points per stream: the inner 64-sample block is
    flushed mid-stream) with m = 32 in d = 3: per-shift sums, mean and error of the full
    fold against the oracle's whole-range sums."""
    q, torch, dev, tab = env
    n, d = 2528147, 3
    tiles, ppt = q.sums_tile_count(n, M)
    assert ppt == 8 * 70
    c, w = W.genz_params(fam, d, 5)
    D = O.shifts(33, M, d)
    z = tab.z_for(n)[:d]
    Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
    res, sums, cnt = q.integrate_device(q.Integrand.genz(fam, c, w), n, z, Dd, tr)
    torch.cuda.synchronize()
    s = sums.cpu().numpy()[: 2 * M].reshape(M, 2)
    o = O.shift_sums(O.genz(fam, c, w), tr, n, z, D)
    S_or = o["re"][:, 0] + o["re"][:, 1]
    worst = _check_sums(s[:, 0] + s[:, 1], S_or, o["abs"], (fam, tr))
    print(f"[parity] whole n={n} fam={fam} {tr}: max |dS|/A = {worst:.2e}")
    qbar, sig = O.shift_reduce(S_or / n)
    res = res.cpu().numpy()
    A = o["abs"].mean() / n
    assert abs(res[0] - qbar) <= TOL * A
    assert abs(res[1] - sig) <= max(1e-9 * sig, 2e-12 * A)


@pytest.mark.parametrize("form", ["regular", "like"])
def test_complex_family_full_size_tiles_match_oracle(env, form):
    """The complex deformed family (the d = 5 Feynman-parameter workload of the
    benchmark's feynman object, and the configuration's literal polynomials) on
    n = 10,560,653 with m = 32: three tiles of the full launch, real and imaginary
    partials, against the oracle at 1e-12 of the tile's sum |g|."""
    q, torch, dev, tab = env
    n = bench.N_LATTICE
    fam, d, tr, fl, _ = bench.workload_items(0, workload="feynman" if form == "regular"
                                             else "feynman_like")[1]
    D = O.shifts(SEED + 1, M, d)
    z = tab.z_for(n)[:d]
    Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
    r = q.rule(n, z, Dd, tr)
    fd = q.Integrand.polynomial(fl).device_struct(dev)
    ws = torch.empty(q.sums_workspace_bytes(r, True, 0, n), dtype=torch.uint8, device=dev)
    sums = torch.zeros(4 * M, dtype=torch.float64, device=dev)
    q.sums(fd, r, 0, n, ws, sums)
    torch.cuda.synchronize()
    tiles, ppt = q.sums_tile_count(n, M)
    part = ws[: 2 * tiles * M * 16].view(torch.float64).cpu().numpy().reshape(2, tiles, M, 2)
    worst = 0.0
    for t in _picks(tiles, 3, 7 + len(form)):
        a, b = t * ppt, min(t * ppt + ppt, n)
        o = O.shift_sums(O.feynman_complex(fl), tr, n, z, D, i0=a, i1=b)
        for comp, key in ((0, "re"), (1, "im")):
            S_gpu = part[comp, t, :, 0] + part[comp, t, :, 1]
            S_or = o[key][:, 0] + o[key][:, 1]
            fin = np.isfinite(S_or)
            worst = max(worst, _check_sums(S_gpu[fin], S_or[fin], o["abs"][fin], (form, t, key)))
            assert np.array_equal(np.isfinite(S_gpu), fin)
    print(f"[parity] complex {form} tiles n={n}: max |dS|/A = {worst:.2e}")


def test_batch_at_config4_sizes_equals_single_launches(env):
    """Sector integrals with n log-uniform in [1e4, 1e8] (the batching configuration's
    range) in one batched launch with the default shape: every item's sums equal a
    qmc_sums call on that item bit for bit, and one tile of the largest item matches the
    oracle."""
    q, torch, dev, tab = env
    rng = np.random.default_rng(11)
    entries, keep = [], []
    for i in range(5):
        d = int(rng.integers(3, 9))
        fl = W.sector_like(500 + i, d, int(rng.integers(10, 401)), int(rng.integers(10, 401)))
        n = q.get_next_n(tab, int(np.exp(rng.uniform(np.log(1e4), np.log(1e8)))))
        if i == 0:
            n = 104019611
        D = q.make_shifts(600 + i, M, d)
        Dd = torch.from_numpy(D.astype(np.int64)).to(dev)
        r = q.rule(n, tab.z_for(n)[:d], Dd, ("korobov", 3))
        f = q.Integrand.polynomial(fl)
        entries.append((f.device_struct(dev), r, 0, n))
        keep.append((fl, D, Dd, f))
    b = q.Batch(entries)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev)
    bsums = torch.zeros(len(entries), 4 * M, dtype=torch.float64, device=dev)
    b.sums(ws, bsums)
    torch.cuda.synchronize()
    got = bsums.cpu().numpy()
    for i, (fd, r, _, n) in enumerate(entries):
        wsi = torch.empty(q.sums_workspace_bytes(r, False, 0, n), dtype=torch.uint8, device=dev)
        one = torch.zeros(4 * M, dtype=torch.float64, device=dev)
        q.sums(fd, r, 0, n, wsi, one)
        torch.cuda.synchronize()
        assert np.array_equal(got[i, : 2 * M], one.cpu().numpy()[: 2 * M]), i
        if i == 0:
            tiles, ppt = q.sums_tile_count(n, M)
            part = wsi[: tiles * M * 16].view(torch.float64).cpu().numpy().reshape(tiles, M, 2)
            t = tiles // 2
            fl, D = keep[0][0], keep[0][1]
            o = O.shift_sums(O.from_feynman(fl), ("korobov", 3), n, tab.z_for(n)[:fl.d], D,
                             i0=t * ppt, i1=min(t * ppt + ppt, n))
            worst = _check_sums(part[t, :, 0] + part[t, :, 1], o["re"][:, 0] + o["re"][:, 1],
                                o["abs"], ("sector", t))
            print(f"[parity] sector tile n={n}: max |dS|/A = {worst:.2e}")
