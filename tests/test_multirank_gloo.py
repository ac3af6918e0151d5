"""Multi-rank paths on CPU with gloo (world size 2): sharding one integral by i-range and
merging per-shift sums, and the benchmark's replica layout (independent integrals per
rank, MAX of the timings).  The per-rank sums come from the CPU oracle; the sharding and
merge logic under test is the package's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as O
    import workloads as W
    from paper_1811_11720_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tab = O.load_genvec_table(os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt"))
    n, d, m = 108863, 5, 8
    c, w = W.genz_params(4, d, 3)
    D = O.shifts(42, m, d)
    a, b = shard.shard_range(n, rank, world)
    r = O.shift_sums(O.genz(4, c, w), ("korobov", 3), n, tab[n], D, i0=a, i1=b, nthreads=1)
    local = torch.from_numpy(np.ascontiguousarray(r["re"].reshape(-1)))
    merged = shard.gather_merge(local)
    # replica layout of the benchmark: MAX over ranks of a per-rank time
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"merged{rank}.npy"), merged)
    np.save(os.path.join(out_dir, f"tmax{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_exactly():
    from paper_1811_11720_gb300 import shard
    for n in (1, 7, 108863, 10 ** 9 + 7):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_merge_is_compensated():
    from paper_1811_11720_gb300 import shard
    parts = [np.array([1e16, 0.0]), np.array([1.0, 0.0]), np.array([-1e16, 0.0])]
    out = shard.merge_sums(parts)
    assert out[0] + out[1] == 1.0


def test_two_rank_shard_and_merge_matches_whole(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_shard_worker, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    import oracle as O
    import workloads as W
    tab = O.load_genvec_table(os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt"))
    n, d, m = 108863, 5, 8
    c, w = W.genz_params(4, d, 3)
    D = O.shifts(42, m, d)
    whole = O.shift_sums(O.genz(4, c, w), ("korobov", 3), n, tab[n], D)
    S_whole = whole["re"][:, 0] + whole["re"][:, 1]
    for rank in range(world):
        merged = np.load(tmp_path / f"merged{rank}.npy")
        S = merged[0::2] + merged[1::2]
        assert np.allclose(S, S_whole, rtol=1e-15, atol=0)
        assert np.load(tmp_path / f"tmax{rank}.npy")[0] == world


def test_bench_replicas_draw_independent_integrals():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a = bench.workload_items(0)
    b = bench.workload_items(1)
    assert len(a) == len(b) == 45
    assert not any(np.array_equal(x[3], y[3]) for x, y in zip(a, b))
    assert bench.workload_items(0, "4:10:korobov3")[0][:3] == (4, 10, ("korobov", 3))


def _tiles_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    from paper_1811_11720_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tiles, m = 11, 3
    counts = [shard.shard_tiles(tiles, r, world)[1] - shard.shard_tiles(tiles, r, world)[0]
              for r in range(world)]
    a, b = shard.shard_tiles(tiles, rank, world)
    # synthetic partials: value = tile * 1000 + slot, re block then im block
    re = np.array([t * 1000.0 + s for t in range(a, b) for s in range(2 * m)])
    im = -re
    local = torch.from_numpy(np.concatenate([re, im]))
    out = shard.gather_tile_partials(local, counts, m, True)
    np.save(os.path.join(out_dir, f"tiles{rank}.npy"), out)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_tile_partials_assemble_in_tile_order(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_tiles_worker, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    m, tiles = 3, 11
    re = np.array([t * 1000.0 + s for t in range(tiles) for s in range(2 * m)])
    want = np.concatenate([re, -re])
    for rank in range(world):
        assert np.array_equal(np.load(tmp_path / f"tiles{rank}.npy"), want)


def test_shard_tiles_cover_exactly():
    from paper_1811_11720_gb300 import shard
    for tiles in (1, 5, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_tiles(tiles, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == tiles
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
