"""Sharding one lattice rule over ranks and merging the per-shift sums.

Points i of a rank-1 lattice and shifts k are independent (Eq. (lattice)), so one
integral splits into contiguous pieces and the only exchange step is a gather.  Two forms:

* tile-aligned (bit-identical to one device): the ranks split the tiles of qmc_sums'
  decomposition (shard_tiles), each computes its tiles' partials (qmc_sums_tiles), the
  partials are gathered in rank order (gather_tile_partials, 2m doubles per tile) and folded
  by qmc_reduce_tiles exactly as qmc_sums folds them;
* i-range (shard_range, merge_sums): each rank runs qmc_sums on its own range and the
  per-shift double-double sums (2m or 4m doubles per rank) are added in rank order by the
  library (qmc_merge_sums); equal to the whole within rounding, independent of arrival
  order.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous balanced split of [0, n): rank r gets [r n / W, (r+1) n / W)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return (n * rank) // world, (n * (rank + 1)) // world


def shard_tiles(tiles: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous balanced split of the tiles [0, tiles) of one rule's decomposition
    (qmc_sums_tile_count): rank r gets [r T / W, (r+1) T / W).  Shards cut at tile
    boundaries reproduce qmc_sums bit for bit once their partials are folded in order."""
    return shard_range(tiles, rank, world)


def assemble_tile_partials(parts, m: int, is_complex: bool) -> np.ndarray:
    """Concatenate per-shard tile partials (each laid out as qmc_sums_tiles writes them:
    T_r x m (sum, comp) pairs for the real part, then the same for the imaginary part) in
    shard order into the layout of the whole tile range."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    blk = 2 * m
    re, im = [], []
    for p in parts:
        per = p.size // (2 if is_complex else 1)
        if per % blk:
            raise ValueError("partials size is not a multiple of 2 m")
        re.append(p[:per])
        if is_complex:
            im.append(p[per:])
    return np.concatenate(re + im)


def gather_tile_partials(local, tiles_per_rank, m: int, is_complex: bool, group=None) -> np.ndarray:
    """All-gather every rank's tile partials (torch tensor, CPU or CUDA; rank r holds
    tiles_per_rank[r] tiles) and assemble them in rank order (assemble_tile_partials)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    per = 2 * m * (2 if is_complex else 1)
    mx = max(tiles_per_rank) * per
    buf = torch.zeros(mx, dtype=torch.float64, device=local.device)
    buf[: local.numel()] = local.reshape(-1)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    parts = [b[: tiles_per_rank[r] * per].detach().cpu().numpy() for r, b in enumerate(bufs)]
    return assemble_tile_partials(parts, m, is_complex)


def merge_sums(parts) -> np.ndarray:
    """Sum per-shard double-double arrays laid out as (hi, lo) pairs in fixed (list) order
    (qmc_merge_sums).  Each part is a float64 array of the same even length; returns the
    same layout."""
    from . import _check, lib
    parts = [np.ascontiguousarray(np.asarray(p, dtype=np.float64)).reshape(-1) for p in parts]
    if not parts:
        raise ValueError("nothing to merge")
    if any(p.size != parts[0].size for p in parts):
        raise ValueError("parts differ in length")
    stacked = np.ascontiguousarray(np.stack(parts))
    out = np.empty(parts[0].size)
    _check(lib().qmc_merge_sums(stacked.ctypes.data, len(parts), int(parts[0].size),
                                out.ctypes.data), "merge_sums")
    return out


def gather_merge(local_sums, group=None) -> np.ndarray:
    """All-gather every rank's sums (a torch tensor, CPU or CUDA) and merge them in rank
    order.  Every rank receives the merged array."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(local_sums) for _ in range(world)]
    dist.all_gather(bufs, local_sums, group=group)
    return merge_sums([b.detach().cpu().numpy() for b in bufs])
