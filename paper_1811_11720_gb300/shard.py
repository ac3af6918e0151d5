"""Sharding one lattice rule over ranks and merging the per-shift sums.

Points i of a rank-1 lattice and shifts k are independent (Eq. (lattice)), so one
integral splits into contiguous i-ranges; each rank runs ``qmc_sums`` on its range and the
per-shift double-double sums add.  The merge is the single exchange step: an all-gather of
2m (real) or 4m (complex) doubles per rank, summed in rank order with TwoSum so that the
result does not depend on arrival order, then ``qmc_finalize`` on the merged sums.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous balanced split of [0, n): rank r gets [r n / W, (r+1) n / W)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return (n * rank) // world, (n * (rank + 1)) // world


def _two_sum(a, b):
    s = a + b
    bp = s - a
    e = (a - (s - bp)) + (b - bp)
    return s, e


def merge_sums(parts) -> np.ndarray:
    """Sum per-shard double-double arrays laid out as (hi, lo) pairs in fixed (list) order.
    Each part is a float64 array of even length; returns the same layout."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    if not parts:
        raise ValueError("nothing to merge")
    hi = parts[0][0::2].copy()
    lo = parts[0][1::2].copy()
    for p in parts[1:]:
        s, e = _two_sum(hi, p[0::2])
        e = e + lo + p[1::2]
        hi = s + e
        lo = e - (hi - s)
    out = np.empty_like(parts[0])
    out[0::2] = hi
    out[1::2] = lo
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
