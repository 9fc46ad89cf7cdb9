"""Splitting independent AES work across ranks (one process per GPU).

Blocks and messages are independent (each block is its own one-block CBC message), so the work
shards with no data-path collective: contiguous block ranges (strong scaling) or one batch per
rank (weak scaling).  The only collective is the reduction of timings for reporting.
"""
from __future__ import annotations


def block_range(nblocks: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) share of nblocks for `rank`; shares differ by at most one block."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return nblocks * rank // world, nblocks * (rank + 1) // world


def message_ranges(lengths, world: int) -> list[tuple[int, int]]:
    """Whole messages per rank, cut so that every rank gets about the same number of bytes
    (a message is never split).  Returns [first, last) message indices per rank."""
    total = int(sum(int(x) for x in lengths))
    cuts, acc, r = [0], 0, 1
    for i, x in enumerate(lengths):
        acc += int(x)
        while r < world and acc >= total * r / world:
            cuts.append(i + 1)
            r += 1
    while len(cuts) < world:
        cuts.append(len(lengths))
    cuts.append(len(lengths))
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def weak_scaling_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's own batch in a weak-scaling run (rank 0 keeps the base workload)."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
