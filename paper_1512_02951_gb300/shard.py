"""Partition of independent images across ranks (one process per GPU).

Every image (and, inside an image, every 8x8 block and every 16-byte CTR keystream block) is
processed independently: the method has no exchange step (Sect. 6.5: data parallelism over
blocks and images).  Multi-GPU work is therefore a partition of the request list, with no
collective on the data path; the only cross-rank operation is taking the slowest rank's time.
"""
from __future__ import annotations

from typing import Sequence


def shard(costs: Sequence[int], world: int) -> list[list[int]]:
    """Split item indices into `world` lists of near-equal total cost (largest first, each
    to the currently lightest rank).  Deterministic: ties go to the lower rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(i)
        load[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value: float) -> float:
    """The largest `value` over all ranks of the default process group (identity when no
    group is initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
