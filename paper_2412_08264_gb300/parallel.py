"""Data parallelism over training pairs (eq. (5.2)): the only exchange is the hypergradient mean.

Each rank holds whole pairs (their lower solves, Hessian solves and recycle spaces never move); the
upper loss and its hypergradient are means over all pairs, so ranks combine their local means
weighted by their pair counts with one all-reduce per outer step.
"""
from __future__ import annotations

from typing import List, Sequence

import torch


def shard_pairs(pixels: Sequence[int], world: int) -> List[List[int]]:
    """Split pair indices over `world` ranks, balancing pixel counts (largest first, greedy)."""
    order = sorted(range(len(pixels)), key=lambda k: (-pixels[k], k))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        out[r].append(k)
        load[r] += pixels[k]
    return [sorted(o) for o in out]


def allreduce_mean(local_mean: torch.Tensor, local_count: int, group=None) -> torch.Tensor:
    """Global mean over all pairs from per-rank means of `local_count` pairs (one all-reduce)."""
    import torch.distributed as dist
    buf = torch.cat([local_mean.reshape(-1) * local_count,
                     torch.tensor([float(local_count)], dtype=local_mean.dtype, device=local_mean.device)])
    dist.all_reduce(buf, group=group)
    return (buf[:-1] / buf[-1]).reshape(local_mean.shape)
