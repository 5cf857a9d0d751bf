"""Source-parallel gradient across ranks (one process per GPU).

Sources are independent (the paper parallelises its inversion over sources):
each rank models a contiguous share of the source batch on the full model, and
the per-rank gradients and misfits are summed by one all-reduce per gradient --
the only exchange the method has.  Rank count and placement come from the
standard torch.distributed environment (RANK, WORLD_SIZE, MASTER_ADDR, ...).
"""
from __future__ import annotations

import numpy as np


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of n_items for this rank (shares differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def towline(points, n: int, spacing: float = 250.0):
    """n sources along x, `spacing` apart, centred on the first point of `points`."""
    from .workloads import Points
    x0, y0, z0, c0 = points.x[0], points.y[0], points.z[0], int(points.comp[0])
    xs = x0 + spacing * (np.arange(n) - n // 2)
    return Points.make([[x, y0, z0] for x in xs], c0)


def rank_sources(points, rank: int, world: int):
    """The sources one rank models under weak scaling: a towline of world x points.n sources
    (`towline`, centred on the first point) split into contiguous shares (`shard`).  With one
    rank the points are returned as they are."""
    if world <= 1:
        return points
    line = towline(points, world * points.n)
    return line.subset(list(shard(line.n, rank, world)))


def sum_over_ranks(*tensors):
    """In-place sum of each tensor over all ranks (no-op without a process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        for t in tensors:
            dist.all_reduce(t)
    return tensors


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([value], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(value)
