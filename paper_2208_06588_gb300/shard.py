"""Sharding of a batch over ranks (one process per GPU), host logic only.

Instances are independent, so a batch splits into contiguous instance ranges, one per rank,
balanced by cell count (the work of a step is proportional to the cells); there is no exchange
on the data path. The only collectives are for timing: a barrier and the max over ranks.
"""
from __future__ import annotations

import numpy as np


def partition(off, world: int, rank: int):
    """Instance range [i0, i1) of ``rank`` among ``world`` ranks for cell offsets ``off`` (B+1):
    the cut before instance i goes to the rank whose share of the total cells contains the
    instance's first cell, so every rank gets a contiguous run and the cell counts differ by at
    most one instance's size. Ranks may get an empty range when B < world."""
    off = np.asarray(off, dtype=np.int64)
    B = off.size - 1
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    total = int(off[-1])
    # Rank r owns the instances whose first cell lies in [r*total/world, (r+1)*total/world).
    bounds = [(r * total) // world for r in range(world + 1)]
    starts = off[:-1]
    i0 = int(np.searchsorted(starts, bounds[rank], side="left")) if rank > 0 else 0
    i1 = int(np.searchsorted(starts, bounds[rank + 1], side="left")) if rank + 1 < world else B
    return i0, max(i0, i1)


def subset(batch, i0: int, i1: int):
    """The instances [i0, i1) of a workloads.Batch as a Batch of their own (offsets rebased)."""
    from .workloads import Batch
    off = batch.off
    a, c = int(off[i0]), int(off[i1])
    return Batch(name=f"{batch.name}[{i0}:{i1}]", off=(off[i0:i1 + 1] - a).astype(np.int64),
                 x=batch.x[a + i0:c + i1], h=batch.h[a:c], hu=batch.hu[a:c], b=batch.b[a:c], E=batch.E[a:c],
                 profile=batch.profile[a + i0:c + i1], cfl=batch.cfl[i0:i1], bc=batch.bc, mesh=batch.mesh,
                 mesh_T=batch.mesh_T, g=batch.g, eps_weno=batch.eps_weno)


def barrier():
    """dist.barrier() when a process group with more than one rank is up."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over the ranks of the default process group (the value itself without
    one). ``device``: where the reduction tensor lives (a CUDA device for NCCL, None for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
