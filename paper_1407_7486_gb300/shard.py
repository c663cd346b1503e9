"""Sharding the loop ensemble across ranks by jackknife group.

One process per GPU.  Rank r of W holds the loops of groups
[r G/W, (r+1) G/W), i.e. the global loops [r N_l/W, (r+1) N_l/W).  Loops
are counter-based (the Philox counter word is the global loop index), so a
rank generates exactly its own loops with `gen_loops(..., loop0=...)`, and
its group sums are the sums the same groups would have in one process.
Groups are disjoint, so the only exchange is a concatenation of per-group
sums (an all-gather, no reduction); the jackknife and the quadrature then
run on the gathered sums.  The data path has no collective.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Shard:
    loop0: int          # first global loop of this rank
    n_loops: int        # loops held by this rank
    group0: int         # first global group of this rank
    n_groups: int       # groups held by this rank


def shard(n_loops: int, n_groups: int, world: int, rank: int) -> Shard:
    if n_groups % world or n_loops % n_groups:
        raise ValueError("groups must divide evenly over ranks and loops over groups")
    g = n_groups // world
    lpg = n_loops // n_groups
    return Shard(loop0=rank * g * lpg, n_loops=g * lpg, group0=rank * g, n_groups=g)


def gather_group_sums(local, world: int, group=None):
    """All-gather per-rank group sums [n_points][G/W][K] into [n_points][G][K]
    (group order = rank order).  `local` is a torch tensor on the rank's
    device (CPU for gloo, CUDA for nccl)."""
    import torch
    import torch.distributed as dist
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    return torch.cat(parts, dim=1)
