"""Host logic for runs with one process per GPU (torchrun).

The single-domain step does not shard (one box per GPU; a slab decomposition
is not built), so several GPUs run independent replicas.  The batched
parameter sweep does shard: its domains are independent, so each rank takes a
share of them and no data crosses ranks.  This module holds the rank-side
plumbing both need; it works with any torch.distributed backend (NCCL on the
GPUs, gloo on CPU in the tests).
"""
from __future__ import annotations

import os


class Ranks:
    """world/rank from the torchrun environment, with a barrier and a
    max-over-ranks reduction of host scalars (timings)."""

    def __init__(self, device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device  # torch device the reductions use ("cuda" for NCCL, "cpu" for gloo)

    @property
    def distributed(self):
        return self.world > 1

    def barrier(self):
        if self.distributed:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(self, x):
        if not self.distributed:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(self, x):
        if not self.distributed:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())


def partition_domains(cells, world):
    """Split domains (given by their node counts) into `world` shares of
    near-equal total nodes: largest first, each to the currently lightest
    share (ties to the lower rank).  Deterministic; every domain lands in
    exactly one share; each share lists its domains in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    shares = [[] for _ in range(world)]
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        shares[r].append(i)
        loads[r] += int(cells[i])
    return [sorted(s) for s in shares]
