"""Host-side work division across ranks (one process per GPU).

Eigenpairs are independent (Sec. 1: each is computed from the shifted
inverse of its own nearest pole), so the work shards with no collective on
the data path:

* independent instances (the benchmark's weak scaling: one instance per rank,
  seeded by rank) -- `rank_seed`;
* a batch of instances of uneven orders: greedy bin-packing on n^2, the
  per-instance work (each of n eigenpairs is an O(n) computation) --
  `pack_instances`.

(One instance is not split across GPUs: at the orders this library serves
one GPU holds it whole, and a split by eigenpair ranges would need, besides a
one-eigenpair halo for the remedy test of Eq. K0, every rank's eigenvalues to
place the deflated rows.)

Collectives appear only around the data path: a barrier and the max of the
ranks' times for the measurement (`max_over_ranks`), and an optional gather
of results to rank 0 (`gather_to_root`).  Everything here is plain Python on
host data; torch.distributed is used only through the process group passed in.
"""
from __future__ import annotations

import heapq

import numpy as np


def rank_seed(base: int, rank: int) -> int:
    """Seed of the instance rank `rank` solves in a weak-scaling run."""
    return base + rank


def pack_instances(orders, world: int):
    """Assign instances (orders n_i) to `world` ranks, balancing sum n_i^2.

    Greedy longest-processing-time: instances in decreasing n^2, each to the
    currently lightest rank (ties to the lower rank).  Returns a list of index
    lists, each in increasing instance order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    orders = np.asarray(orders, dtype=np.int64)
    cost = orders * orders
    order = sorted(range(len(orders)), key=lambda i: (-int(cost[i]), i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(cost[i]), r))
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The largest `value` over the ranks of `group` (a plain float on one rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_to_root(array, group=None):
    """Rank 0 receives every rank's host array (in rank order); others get None."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return [array]
    world = dist.get_world_size(group)
    out = [None] * world if dist.get_rank(group) == 0 else None
    dist.gather_object(array, out, dst=0, group=group)
    return out
