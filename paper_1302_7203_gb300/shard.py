"""Host-side work division across ranks (one process per GPU).

Eigenpairs are independent (Sec. 1: each is computed from the shifted
inverse of its own nearest pole), so the work shards with no collective on
the data path:

* independent instances (the benchmark's weak scaling: one instance per rank,
  seeded by rank) -- `rank_seed`;
* a batch of instances of uneven orders: greedy bin-packing on n^2, the
  per-instance work (each of n eigenpairs is an O(n) computation) --
  `pack_instances`;
* one instance split by eigenpair ranges (arrow_eig_part in the library):
  every rank repeats the O(n log n) reduction, solves an even share of the
  computed eigenpairs plus the deflated rows whose values fall in its range,
  and owns a contiguous block of output positions -- `part_bounds`,
  `part_items` give the same index arithmetic on the host, `merge_parts`
  puts the blocks side by side.  The remedy test of Eq. (K0) needs the
  eigenvalue on each side of a range; each rank recomputes those two rather
  than receiving them, so nothing is exchanged before the results.

Collectives appear only around the data path: a barrier and the max of the
ranks' times for the measurement (`max_over_ranks`), an optional gather of
results to rank 0 (`gather_to_root`), and a heartbeat between steps through a
key-value store (`arrive`, `missing_ranks`) so that the ranks learn on the
host that one of them has left, before their next launch.  Everything here is
plain Python on host data; torch.distributed is used only through the
process group or store passed in.
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


def part_bounds(ncomp: int, part: int, nparts: int):
    """Computed-eigenpair range [k0, k1) of part `part` of `nparts`: an even
    split of the ncomp = m + 1 eigenvalues of the reduced arrowhead (the
    library's arrow_eig_part uses the same integer arithmetic)."""
    if nparts < 1 or not 0 <= part < nparts:
        raise ValueError("need 0 <= part < nparts")
    return part * ncomp // nparts, (part + 1) * ncomp // nparts


def part_items(poles, deflated, part: int, nparts: int):
    """(k0, k1, u0, u1, pos0, count) of one part of a split instance.

    `poles`: the reduced poles, decreasing (m of them, m + 1 computed
    eigenvalues); `deflated`: the deflated rows' values in sorted
    (non-increasing) order.  The part owns the computed eigenpairs [k0, k1)
    and the deflated rows [u0, u1) whose values lie in [p_{k1-1}, p_{k0-1});
    together they fill the output positions [pos0, pos0 + count)."""
    poles = np.asarray(poles, dtype=np.float64)
    deflated = np.asarray(deflated, dtype=np.float64)
    ncomp, nd = poles.size + 1, deflated.size

    def at_least(x):                         # entries >= x of a non-increasing array
        return int(np.searchsorted(-deflated, -x, side="right"))

    k0, k1 = part_bounds(ncomp, part, nparts)
    u0 = 0 if k0 == 0 else at_least(poles[k0 - 1])
    u1 = nd if k1 == ncomp else (0 if k1 == 0 else at_least(poles[k1 - 1]))
    u1 = max(u1, u0)
    return k0, k1, u0, u1, k0 + u0, (k1 - k0) + (u1 - u0)


def merge_parts(n: int, blocks):
    """The whole decomposition from its parts' blocks: `blocks` holds
    (pos0, lam, V) per part (V n x count, or None).  Raises when the blocks
    do not cover the n output positions exactly once."""
    lam = np.empty(n)
    V = None if any(b[2] is None for b in blocks) else np.empty((n, n))
    seen = np.zeros(n, dtype=np.int64)
    for pos0, l, v in blocks:
        c = len(l)
        seen[pos0:pos0 + c] += 1
        lam[pos0:pos0 + c] = l
        if V is not None:
            V[:, pos0:pos0 + c] = v
    if not np.all(seen == 1):
        raise ValueError("the parts do not cover every output position once")
    return lam, V


def arrive(store, step: int, rank: int) -> None:
    """Heartbeat: rank `rank` has finished step `step` and will take the next."""
    store.set(f"ae/step{step}/rank{rank}", "1")


def missing_ranks(store, step: int, world: int, timeout_s: float = 5.0):
    """Ranks that have not arrived at `step` within `timeout_s` (an empty list
    when all have).  Checked on the host between steps, before any launch of
    the next one, so a rank that left is reported instead of a collective
    waiting for it."""
    import time
    keys = [f"ae/step{step}/rank{r}" for r in range(world)]
    deadline = time.monotonic() + timeout_s
    while True:
        gone = [r for r, k in enumerate(keys) if not store.check([k])]
        if not gone or time.monotonic() >= deadline:
            return gone
        time.sleep(0.01)


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
