"""Multi-rank host logic on CPU: world_size 2 over gloo (no GPU).

The data path shards with no collective: a batch of instances is bin-packed
on n^2 across ranks, every rank solves its own instances, and only the
measurement (max of the ranks' times) and an optional gather to rank 0 use the
process group.  Here each rank solves its share with the CPU oracle; the
gathered results must equal solving the whole batch in one process, bit for
bit, and the packing must cover every instance once and balance the work.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

from paper_1302_7203_gb300 import shard, workloads as W   # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_pack_instances_covers_and_balances():
    orders = W.batch_sizes(500, lo=32, hi=4096, seed=2)
    for world in (1, 2, 3, 8):
        parts = shard.pack_instances(orders, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(orders)))
        loads = [int(sum(int(orders[i]) ** 2 for i in p)) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest item
        assert max(loads) - sum(loads) / world <= max(int(o) ** 2 for o in orders)
    with pytest.raises(ValueError):
        shard.pack_instances(orders, 0)


def test_rank_seed_distinct():
    assert len({shard.rank_seed(1, r) for r in range(8)}) == 8


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        sizes = W.batch_sizes(12, lo=4, hi=120, seed=7)
        inst = [W.uniform_arrow(int(n), seed=700 + i) for i, n in enumerate(sizes)]
        mine = shard.pack_instances(sizes, world)[rank]
        res = {i: oracle.arrow_eig(*inst[i], nthreads=1) for i in mine}
        lam = {i: r["lam"] for i, r in res.items()}
        V = {i: r["V"] for i, r in res.items()}
        t = shard.max_over_ranks(float(rank + 1))
        got = shard.gather_to_root((lam, V))
        if rank == 0:
            merged_l, merged_v = {}, {}
            for l, v in got:
                merged_l.update(l)
                merged_v.update(v)
            np.savez(out_path, t=t, keys=np.array(sorted(merged_l)),
                     **{f"l{i}": merged_l[i] for i in merged_l},
                     **{f"v{i}": merged_v[i] for i in merged_v})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_a_packed_batch(tmp_path):
    import oracle
    oracle.threads()                         # build the oracle before the workers start
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    data = np.load(out)
    assert float(data["t"]) == 2.0           # the max over ranks
    sizes = W.batch_sizes(12, lo=4, hi=120, seed=7)
    assert list(data["keys"]) == list(range(len(sizes)))
    for i, n in enumerate(sizes):
        d, z, a = W.uniform_arrow(int(n), seed=700 + i)
        ref = oracle.arrow_eig(d, z, a, nthreads=1)
        np.testing.assert_array_equal(data[f"l{i}"], ref["lam"])
        np.testing.assert_array_equal(data[f"v{i}"], ref["V"])


# ----------------------------------------------------------------------------
# one instance split by eigenpair ranges
# ----------------------------------------------------------------------------
def _reduced(d, z):
    """Reduced poles and deflated values (sorted order) from the oracle's reduction."""
    import oracle
    order, kind, head, m = oracle.reduce(d, z)
    poles = np.array([d[r] for r in order if kind[r] == 0])
    defl = np.array([d[r] for r in order if kind[r] != 0])
    assert poles.size == m
    return poles, defl


def _deflating_instance(n=61, seed=3):
    d, z, a = W.uniform_arrow(n, seed=seed)
    d = d.copy()
    z = z.copy()
    z[[4, 20, 21]] = 0.0                   # zero spikes
    d[[9, 10]] = d[8]                      # a run of three equal poles
    d[[30, 31]] = d[29]
    z[31] = 0.0                            # a zero spike inside a run
    return d, z, a


@pytest.mark.parametrize("nparts", [1, 2, 3, 5, 8])
def test_part_items_cover_the_output_in_order(nparts):
    import oracle
    for d, z, a in (_deflating_instance(), W.uniform_arrow(40, seed=1)):
        n = len(d) + 1
        poles, defl = _reduced(d, z)
        ref = oracle.arrow_eig(d, z, a, vectors=False)["lam"]
        nxt = 0
        for p in range(nparts):
            k0, k1, u0, u1, pos0, cnt = shard.part_items(poles, defl, p, nparts)
            assert pos0 == nxt                 # contiguous, in part order
            nxt += cnt
            hi = np.inf if k0 == 0 else poles[k0 - 1]
            lo = -np.inf if k1 == poles.size + 1 else (np.inf if k1 == 0 else poles[k1 - 1])
            block = ref[pos0:pos0 + cnt]
            # the part's items are exactly the values in [p_{k1-1}, p_{k0-1})
            assert np.all(block < hi) and np.all(block >= lo)
            assert cnt == (k1 - k0) + (u1 - u0)
        assert nxt == n
    with pytest.raises(ValueError):
        shard.part_bounds(10, 2, 2)


def _split_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        out = {}
        # (1) an instance with deflation: each rank solves its block with the
        # oracle; rank 0 merges the blocks
        d, z, a = _deflating_instance()
        n = len(d) + 1
        poles, defl = _reduced(d, z)
        _, _, _, _, pos0, cnt = shard.part_items(poles, defl, rank, world)
        ks = np.arange(pos0, pos0 + cnt)
        r = oracle.arrow_eig(d, z, a, ks=ks, nthreads=1) if cnt else {"lam": np.zeros(0),
                                                                       "V": np.zeros((n, 0))}
        got = shard.gather_to_root((pos0, r["lam"], r["V"]))
        if rank == 0:
            out["lam"], out["V"] = shard.merge_parts(n, got)
        # (2) the one-eigenpair halo on an instance without deflation: each rank
        # recomputes the eigenvalue just outside each end of its range; the
        # edge values every rank owns are gathered and must match bit for bit
        d2, z2, a2 = W.graded_arrow(97, seed=5)
        n2 = len(d2) + 1
        k0, k1 = shard.part_bounds(n2, rank, world)
        halo = [k for k in (k0 - 1, k1) if 0 <= k < n2]
        mine = oracle.arrow_eig(d2, z2, a2, ks=np.arange(k0, k1), vectors=False, nthreads=1)
        hal = oracle.arrow_eig(d2, z2, a2, ks=np.array(halo), vectors=False, nthreads=1)
        edges = shard.gather_to_root(({k0: mine["lam"][0], k1 - 1: mine["lam"][-1]},
                                      dict(zip(halo, hal["lam"]))))
        if rank == 0:
            owned = {}
            for e, _ in edges:
                owned.update(e)
            out["halo_ok"] = all(owned[k] == v for _, h in edges for k, v in h.items())
            out["halo_count"] = sum(len(h) for _, h in edges)
            np.savez(out_path, **out)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_instance_merges_to_the_whole(tmp_path, world):
    import oracle
    oracle.threads()
    path = str(tmp_path / "split.npz")
    mp.start_processes(_split_worker, args=(world, _free_port(), path), nprocs=world,
                       join=True, start_method="spawn")
    data = np.load(path)
    d, z, a = _deflating_instance()
    ref = oracle.arrow_eig(d, z, a, nthreads=1)
    np.testing.assert_array_equal(data["lam"], ref["lam"])
    np.testing.assert_array_equal(data["V"], ref["V"])
    assert bool(data["halo_ok"]) and int(data["halo_count"]) == 2 * (world - 1)


def _leaving_worker(rank, world, port, out_path):
    from datetime import timedelta
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timedelta(seconds=30))
    import oracle
    d, z, a = W.uniform_arrow(30, seed=rank)
    oracle.arrow_eig(d, z, a, nthreads=1)            # step 0
    shard.arrive(store, 0, rank)
    if rank == world - 1:
        return                                       # leaves between steps
    missing0 = shard.missing_ranks(store, 0, world, timeout_s=10.0)
    shard.arrive(store, 1, rank)                     # done with step 1's host part
    missing1 = shard.missing_ranks(store, 1, world, timeout_s=1.0)
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(f"{missing0} {missing1}")
    store.set(f"done/{rank}", "1")
    if rank == 0:                                    # keep the store up for the others
        store.wait([f"done/{r}" for r in range(world - 1)])


def test_a_rank_that_leaves_between_steps_is_reported(tmp_path):
    import oracle
    oracle.threads()
    path = str(tmp_path / "gone")
    world = 3
    mp.start_processes(_leaving_worker, args=(world, _free_port(), path), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world - 1):
        with open(f"{path}.{r}") as f:
            assert f.read() == "[] [2]"
