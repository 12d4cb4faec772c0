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
