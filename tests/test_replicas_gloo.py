"""The N > 1 path on CPU: two gloo ranks, max over ranks and instance shards."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2208_01339_gb300 import replicas as R  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = R.rank_env()
    R.barrier()
    m = R.max_over_ranks(10.0 + rank)
    items = list(R.shard(7, r, w))
    weights = [5.0, 1.0, 3.0, 3.0, 8.0, 2.0, 1.0]
    q.put((rank, m, items, R.shard_balanced(weights, r, w)))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(m == 11.0 for _, m, _, _ in out)
    assert out[0][2] + out[1][2] == list(range(7))
    # the balanced shards partition the items, and each rank computed the same split
    assert sorted(out[0][3] + out[1][3]) == list(range(7))
    assert out[0][3] == R.shard_balanced([5.0, 1.0, 3.0, 3.0, 8.0, 2.0, 1.0], 0, 2)


def test_shard_partitions():
    for n in (0, 1, 5, 64):
        for w in (1, 2, 3, 8):
            got = [i for r in range(w) for i in R.shard(n, r, w)]
            assert got == list(range(n))
    assert R.max_over_ranks(3.5) == 3.5


def test_shard_balanced_partitions_and_balances():
    import random

    rng = random.Random(3)
    for n in (0, 1, 5, 64):
        w = [rng.uniform(1, 100) for _ in range(n)]
        for world in (1, 2, 3, 8):
            parts = [R.shard_balanced(w, r, world) for r in range(world)]
            assert sorted(i for p in parts for i in p) == list(range(n))
            if n >= world:
                loads = [sum(w[i] for i in p) for p in parts]
                # greedy largest-first: no rank exceeds the mean by more than the largest item
                assert max(loads) <= sum(w) / world + max(w) + 1e-9
