"""The multi-rank path of bench.py, on CPU ranks (gloo): the whole-job time is
the slowest rank's, the counted units are summed over the ranks, and the
particles of a batch are dealt to the ranks with none missing or repeated.
(The library path itself does not shard: one process per GPU runs an
independent replica.)"""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, counts = bench.reduce_over_ranks(1.0 + 0.5 * rank, [10 * (rank + 1), rank, 3], "cpu")
        mine = bench.deal(list(range(11)), rank, world)
        dist.barrier()
        q.put((rank, t, counts, mine))
    finally:
        dist.destroy_process_group()


def test_single_process_values_pass_through():
    import bench
    assert bench.reduce_over_ranks(2.5, [7, 1], "cpu") == (2.5, [7, 1])
    assert bench.deal(list(range(5)), 0, 1) == list(range(5))


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_take_max_time_and_sum_counts(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    t_max = 1.0 + 0.5 * (world - 1)
    total = [sum(10 * (r + 1) for r in range(world)), sum(range(world)), 3 * world]
    dealt = []
    for rank, t, counts, mine in res:
        assert t == t_max
        assert counts == total
        dealt += mine
    assert sorted(dealt) == list(range(11))
