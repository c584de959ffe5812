"""Replica (N > 1) host logic of bench.py on CPU: two gloo ranks, no GPU."""
import os
import socket

import torch.multiprocessing as mp


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
    import bench
    t, m = bench.aggregate_over_ranks(1.5 + rank, 1000 * (rank + 1))
    q.put((rank, t, m, bench.replica_seed(1, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_max_time_sum_messages():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, m, seed in got:
        assert t == 2.5          # the slowest rank's time
        assert m == 3000.0       # all ranks' messages
    assert got[0][3] != got[1][3]   # each rank replays its own episode


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_over_ranks(2.0, 7) == (2.0, 7)
