"""Multi-rank timing aggregation of bench.py on CPU (gloo, world size 2): every rank solves its own
request, the job time is the max over ranks and the throughput counts all ranks' solves."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 1000.0 * (rank + 1)            # rank 1 is the slowest
        t = bench.max_over_ranks(my_ms, world)
        bench.barrier(world)
        out[rank] = (t, bench.aggregate(t, 3, world))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        t, v = out[r]
        assert t == 2000.0                      # max over ranks
        assert v == pytest.approx(world * 3 / 2.0)  # all ranks' solves over the slowest time
