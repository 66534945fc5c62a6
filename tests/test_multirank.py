"""The multi-GPU path is replicas: each rank takes its own pairs and the
whole-job value is all pixels over the slowest rank's time.  Its host logic
runs here as two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    first, count = bench.rank_shard(rank, 4)
    my_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    dist.barrier()
    max_ms = bench.max_over_ranks(my_ms, world, dist)
    value = bench.whole_job_mpix_s(1_000_000, 2, world, max_ms)
    out[rank] = (first, count, max_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    assert (r0[0], r0[1]) == (0, 4) and (r1[0], r1[1]) == (4, 4)  # disjoint shards
    assert r0[2] == r1[2] == 200.0                                  # max over ranks
    assert r0[3] == pytest.approx(2 * 1e6 * 2 / 0.2 / 1e6)          # all pixels / slowest time
