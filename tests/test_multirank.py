"""The N > 1 path of bench.py on CPU: two gloo ranks, each its own disorder
realisation (independent replicas, no data-path collective), the job time
is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank)              # rank 1 is slower
    out[rank] = (t, bench.replica_seed(1, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_replica_seeds():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] != out[1][1]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
