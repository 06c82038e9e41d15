"""The multi-GPU path of bench.py runs one independent replica per rank (the
solve does not shard across GPUs here): the job time is the slowest rank's
and the work the sum over ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + 5.0 * rank, "cpu")
    work = bench.reduce_sum(1000.0 * (rank + 1), "cpu")
    out[rank] = torch.tensor([ms, work])
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    out = torch.zeros(world, 2).share_memory_()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        assert out[r, 0].item() == 15.0      # slowest rank's time
        assert out[r, 1].item() == 3000.0    # all ranks' work


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.reduce_sum(7.0, "cpu") == 7.0
