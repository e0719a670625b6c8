"""The multi-GPU form is replicas: every rank runs its own job and the bench reports the
slowest rank's time.  The aggregation runs here as two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 17.25][rank]                       # the ranks' own step times
    out[rank] = bench.replica_max(ms, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        assert dict(out) == {0: 17.25, 1: 17.25}


def test_without_a_group_the_value_is_unchanged():
    import bench
    assert bench.replica_max(3.5) == 3.5
