"""The multi-GPU path of bench.py is replicas only: every rank runs the whole
workload, the job time is the slowest rank's and throughput adds up.  This
checks that plumbing with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    ms = 100.0 * (rank + 1)          # rank 1 is the slowest
    m = bench.max_over_ranks(ms, dist)
    out[rank] = (m, bench.job_throughput(50, world, m))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (200.0, 2 * 50 / 0.2)
