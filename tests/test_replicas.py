"""Replicas on several ranks (the multi-GPU mode of the benchmark): the slowest rank's time
and the whole-job throughput, over a world_size-2 gloo group on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [3.0, 5.0][rank]  # seconds each replica took for its steps
    dist.barrier()
    t_max = bench.max_over_ranks(t, dist, "cpu")
    out[rank] = (t_max, bench.job_throughput(world, 4, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_throughput():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (5.0, 2 * 4 / 5.0)
