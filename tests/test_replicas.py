"""Replicas on several ranks (the multi-GPU mode of the benchmark), over a world_size-2 gloo
group on CPU.

A single chain's GSE-TDVP1 sweep is sequential, so the benchmark's N-GPU mode runs one
independent replica per rank and exchanges nothing on the data path: only the slowest rank's
time is reduced.  Here each rank advances its own random-field Heisenberg chain by GSE-TDVP1
steps (Sec. I.C) with the CPU oracle standing in for the device path; the test checks that
every rank's trajectory equals the same replica run alone (no data crosses ranks) and that the
whole-job throughput is set by the slowest rank."""
import os
import socket
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

STEPS = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica(rank):
    """Rank r's own problem: an 8-site chain with seeded random fields (seed r), Neel start,
    real time dt = 0.05, k = 2, chi_max 8 (a small case of the batched workload)."""
    from paper_2005_06104_gb300 import workloads as wl
    rng = np.random.default_rng(rank)
    lat = wl.chain(8, 1.0, fields=rng.uniform(-2.0, 2.0, size=8))
    W = wl.heisenberg_mpo(lat)
    p = dict(tau=0.05, k=2, eps_k=1e-8, eps_m=1e-8, chi_max=8, dt=0.05, kind="real")
    return W, wl.neel_state(lat), p


def _run_replica(rank):
    import oracle as O
    W, psi, p = _replica(rank)
    for _ in range(STEPS):
        psi = O.gse_tdvp1_step(psi, W, p)
    return psi, O.energy_at_center(psi, W, 0)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t0 = time.perf_counter()
    psi, e = _run_replica(rank)
    if rank == 1:
        time.sleep(0.5)  # make rank 1 the slowest, so the reduction has something to decide
    t = time.perf_counter() - t0
    dist.barrier()
    t_max = bench.max_over_ranks(t, dist, "cpu")
    out[rank] = dict(t=t, t_max=t_max, throughput=bench.job_throughput(world, STEPS, t_max), energy=e,
                     sites=[np.asarray(a) for a in psi])
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_run_independent_chains_and_the_slowest_rank_sets_the_throughput():
    import oracle as O
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # the reduction: every rank sees the slowest rank's time
    assert res[0]["t_max"] == res[1]["t_max"] == max(res[0]["t"], res[1]["t"])
    assert res[1]["t"] > res[0]["t"]
    assert res[0]["throughput"] == pytest.approx(world * STEPS / res[1]["t"], rel=1e-12)
    # no data path between the ranks: each trajectory is that of its replica run alone
    for r in range(world):
        psi, e = _run_replica(r)
        assert abs(res[r]["energy"] - e) <= 1e-12 * abs(e)
        ov = O.mps_overlap(psi, res[r]["sites"])
        assert abs(abs(ov) - 1.0) <= 1e-12
    # and the two replicas are different problems
    assert abs(res[0]["energy"] - res[1]["energy"]) > 1e-3
