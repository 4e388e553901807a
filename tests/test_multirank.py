"""The benchmark's multi-GPU path is replicas only (each rank an independent
simulation, no data-path collective; a barrier and a MAX over ranks for timing).
Its host logic runs here with two gloo ranks on the CPU: per-rank noise seeds,
the slowest rank's time, the whole-job rate, and that each rank's maps are
exactly those of the same seed run alone (the oracle stands in for the GPU)."""
import os
import socket

import numpy as np

import bench
from oracle.sim import Simulation
from pm_inputs import white_noise, workload

W = dict(nc=8, nmesh=16, nsteps=3, map_npix=8, zs=(1.0,))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workload("pm64", **W)
    seed = bench.rank_noise_seed(w, rank)
    kappa = Simulation(**w).run(white_noise(w["nc"], seed))
    slow = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    rate = bench.aggregate_rate(world, w["nc"] ** 3, w["nsteps"], slow)
    got = [None] * world
    dist.all_gather_object(got, (seed, kappa, slow, rate))
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = workload("pm64", **W)
    seeds = [g[0] for g in got]
    assert seeds == [w["noise_seed"], w["noise_seed"] + 1]
    assert all(g[2] == 15.0 for g in got)                                  # the slowest rank
    assert all(abs(g[3] - 2 * 8 ** 3 * 3 / 0.015) < 1e-6 * g[3] for g in got)
    for s, kappa, _, _ in got:
        assert np.array_equal(kappa, Simulation(**w).run(white_noise(w["nc"], s)))
    assert not np.allclose(got[0][1], got[1][1])


def test_single_rank_helpers():
    w = workload("pm64", **W)
    assert bench.rank_noise_seed(w, 0) == w["noise_seed"]
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate_rate(1, 100, 10, 2.0) == 100 * 10 / 0.002
