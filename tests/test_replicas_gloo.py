"""Multi-process replica path on CPU (gloo, world size 2): each rank tracks its
own seeded sequence (the oracle's tracking stands in for the GPU path here),
and the job's throughput is all ranks' evaluations over the slowest rank's
time, reduced over the process group as bench.py does."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import replicas as R


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    """One replica: its own seeded sequence, a real (CPU oracle) tracking
    workload on it -- the GPU path's stand-in on a machine without GPUs --
    timed, then aggregated over the ranks as bench.py does."""
    import time

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = R.replica_seed(I.CONFIG_SEED_BASE + 2, rank)
        traj = I.trajectory(seed, 2)
        W = H = 40
        g = I.hand_geometry()
        lo, hi = I.search_limits()
        model = oracle.Model.from_geometry(g, lo, hi)
        cam = oracle.camera_tuple(I.kinect_camera(W, H))
        cam[:2] *= 2.5
        depth, hit, _, _ = oracle.render_pose(model, traj[0], cam, W, H, boundary=False)
        Od, S = I.kinect_observation(depth, hit, seed * 100)
        P, gens = 6, 2
        t0 = time.perf_counter()
        sw = oracle.pso_init(P, traj[0], I.perturbation_scale(), model.lo, model.hi, seed, 0)
        for gen in range(1, gens + 1):
            r = oracle.score_batch(model, sw.x, cam, Od.astype(np.float64), S)
            sw = oracle.pso_step(sw, r["E"], model.lo, model.hi, seed, 0, gen)
        secs = time.perf_counter() - t0
        value, tmax, total = R.aggregate(secs, P * gens)
        out[rank] = (seed, float(sw.gbest_E), secs, value, tmax, total)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, e0, l0, v0, t0, n0), (s1, e1, l1, v1, t1, n1) = res[0], res[1]
    assert s0 != s1 and e0 != e1              # independent sequences, independently tracked
    assert t0 == t1 == max(l0, l1)            # the slowest rank's time
    assert n0 == n1 == 2 * 6 * 2              # every rank's evaluations
    assert v0 == v1 == n0 / t0


def test_single_process_aggregate():
    assert R.aggregate(2.0, 100) == (50.0, 2.0, 100)
    assert R.replica_seed(10, 0) == 10 and R.replica_seed(10, 3) == 3010
    assert not np.array_equal(I.trajectory(R.replica_seed(5, 0), 3), I.trajectory(R.replica_seed(5, 1), 3))
