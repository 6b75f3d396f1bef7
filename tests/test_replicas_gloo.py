"""Multi-process replica path on CPU (gloo, world size 2): each rank tracks its
own sequence, and the job's throughput is all ranks' evaluations over the
slowest rank's time."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = R.replica_seed(I.CONFIG_SEED_BASE + 2, rank)
        traj = I.trajectory(seed, 5)
        # a rank that is slower and did more work, deterministic per rank
        secs = 1.0 + rank
        evals = 1000 * (rank + 1)
        value, tmax, total = R.aggregate(secs, evals)
        out[rank] = (seed, float(traj[2, 7]), value, tmax, total)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, a0, v0, t0, n0), (s1, a1, v1, t1, n1) = res[0], res[1]
    assert s0 != s1 and a0 != a1              # independent sequences
    assert t0 == t1 == 2.0                    # max over ranks
    assert n0 == n1 == 3000                   # all ranks' evaluations
    assert v0 == v1 == 1500.0


def test_single_process_aggregate():
    assert R.aggregate(2.0, 100) == (50.0, 2.0, 100)
    assert R.replica_seed(10, 0) == 10 and R.replica_seed(10, 3) == 3010
    assert not np.array_equal(I.trajectory(R.replica_seed(5, 0), 3), I.trajectory(R.replica_seed(5, 1), 3))
