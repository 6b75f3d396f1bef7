"""Oracle work for the GPU tests spread over host processes.

The oracle's complex-step gradient of E_s takes seconds per pose, so the GPU
gradient tests hand it to a pool of processes.  The pool is started with
`spawn` (a fresh interpreter per worker, no CUDA context inherited), and this
module imports nothing but the oracle and numpy, so a worker never touches the
GPU.  Each worker keeps one numpy thread; the pool size is the host's cores.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_SCENE = None


def _init(model, cam, Od, S):
    os.environ["OMP_NUM_THREADS"] = "1"
    global _SCENE
    _SCENE = (model, cam, Od, S)


def _cs_gradient(pose):
    from oracle import soft
    m, cam, Od, S = _SCENE
    return soft.soft_gradient(m, pose, cam, Od, S)


def _central_differences(pose):
    """FP64 central differences at h (1e-4 rad / 1e-2 mm) and at 2h."""
    from oracle import soft
    m, cam, Od, S = _SCENE
    return (soft.central_difference(m, pose, cam, Od, S),
            soft.central_difference(m, pose, cam, Od, S, h_rad=2e-4, h_mm=2e-2))


def _objective(pose):
    from oracle import soft
    m, cam, Od, S = _SCENE
    return soft.soft_objective(m, pose, cam, Od, S)


def run(kind: str, model, cam, Od, S, poses):
    """kind: 'cs' (complex-step gradients), 'fd' (central differences at h and
    2h) or 'E' (E_s) of every pose, computed by a spawn pool."""
    fn = {"cs": _cs_gradient, "fd": _central_differences, "E": _objective}[kind]
    procs = max(1, min(len(poses), os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_init, initargs=(model, np.asarray(cam), np.asarray(Od), np.asarray(S))) as pool:
        return pool.map(fn, [np.asarray(p, np.float64) for p in poses])
