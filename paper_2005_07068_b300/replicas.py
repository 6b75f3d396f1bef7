"""Multi-GPU runs as independent replicas (one process per GPU).

The swarm of one frame never needs another GPU's data, so N GPUs track N
independent sequences: rank r gets its own seed, nothing crosses the
interconnect on the data path, and the only collective is the final timing
reduction (the slowest rank sets the time, every rank's evaluations count).
"""
from __future__ import annotations

import torch


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s sequence (trajectory, noise and swarm streams)."""
    return base + 1000 * rank


def aggregate(local_seconds: float, local_evals: int, device=None) -> tuple[float, float, int]:
    """(whole-job evals/s, max seconds over ranks, total evals) over the
    default process group, or of this process alone when none is initialised."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return local_evals / local_seconds, local_seconds, local_evals
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    n = torch.tensor([local_evals], dtype=torch.int64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return float(n.item()) / float(t.item()), float(t.item()), int(n.item())
