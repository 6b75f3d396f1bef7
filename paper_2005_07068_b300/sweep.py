"""Seconds per frame to track within a joint-angle accuracy (the full-frame sweep).

A sequence is tracked frame by frame (Section III.B: PSO per frame, seeded
from the previous frame's global best) with a fixed generation budget G and
swarm size P.  Each frame is one captured graph timed with CUDA events; after
it, the global best is compared with the ground truth in mean absolute
joint-angle error over the 23 angular DOFs.  A setting "tracks within X
degrees" when at least a given fraction of the frames end within X; the
metric is the shortest frame time among the settings that do.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

ANGULAR = slice(3, 26)  # the 23 angular DOFs (wrist translation excluded)


def mean_joint_error_deg(pose: np.ndarray, gt: np.ndarray) -> np.ndarray:
    """Mean |pose - gt| over the angular DOFs, in degrees (last axis = 26 DOFs)."""
    return np.degrees(np.abs(np.asarray(pose, np.float64)[..., ANGULAR] - np.asarray(gt, np.float64)[..., ANGULAR])
                      .mean(axis=-1))


@dataclass
class FrameResult:
    frame: int
    frame_ms: float           # the whole frame (observation totals, init, FK, G generations), CUDA events
    final_error_deg: float    # global best vs ground truth after the frame
    final_E: float


def track_sequence(trk, obs: list, gt: np.ndarray, start: torch.Tensor, frames: int | None = None,
                   log=None, **log_fields) -> list[FrameResult]:
    """Track obs[0..frames) with `trk` (a Tracker), frame 0 from `start`.  With
    `log` (a runlog.RunLog; the tracker built with record_history=True), every
    frame's generations are written to it, tagged with log_fields."""
    n = len(obs) if frames is None else min(frames, len(obs))
    stream = torch.cuda.current_stream()
    graphs = [trk.graph(obs[f], f, start if f == 0 else None) for f in range(n)]
    out = []
    for f in range(n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graphs[f].replay()
        e1.record(stream)
        torch.cuda.synchronize()
        gbest = trk.swarm.gbest.cpu().numpy()
        out.append(FrameResult(f, e0.elapsed_time(e1), float(mean_joint_error_deg(gbest, gt[f])),
                               float(trk.swarm.gbest_E.cpu()[0])))
        if log is not None:
            log.frame_from(trk, f, gt[f], frame_ms=out[-1].frame_ms, **log_fields)
    return out


def summarize(results: list[FrameResult], threshold_deg: float = 5.0) -> dict:
    err = np.array([r.final_error_deg for r in results])
    return {
        "frames": len(results),
        "within_fraction": float((err <= threshold_deg).mean()) if err.size else 0.0,
        "final_error_deg_mean": float(err.mean()) if err.size else None,
        "final_error_deg_median": float(np.median(err)) if err.size else None,
        "final_error_deg_p90": float(np.percentile(err, 90)) if err.size else None,
        "frame_ms_mean": float(np.mean([r.frame_ms for r in results])) if results else None,
    }


def fastest_within(settings: list[dict], fraction: float = 0.9) -> dict | None:
    """The setting with the shortest mean frame time among those whose frames end
    within the threshold at least `fraction` of the time (None if none does)."""
    ok = [s for s in settings if s["within_fraction"] >= fraction]
    return min(ok, key=lambda s: s["frame_ms_mean"]) if ok else None
