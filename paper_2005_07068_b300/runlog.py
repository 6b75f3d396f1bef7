"""Run records and checkpoints for the trackers (host side, off the hot path).

* RunLog writes JSON lines: one per generation of a tracked frame (the
  swarm's best and mean E -- the quantities of the paper's cost-per-generation
  plots, Section V -- and, with a ground truth, the best pose's mean joint-angle
  error) and one per run (whatever summary the caller passes, e.g. evals/s and
  the render's roofline fraction).  A Tracker built with record_history=True
  keeps each generation's global best and E in device buffers that the frame's
  graph fills; RunLog reads them after the frame.
* save_checkpoint / load_checkpoint store and restore a tracker's whole swarm
  state (positions, velocities, personal and global bests, E, records, kc and
  the seed pose) with the index of the frame that comes next.  Random numbers
  are drawn from (seed, frame, generation, particle) counters, so a tracker
  restored into a fresh process continues bit for bit as if never stopped.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from .sweep import mean_joint_error_deg

CHECKPOINT_VERSION = 1


class RunLog:
    """JSON-lines records of tracked frames and runs.  `out` is a path (opened
    for appending) or a text stream."""

    def __init__(self, out):
        self._own = isinstance(out, str)
        self._f = open(out, "a") if self._own else out

    def close(self) -> None:
        if self._own:
            self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _write(self, rec: dict) -> None:
        self._f.write(json.dumps(rec, sort_keys=True) + "\n")

    def generations(self, frame: int, gbest: np.ndarray, gbest_E: np.ndarray, E: np.ndarray,
                    gt: np.ndarray | None = None, **extra) -> None:
        """One line per generation g = 1..G of frame `frame`: gbest [G, 26] and
        gbest_E [G] after generation g, E [G, P] the swarm's objectives scored
        at generation g; gt [26] the ground-truth pose, if known."""
        gbest = np.asarray(gbest, np.float64)
        gbest_E = np.asarray(gbest_E, np.float64).reshape(-1)
        E = np.asarray(E, np.float64)
        if not (gbest.shape[0] == gbest_E.shape[0] == E.shape[0]):
            raise ValueError("gbest, gbest_E and E must have one row per generation")
        err = mean_joint_error_deg(gbest, gt) if gt is not None else None
        for g in range(E.shape[0]):
            rec = {"type": "generation", "frame": int(frame), "gen": g + 1, "best_E": float(gbest_E[g]),
                   "mean_E": float(E[g].mean()), "min_E": float(E[g].min())}
            if err is not None:
                rec["best_error_deg"] = float(err[g])
            rec.update(extra)
            self._write(rec)

    def frame_from(self, trk, frame: int, gt: np.ndarray | None = None, **extra) -> None:
        """The generations of the frame `trk` (a Tracker with record_history)
        has just tracked."""
        if trk.history is None:
            raise ValueError("the tracker keeps no history (record_history=False)")
        h = trk.history.cpu().numpy()
        self.generations(frame, h[:, :26], h[:, 26], trk.history_E.cpu().numpy(), gt, **extra)

    def run(self, **summary) -> None:
        self._write({"type": "run", **summary})


def _current_index(trk) -> int:
    return 0 if trk.swarm.x.data_ptr() == trk.x_buf[0].data_ptr() else 1


def save_checkpoint(trk, path, next_frame: int) -> None:
    """Store the swarm state of `trk` (Tracker, FrameTracker, HybridTracker,
    BatchTracker or BatchFrameTracker) and the index of the next frame."""
    state = [t.detach().cpu().clone() for t in trk._state()]
    torch.save({"version": CHECKPOINT_VERSION, "kind": type(trk).__name__, "next_frame": int(next_frame),
                "current": _current_index(trk), "gens": int(trk.gens),
                "seed": getattr(trk, "seed", None), "state": state}, path)


def load_checkpoint(trk, path) -> int:
    """Restore a checkpoint into `trk` (the same kind of tracker, built with the
    same swarm sizes, model and seed) and return the index of the next frame.
    Raises ValueError when the checkpoint does not fit the tracker."""
    ck = torch.load(path, map_location="cpu", weights_only=True)
    if ck.get("version") != CHECKPOINT_VERSION:
        raise ValueError(f"checkpoint version {ck.get('version')} (expected {CHECKPOINT_VERSION})")
    if ck["kind"] != type(trk).__name__ or ck["gens"] != trk.gens or ck["seed"] != getattr(trk, "seed", None):
        raise ValueError("the checkpoint was taken from another kind of tracker or other settings")
    dst = trk._state()
    if len(dst) != len(ck["state"]) or any(d.shape != s.shape or d.dtype != s.dtype
                                           for d, s in zip(dst, ck["state"])):
        raise ValueError("the checkpoint's swarm state does not fit this tracker")
    for d, s in zip(dst, ck["state"]):
        d.copy_(s)
    trk.swarm.x = trk.x_buf[ck["current"]]
    return int(ck["next_frame"])
