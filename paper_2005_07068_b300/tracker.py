"""Frame-by-frame tracking on one GPU through the C-ABI (Section III.B loop).

One frame = per-frame observation preparation, swarm initialisation around
the previous frame's global best (tracking) and FK of the initial swarm, then
`gens` generations of render_score_batch -> pso_step_fk (the swarm update
fused with the FK of the new positions; positions alternate between two
buffers).  The whole frame is captured once into a CUDA graph per
(observation buffer, frame index), so a frame costs a single graph launch and
no host round trip; the host reads only the final global best.
"""
from __future__ import annotations

import numpy as np
import torch

from . import handscore as hs


class Tracker:
    def __init__(self, model: hs.Model, cam: hs.HsCamera, P: int = 64, gens: int = 40, *, seed: int = 1,
                 score=None, pso=None, scale=None, device="cuda", record_history: bool = False):
        self.model, self.cam, self.P, self.gens, self.seed = model, cam, P, gens, seed
        self.device = torch.device(device)
        self.score = score if score is not None else hs.score_params()
        self.pso = pso if pso is not None else hs.pso_params(P=P)
        if scale is None:
            scale = np.full(26, np.radians(10.0), np.float32)
            scale[:3] = 10.0
        self.scale = np.asarray(scale, np.float32)
        f = dict(dtype=torch.float32, device=self.device)
        self.swarm = hs.Swarm.empty(P, self.device)
        self.x_buf = (self.swarm.x, torch.zeros_like(self.swarm.x))  # double-buffered positions
        self.prims = torch.zeros(P, model.n_prims, 16, **f)
        self.kc = torch.zeros(P, **f)
        self.ws = hs.new_workspace(P, self.device)
        self.seed_pose = torch.zeros(26, **f)
        self.record_history = record_history
        self.history = torch.zeros(gens, 27, **f) if record_history else None
        self._graphs: dict = {}

    # ---- one frame, enqueued on the current stream ---------------------------------
    def enqueue_frame(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None) -> None:
        """seed_pose: device [26] to start from; None = the current global best."""
        src = self.swarm.gbest if seed_pose is None else seed_pose
        self.seed_pose.copy_(src)
        hs.hs_obs_prepare(obs)
        cur, nxt = self.x_buf
        self.swarm.x = cur
        hs.pso_init(self.model, self.swarm, self.seed_pose, self.scale, self.seed, frame)
        hs.pose_fk(self.model, cur, self.cam, self.prims, self.kc)
        for g in range(1, self.gens + 1):
            hs.render_score_batch(self.model, obs, self.cam, self.prims, self.kc, self.score, self.ws, self.swarm.E)
            self.swarm.x = cur
            hs.pso_step_fk(self.model, self.swarm, nxt, self.pso, self.seed, frame, g, self.cam, self.prims, self.kc)
            cur, nxt = nxt, cur
            if self.record_history:
                self.history[g - 1, :26].copy_(self.swarm.gbest)
                self.history[g - 1, 26:].copy_(self.swarm.gbest_E)
        self.swarm.x = cur

    def graph(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None) -> torch.cuda.CUDAGraph:
        """The captured graph of enqueue_frame(obs, frame, seed_pose) (cached)."""
        key = (id(obs), frame, None if seed_pose is None else seed_pose.data_ptr())
        g = self._graphs.get(key)
        if g is None:
            s = torch.cuda.Stream(self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):  # one eager pass resolves every lazy set-up before capture
                self.enqueue_frame(obs, frame, seed_pose)
            torch.cuda.current_stream(self.device).wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                self.enqueue_frame(obs, frame, seed_pose)
            self._graphs[key] = g
        return g

    def run_frame(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None, graph: bool = True) -> None:
        if graph:
            self.graph(obs, frame, seed_pose).replay()
        else:
            self.enqueue_frame(obs, frame, seed_pose)

    def launches_per_frame(self) -> int:
        """Kernels of this library per frame: obs stats, init, FK, 2 per generation."""
        return 3 + 2 * self.gens

    # ---- end to end from host memory ---------------------------------------------------
    def track(self, depth_host: torch.Tensor, skin_host: torch.Tensor, staging: hs.Obs, frame: int,
              out_host: torch.Tensor, seed_pose: torch.Tensor | None = None) -> None:
        """Copy one pinned host frame into `staging`, run the frame's graph and copy
        the global best (26 pose values + its E) into pinned `out_host` [27]."""
        staging.depth.copy_(depth_host, non_blocking=True)
        staging.skin.copy_(skin_host, non_blocking=True)
        self.run_frame(staging, frame, seed_pose)
        out_host[:26].copy_(self.swarm.gbest, non_blocking=True)
        out_host[26:].copy_(self.swarm.gbest_E, non_blocking=True)
