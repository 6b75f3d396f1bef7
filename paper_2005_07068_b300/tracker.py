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


def _capture(device, state: list, enqueue) -> torch.cuda.CUDAGraph:
    """Capture enqueue() into a CUDA graph.  One eager pass first resolves every
    lazy set-up (module loading, symbol lookups) that capture forbids; the
    tensors in `state` are saved before it and restored after, so capturing
    has no effect on the tracker."""
    cur = torch.cuda.current_stream(device)
    saved = [t.clone() for t in state]
    s = torch.cuda.Stream(device)
    s.wait_stream(cur)
    with torch.cuda.stream(s):
        enqueue()
    cur.wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        enqueue()
    for t, v in zip(state, saved):
        t.copy_(v)
    return g


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
        # record_history: each generation's global best and E kept on the device
        # by the frame's graph (runlog.RunLog reads them after the frame)
        self.record_history = record_history
        self.history = torch.zeros(gens, 27, **f) if record_history else None
        self.history_E = torch.zeros(gens, P, **f) if record_history else None
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
            self._after_render(obs, cur)
            if self.record_history:
                self.history_E[g - 1].copy_(self.swarm.E)
            self.swarm.x = cur
            hs.pso_step_fk(self.model, self.swarm, nxt, self.pso, self.seed, frame, g, self.cam, self.prims, self.kc)
            cur, nxt = nxt, cur
            if self.record_history:
                self.history[g - 1, :26].copy_(self.swarm.gbest)
                self.history[g - 1, 26:].copy_(self.swarm.gbest_E)
        self.swarm.x = cur

    def _after_render(self, obs: hs.Obs, x: torch.Tensor) -> None:
        """Hook between a generation's scoring and its swarm update (plain PSO: none)."""

    def _state(self) -> list:
        sw = self.swarm
        return [*self.x_buf, sw.v, sw.pbest, sw.pbest_E, sw.gbest, sw.gbest_E, sw.E, self.prims, self.kc,
                self.seed_pose]

    def graph(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None) -> torch.cuda.CUDAGraph:
        """The captured graph of enqueue_frame(obs, frame, seed_pose) (cached).
        Capturing leaves the tracker's state as it was."""
        key = (id(obs), frame, None if seed_pose is None else seed_pose.data_ptr())
        g = self._graphs.get(key)
        if g is None:
            g = _capture(self.device, self._state(), lambda: self.enqueue_frame(obs, frame, seed_pose))
            self._graphs[key] = g
        return g

    def run_frame(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None, graph: bool = True) -> None:
        if graph:
            self.graph(obs, frame, seed_pose).replay()
        else:
            self.enqueue_frame(obs, frame, seed_pose)

    def autotune(self, obs: hs.Obs, seed_pose: torch.Tensor, reps: int = 5) -> dict:
        """Pick the fastest render launch shape for this workload (the initial
        swarm of a frame around seed_pose) and use it from now on; returns the
        timing table.  Leaves the tracker's state as it was."""
        saved = [t.clone() for t in self._state()]
        self.seed_pose.copy_(seed_pose)
        hs.hs_obs_prepare(obs)
        self.swarm.x = self.x_buf[0]
        hs.pso_init(self.model, self.swarm, self.seed_pose, self.scale, self.seed, 0)
        hs.pose_fk(self.model, self.swarm.x, self.cam, self.prims, self.kc)
        self.score, table = hs.render_score_batch_autotune(self.model, obs, self.cam, self.prims, self.kc, self.score,
                                                           self.ws, self.swarm.E, reps)
        for t, v in zip(self._state(), saved):
            t.copy_(v)
        self._graphs.clear()
        return table

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


class FrameTracker(Tracker):
    """Plain PSO tracking with each frame in ONE cooperative launch (track_frame):
    `ctas` CTAs, dealt evenly to the particles, stay resident for the whole
    frame and meet at one grid barrier per generation.  Bit for bit the same
    swarm as Tracker (same observation, camera, P, seed); no CUDA graph is
    needed, a frame is a single launch.  ctas = 0 lets the library choose."""

    def __init__(self, model: hs.Model, cam: hs.HsCamera, P: int = 64, gens: int = 40, *, ctas: int = 0, **kw):
        super().__init__(model, cam, P, gens, **kw)
        if P > hs.FRAME_MAX_PARTICLES:
            raise ValueError(f"track_frame takes at most {hs.FRAME_MAX_PARTICLES} particles")
        if self.record_history:
            raise ValueError("the per-generation history is recorded by the step-by-step path (Tracker) only")
        self.ctas = ctas
        self.fws = hs.new_frame_workspace(P, self.device)

    def enqueue_frame(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None) -> None:
        src = self.swarm.gbest if seed_pose is None else seed_pose
        self.seed_pose.copy_(src)
        x0, x1 = self.x_buf
        self.swarm.x = x0
        hs.track_frame(self.model, obs, self.cam, self.swarm, x1, self.gens, self.score, self.pso, self.seed_pose,
                       self.scale, self.seed, frame, self.ctas, self.fws, self.kc, self.prims)
        self.swarm.x = self.x_buf[self.gens & 1]

    def run_frame(self, obs: hs.Obs, frame: int, seed_pose: torch.Tensor | None = None, graph: bool = True) -> None:
        self.enqueue_frame(obs, frame, seed_pose)

    def candidates(self) -> list[int]:
        """Grid sizes to try at this P: whole CTAs per particle (1, 2, 3, 4, 6, 8)
        and whole waves of the device's SMs, within the resident capacity."""
        cap = hs.frame_capacity()
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        sizes = {self.P * c for c in (1, 2, 3, 4, 6, 8)} | {sms * k for k in range(1, 9)} | {cap}
        return sorted(n for n in sizes if self.P <= n <= cap)

    def autotune(self, obs: hs.Obs, seed_pose: torch.Tensor, reps: int = 5) -> dict:
        """Pick the fastest grid size for this workload (whole frames from
        seed_pose, timed with CUDA events) and use it from now on; returns the
        timing table (us per frame).  Leaves the tracker's state as it was."""
        saved = [t.clone() for t in self._state()]
        keep = self.ctas
        table = {}
        for n in self.candidates():
            self.ctas = n
            self.enqueue_frame(obs, 0, seed_pose)  # warm
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(reps):
                self.enqueue_frame(obs, 0, seed_pose)
            t1.record()
            t1.synchronize()
            table[f"frame/n{n}"] = 1e3 * t0.elapsed_time(t1) / reps
        self.ctas = min(self.candidates(), key=lambda n: table[f"frame/n{n}"]) if table else keep
        for t, v in zip(self._state(), saved):
            t.copy_(v)
        self.swarm.x = self.x_buf[0]
        return table

    def launches_per_frame(self) -> int:
        """One cooperative launch per frame (plus the reset of the observation totals)."""
        return 1


class HybridTracker(Tracker):
    """Plain PSO plus, every generation, a gradient polish of the k best
    particles: `steps` normalised descent steps on the smoothed objective E_s
    (step lengths eta0, eta0 decay, ... in units of the per-parameter scale),
    then the polished poses are scored with the exact E and kept only where E
    fell.  The swarm update then proceeds as in plain PSO."""

    def __init__(self, model: hs.Model, cam: hs.HsCamera, P: int = 64, gens: int = 40, *, k: int = 8,
                 steps: int = 5, eta0: float = 0.3, decay: float = 0.7, soft=None, **kw):
        super().__init__(model, cam, P, gens, **kw)
        if not 1 <= k <= min(P, 256):
            raise ValueError("k must be in 1..min(P, 256)")
        self.k, self.steps = k, steps
        self.etas = [eta0 * decay ** i for i in range(steps)]
        self.soft = soft if soft is not None else hs.soft_params()
        self.score_k = hs.score_params(self.score.d_m, self.score.d_M, self.score.lambda_, self.score.lambda_k)
        f = dict(dtype=torch.float32, device=self.device)
        self.sel = torch.zeros(k, dtype=torch.int32, device=self.device)
        self.x_sel = torch.zeros(k, 26, **f)
        self.E_sel = torch.zeros(k, **f)
        self.E_new = torch.zeros(k, **f)
        self.E_soft = torch.zeros(k, **f)
        self.prims_k = torch.zeros(k, model.n_prims, 16, **f)
        self.kc_k = torch.zeros(k, **f)
        self.ws_k = hs.new_workspace(k, self.device)
        self.sums_k = torch.zeros(k, 3, **f)
        self.adj_k = torch.zeros(k, model.n_prims, hs.SOFT_ADJ, dtype=torch.int64, device=self.device)
        self.grad_k = torch.zeros(k, 26, **f)

    def _after_render(self, obs: hs.Obs, x: torch.Tensor) -> None:
        m, cam, k = self.model, self.cam, self.k
        hs.polish_select(self.swarm.E, k, self.sel)
        hs.polish_gather(x, self.swarm.E, self.sel, self.x_sel, self.E_sel)
        for eta in self.etas:
            hs.pose_fk(m, self.x_sel, cam, self.prims_k, self.kc_k)
            hs.soft_score(m, obs, cam, self.prims_k, self.kc_k, self.score_k, self.soft, self.ws_k, self.E_soft,
                          self.sums_k)
            hs.soft_score_backward(m, obs, cam, self.prims_k, self.score_k, self.soft, self.sums_k, self.adj_k)
            hs.pose_grad(m, self.x_sel, cam, self.score_k, self.prims_k, self.kc_k, self.adj_k, self.grad_k)
            hs.polish_step(m, self.x_sel, self.grad_k, eta, self.scale)
        hs.pose_fk(m, self.x_sel, cam, self.prims_k, self.kc_k)
        hs.render_score_batch(m, obs, cam, self.prims_k, self.kc_k, self.score_k, self.ws_k, self.E_new)
        hs.polish_keep_better(x, self.swarm.E, self.sel, self.x_sel, self.E_sel, self.E_new)

    def launches_per_frame(self) -> int:
        return super().launches_per_frame() + self.gens * (5 + 5 * self.steps)


# ---- many sequences at once ------------------------------------------------------------

def _round_up(n: int, a: int) -> int:
    return (n + a - 1) // a * a


class PackedObs:
    """The observations of S sequences in ONE device buffer, with a pinned host
    twin of the same layout, so a new frame for every sequence is one copy.
    Swarm s has a depth image [H_s, pitch] (uint16 mm, or float32 mm) and a skin
    mask [H_s, pitch] uint8, each starting on a 256-byte boundary with a row
    pitch that is a multiple of 16 bytes (the TMA requirement)."""

    def __init__(self, sizes, depth_f32: bool = False, device="cuda", pinned: bool = True):
        self.sizes = [(int(W), int(H)) for W, H in sizes]
        esz = 4 if depth_f32 else 2
        self.depth_dtype = torch.float32 if depth_f32 else torch.uint16
        self.layout = []  # (depth offset, depth pitch, skin offset, skin pitch) in bytes
        off = 0
        for W, H in self.sizes:
            dp, sp = _round_up(W * esz, 16), _round_up(W, 16)
            d0 = off
            s0 = _round_up(d0 + dp * H, 256)
            off = _round_up(s0 + sp * H, 256)
            self.layout.append((d0, dp, s0, sp))
        self.nbytes = off
        self.device = torch.device(device)
        self.dev = torch.zeros(self.nbytes, dtype=torch.uint8, device=self.device)
        self.host = torch.zeros(self.nbytes, dtype=torch.uint8, pin_memory=pinned)
        self.stats = torch.zeros(len(self.sizes), 2, dtype=torch.int32, device=self.device)
        self.obs = [self._obs(s) for s in range(len(self.sizes))]

    def _views(self, buf: torch.Tensor, s: int):
        (W, H), (d0, dp, s0, sp) = self.sizes[s], self.layout[s]
        esz = 4 if self.depth_dtype == torch.float32 else 2
        depth = buf[d0:d0 + dp * H].view(self.depth_dtype).view(H, dp // esz)
        skin = buf[s0:s0 + sp * H].view(H, sp)
        return depth, skin

    def _obs(self, s: int) -> hs.Obs:
        depth, skin = self._views(self.dev, s)
        W, H = self.sizes[s]
        return hs.Obs(depth, skin, W, H, self.stats[s])

    def write_host(self, s: int, depth: np.ndarray, skin: np.ndarray) -> None:
        """Place swarm s's frame (depth [H, W], skin [H, W]) into the host twin."""
        W, H = self.sizes[s]
        d, k = self._views(self.host, s)
        d[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(depth)).to(self.depth_dtype))
        k[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(skin).astype(np.uint8)))

    def upload(self, non_blocking: bool = True) -> None:
        """Host twin -> device buffer (a single copy)."""
        self.dev.copy_(self.host, non_blocking=non_blocking)


class BatchTracker:
    """Tracks S independent sequences together: every kernel of the frame loop
    runs once for all swarms (uneven ROI sizes and particle counts), and one
    CUDA graph holds a whole frame of every sequence.  Sequence s reproduces,
    bit for bit, a Tracker run with the same observation, camera, P and seed."""

    def __init__(self, model: hs.Model, batch: hs.Batch, gens: int = 40, *, score=None, pso=None, scale=None,
                 device="cuda"):
        self.model, self.batch, self.gens = model, batch, gens
        self.device = torch.device(device)
        self.score = score if score is not None else hs.score_params()
        self.pso = pso if pso is not None else hs.pso_params()  # n_mutate comes from each swarm
        if scale is None:
            scale = np.full(26, np.radians(10.0), np.float32)
            scale[:3] = 10.0
        self.scale = np.asarray(scale, np.float32)
        f = dict(dtype=torch.float32, device=self.device)
        self.swarm = hs.batch_swarm(batch, self.device)
        self.x_buf = (self.swarm.x, torch.zeros_like(self.swarm.x))
        self.prims = torch.zeros(batch.P_total, model.n_prims, 16, **f)
        self.kc = torch.zeros(batch.P_total, **f)
        self.ws = hs.new_workspace(batch.P_total, self.device)
        self.seed_poses = torch.zeros(batch.S, 26, **f)
        self._graphs: dict = {}

    def enqueue_frame(self, frame: int, seed_poses: torch.Tensor | None = None) -> None:
        """seed_poses: device [S, 26]; None = every swarm's current global best."""
        src = self.swarm.gbest if seed_poses is None else seed_poses
        self.seed_poses.copy_(src)
        hs.hs_obs_prepare_multi(self.batch)
        cur, nxt = self.x_buf
        self.swarm.x = cur
        hs.pso_init_multi(self.model, self.batch, self.swarm, self.seed_poses, self.scale, frame)
        hs.pose_fk_multi(self.model, self.batch, cur, self.prims, self.kc)
        for g in range(1, self.gens + 1):
            hs.render_score_multi(self.model, self.batch, self.prims, self.kc, self.score, self.ws, self.swarm.E)
            self.swarm.x = cur
            hs.pso_step_fk_multi(self.model, self.batch, self.swarm, nxt, self.pso, frame, g, self.prims, self.kc)
            cur, nxt = nxt, cur
        self.swarm.x = cur

    def _state(self) -> list:
        sw = self.swarm
        return [*self.x_buf, sw.v, sw.pbest, sw.pbest_E, sw.gbest, sw.gbest_E, sw.E, self.prims, self.kc,
                self.seed_poses]

    def graph(self, frame: int, seed_poses: torch.Tensor | None = None) -> torch.cuda.CUDAGraph:
        """The captured graph of enqueue_frame(frame, seed_poses) (cached); capturing
        leaves the state as it was."""
        key = (frame, None if seed_poses is None else seed_poses.data_ptr())
        g = self._graphs.get(key)
        if g is None:
            g = _capture(self.device, self._state(), lambda: self.enqueue_frame(frame, seed_poses))
            self._graphs[key] = g
        return g

    def run_frame(self, frame: int, seed_poses: torch.Tensor | None = None, graph: bool = True) -> None:
        if graph:
            self.graph(frame, seed_poses).replay()
        else:
            self.enqueue_frame(frame, seed_poses)

    def autotune(self, seed_poses: torch.Tensor, reps: int = 5) -> dict:
        """Pick the fastest render launch shape for the batch (the initial swarms
        around seed_poses [S, 26], the observations currently bound) and use it
        from now on; returns the timing table.  Leaves the state as it was."""
        saved = [t.clone() for t in self._state()]
        self.seed_poses.copy_(seed_poses)
        hs.hs_obs_prepare_multi(self.batch)
        self.swarm.x = self.x_buf[0]
        hs.pso_init_multi(self.model, self.batch, self.swarm, self.seed_poses, self.scale, 0)
        hs.pose_fk_multi(self.model, self.batch, self.swarm.x, self.prims, self.kc)
        self.score, table = hs.render_score_multi_autotune(self.model, self.batch, self.prims, self.kc, self.score,
                                                           self.ws, self.swarm.E, reps)
        for t, v in zip(self._state(), saved):
            t.copy_(v)
        self._graphs.clear()
        return table

    def launches_per_frame(self) -> int:
        """Kernels per frame for all swarms: 2 observation passes, init, FK, 2 per generation."""
        return 4 + 2 * self.gens

    def evals_per_frame(self) -> int:
        return self.batch.P_total * self.gens


class BatchFrameTracker(BatchTracker):
    """BatchTracker with each frame of every sequence in ONE cooperative launch
    (track_frame_multi, after the two observation passes): the resident CTAs
    take per-particle tasks (a particle's step, FK, render and E) generation by
    generation, each swarm advancing as soon as all its particles are scored,
    with no grid barrier.  Bit for bit the same swarms as BatchTracker.  ctas =
    0 uses every CTA the device keeps resident."""

    def __init__(self, model: hs.Model, batch: hs.Batch, gens: int = 40, *, ctas: int = 0, **kw):
        super().__init__(model, batch, gens, **kw)
        if max(batch.P) > hs.FRAME_MAX_PARTICLES:
            raise ValueError(f"track_frame_multi takes at most {hs.FRAME_MAX_PARTICLES} particles per swarm")
        self.ctas = ctas
        self.fws = hs.new_frame_multi_workspace(batch, self.device)

    def enqueue_frame(self, frame: int, seed_poses: torch.Tensor | None = None) -> None:
        src = self.swarm.gbest if seed_poses is None else seed_poses
        self.seed_poses.copy_(src)
        x0, x1 = self.x_buf
        self.swarm.x = x0
        hs.track_frame_multi(self.model, self.batch, self.swarm, x1, self.gens, self.score, self.pso,
                             self.seed_poses, self.scale, frame, self.ctas, self.fws, self.prims, self.kc)
        self.swarm.x = self.x_buf[self.gens & 1]

    def run_frame(self, frame: int, seed_poses: torch.Tensor | None = None, graph: bool = True) -> None:
        self.enqueue_frame(frame, seed_poses)

    def candidates(self) -> list[int]:
        """Grid sizes to try: whole waves of the device's SMs up to the batch's resident capacity."""
        cap = hs.frame_multi_capacity(self.batch, self.model)
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        return sorted({sms * k for k in range(1, 8)} & set(range(1, cap + 1)) | {cap})

    def autotune(self, seed_poses: torch.Tensor, reps: int = 3) -> dict:
        """Pick the fastest grid size (the kernel renders with its own unit
        renderer, so there is no render kernel to choose): whole frames from
        seed_poses [S, 26], timed with CUDA events; returns the table (us per
        frame) and leaves the tracker's state as it was."""
        saved = [t.clone() for t in self._state()]
        keep, cur = self.ctas, self.swarm.x
        table = {}
        for n in self.candidates():
            self.ctas = n
            self.enqueue_frame(0, seed_poses)  # warm
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(reps):
                self.enqueue_frame(0, seed_poses)
            t1.record()
            t1.synchronize()
            table[f"frame_multi/n{n}"] = 1e3 * t0.elapsed_time(t1) / reps
        self.ctas = min(self.candidates(), key=lambda n: table[f"frame_multi/n{n}"]) if table else keep
        for t, v in zip(self._state(), saved):
            t.copy_(v)
        self.swarm.x = cur
        return table

    def launches_per_frame(self) -> int:
        """The two observation passes and the frame."""
        return 3
