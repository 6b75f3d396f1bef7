"""The smoothed objective E_s as a differentiable PyTorch function.

SoftScorer binds a model, an observation and a camera; scorer(poses) returns
E_s [P] for poses [P, 26] (float32, CUDA) through SoftObjective, whose
backward runs the library's adjoint kernels (soft_score_backward, then
pose_grad).  Argument marshalling only: every step runs in the CUDA kernels.
"""
from __future__ import annotations

import torch

from . import handscore as hs


class SoftScorer:
    def __init__(self, model: hs.Model, obs: hs.Obs, cam: hs.HsCamera, params: hs.HsScoreParams | None = None,
                 soft: hs.HsSoftParams | None = None, max_particles: int = 64, device="cuda"):
        self.model, self.obs, self.cam = model, obs, cam
        self.params = params if params is not None else hs.score_params()
        self.soft = soft if soft is not None else hs.soft_params()
        self.device = torch.device(device)
        self._alloc(max_particles)

    def _alloc(self, P: int) -> None:
        f = dict(dtype=torch.float32, device=self.device)
        self.cap = P
        self.prims = torch.zeros(P, self.model.n_prims, 16, **f)
        self.kc = torch.zeros(P, **f)
        self.ws = hs.new_workspace(P, self.device)
        self.sums = torch.zeros(P, 3, **f)
        self.adj = torch.zeros(P, self.model.n_prims, hs.SOFT_ADJ, dtype=torch.int64, device=self.device)
        self.grad = torch.zeros(P, 26, **f)

    def forward(self, poses: torch.Tensor) -> torch.Tensor:
        """E_s [P] (no graph)."""
        P = poses.shape[0]
        if P > self.cap:
            self._alloc(P)
        E = torch.empty(P, dtype=torch.float32, device=self.device)
        hs.pose_fk(self.model, poses, self.cam, self.prims[:P], self.kc[:P])
        hs.soft_score(self.model, self.obs, self.cam, self.prims[:P], self.kc[:P], self.params, self.soft,
                      self.ws, E, self.sums[:P])
        return E

    def gradient(self, poses: torch.Tensor) -> torch.Tensor:
        """dE_s/dpose [P, 26]; call after forward(poses) with the same poses."""
        P = poses.shape[0]
        hs.soft_score_backward(self.model, self.obs, self.cam, self.prims[:P], self.params, self.soft,
                               self.sums[:P], self.adj[:P])
        hs.pose_grad(self.model, poses, self.cam, self.params, self.prims[:P], self.kc[:P], self.adj[:P],
                     self.grad[:P])
        return self.grad[:P]

    def __call__(self, poses: torch.Tensor) -> torch.Tensor:
        return SoftObjective.apply(poses, self)


class SoftObjective(torch.autograd.Function):
    """E_s(poses) with dE_s/dposes from the adjoint kernels."""

    @staticmethod
    def forward(ctx, poses: torch.Tensor, scorer: SoftScorer) -> torch.Tensor:
        poses = poses.detach().contiguous()
        E = scorer.forward(poses)
        ctx.scorer = scorer
        ctx.save_for_backward(poses)
        return E

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        (poses,) = ctx.saved_tensors
        sc = ctx.scorer
        sc.forward(poses)  # the records and sums of these poses (another call may have replaced them)
        g = sc.gradient(poses)
        return gE.to(g.dtype)[:, None] * g, None
