"""GPU: the smoothed objective E_s and its gradient dE_s/dpose (FP32 adjoint
kernels) against the FP64 oracle: its E_s on every pose, its complex-step
gradient (which the CPU suite pins to FP64 central differences) on 32 poses,
and FP64 central differences of E_s (h = 1e-4 rad / 1e-2 mm) directly on 8
poses.  The scene is the differentiation workload: a 128x128 ROI, seeded poses
around a seeded ground truth; plus the autograd wrapper.  The oracle's work
runs in a spawn pool of host processes (tests/oracle_pool.py)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import grad as G
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I
from tests import gpu_common as C
from tests import oracle_pool as OP

pytestmark = pytest.mark.gpu

REPORT = {}
N_POSES = 256          # poses scored and differentiated on the GPU
N_ORACLE_GRAD = 32     # of which this many get the oracle's complex-step gradient (26 complex evaluations each)
N_FD = 8               # and this many FP64 central differences at h and 2h (104 evaluations each)
# Tolerances, derived from FP32 rounding (not fitted to the measured errors):
#  * E_s: every pixel term is a chain of at most ~300 FP32 roundings (the
#    smoothed evaluation of each touching primitive, the front-to-back
#    compositing of up to a few of them, the soft |.|, clamp and sigmoids), so
#    it carries at most 300 u = 1.8e-5 relative error (u = 2^-24); the three
#    sums add non-negative terms exactly (fixed point), which keeps that
#    relative bound, and E_s is formed from two ratios of them, which at most
#    doubles it: 3.6e-5 -> 4e-5 relative.  The floor is the hard objective's:
#    FP32 records place surfaces to ~1e-4 mm.
#  * gradient: the FP32 records place each silhouette within ~1.5e-4 px of
#    its FP64 position (the cones; ellipsoids 2e-5 px), and the smoothed
#    coverage sigma(delta / tau) has a slope that changes by sigma''/sigma' ~
#    1 / tau per pixel of shift, so a silhouette pixel's contribution to the
#    gradient carries up to 1.5e-4 / 0.5 = 3e-4 relative error, all of one
#    sign along a silhouette (a systematic shift).  Silhouette pixels carry at
#    most about half of a component's magnitude, and the largest component
#    bounds every other's, so the bound is 3e-4 / 2 = 1.5e-4 -> 2e-4 of the
#    largest component.  Rounding in the adjoint chains (~200 roundings,
#    1.2e-5 relative per contribution, summed exactly in 2^-40 fixed point)
#    is an order of magnitude below that.
E_S_REL_TOL = 4e-5
E_S_ABS_TOL = 1e-4
GRAD_TOL = 2e-4        # of the gradient's largest component


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)
    yield
    out = os.environ.get("HS_GRAD_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)


@pytest.fixture(scope="module")
def scene():
    sc = C.make_scene(128, 128, 1, 2005070683, zoom=2.2, noisy=True, f32=False)
    lo, hi = I.search_limits()
    margin = np.where(np.arange(26) < 3, 1.0, 0.02)  # strictly inside the limits (the clamp is one-sided there)
    rng = np.random.default_rng(2005070683)
    poses = sc.gt[None].astype(np.float64) + rng.uniform(-1, 1, (N_POSES, 26)) * I.perturbation_scale()
    poses = np.clip(poses, lo + margin, hi - margin).astype(np.float32)
    return sc, poses


def _gpu(sc, poses):
    dev = torch.device("cuda")
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    hs.hs_obs_prepare(obs)
    cam = hs.camera(*[float(v) for v in sc.cam])
    scorer = G.SoftScorer(sc.model_g, obs, cam, max_particles=poses.shape[0])
    tp = torch.from_numpy(poses).to(dev)
    E = scorer.forward(tp)
    g = scorer.gradient(tp)
    torch.cuda.synchronize()
    return scorer, tp, E.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)


def _oracle_args(sc):
    return sc.model_o, sc.cam.astype(np.float64), sc.Od.astype(np.float64), sc.S


def test_soft_objective_and_gradient_match_oracle(scene):
    sc, poses = scene
    _, _, E_gpu, g_gpu = _gpu(sc, poses)
    assert hs.hs_get_device_status(clear=True) == 0
    E_o = np.array(OP.run("E", *_oracle_args(sc), poses))
    e_err = np.abs(E_gpu - E_o)
    REPORT["E_s_max_abs_err"] = float(e_err.max())
    REPORT["E_s_max_rel_err"] = float((e_err / np.abs(E_o)).max())
    assert np.all(e_err <= E_S_REL_TOL * np.abs(E_o) + E_S_ABS_TOL), (e_err.max(), (e_err / np.abs(E_o)).max())
    idx = np.linspace(0, N_POSES - 1, N_ORACLE_GRAD).astype(int)
    rels = []
    for k, go in zip(idx, OP.run("cs", *_oracle_args(sc), poses[idx])):
        scale = np.abs(go).max()
        rel = np.abs(g_gpu[k] - go).max() / scale
        cos = float(g_gpu[k] @ go / (np.linalg.norm(g_gpu[k]) * np.linalg.norm(go)))
        rels.append((float(rel), cos))
    REPORT["grad_poses"] = len(rels)
    REPORT["grad_max_err_over_max_abs"] = max(r for r, _ in rels)
    REPORT["grad_min_cosine"] = min(c for _, c in rels)
    assert all(r <= GRAD_TOL for r, _ in rels), rels
    # a relative error e of the largest component bounds 1 - cos by 26 e^2 / 2
    assert all(c >= 1 - 26 * GRAD_TOL ** 2 / 2 for _, c in rels), rels
    assert np.all(np.isfinite(g_gpu))


def test_gradient_matches_central_differences(scene):
    """The GPU gradient against FP64 central differences of the oracle's E_s
    (h = 1e-4 rad / 1e-2 mm), with no complex step in between.  The tolerance
    per component is the FP32 bound above plus twice the differences' own
    truncation error, estimated by Richardson from the differences at 2h
    (error(h) ~ (D(2h) - D(h)) / 3 for a central difference)."""
    sc, poses = scene
    _, _, _, g_gpu = _gpu(sc, poses)
    idx = np.linspace(3, N_POSES - 4, N_FD).astype(int)
    worst = []
    for k, (d1, d2) in zip(idx, OP.run("fd", *_oracle_args(sc), poses[idx])):
        scale = np.abs(d1).max()
        assert scale > 1.0
        trunc = np.abs(d2 - d1) / 3.0
        tol = GRAD_TOL * scale + 2.0 * trunc
        err = np.abs(g_gpu[k] - d1)
        assert np.all(err <= tol), (k, (err / scale).max(), (trunc / scale).max())
        worst.append(float((err / scale).max()))
    REPORT["grad_vs_fd_max_err_over_max_abs"] = max(worst)


def test_autograd_function_matches_direct_calls(scene):
    sc, poses = scene
    scorer, tp, E_gpu, g_gpu = _gpu(sc, poses[:16])
    x = tp.clone().requires_grad_(True)
    E = scorer(x)
    w = torch.linspace(0.5, 1.5, 16, device=x.device)
    (E * w).sum().backward()
    torch.cuda.synchronize()
    assert np.allclose(E.detach().cpu().numpy(), E_gpu, rtol=0, atol=0)
    expect = g_gpu * w.cpu().numpy()[:, None]
    assert np.allclose(x.grad.cpu().numpy(), expect, rtol=1e-6, atol=1e-6)


def test_gradient_descends_and_respects_limits(scene):
    """A small step against the gradient lowers E_s; parameters outside their
    limits get no gradient."""
    sc, poses = scene
    scorer, tp, E0, g = _gpu(sc, poses[:32])
    scale = torch.from_numpy(I.perturbation_scale().astype(np.float32)).cuda()
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    step = scale * scale * gt
    step = step / (step.norm(dim=1, keepdim=True) / scale.norm() + 1e-12) * 1e-3
    E1 = scorer.forward(tp - step).cpu().numpy()
    assert (E1 < E0).mean() >= 0.9
    out = tp[:4].clone()
    out[:, 13] = sc.model_o.hi[13] + 0.3
    scorer.forward(out)
    g_out = scorer.gradient(out).cpu().numpy()
    assert np.all(g_out[:, 13] == 0.0)


def test_polish_select_and_keep_better():
    dev = torch.device("cuda")
    E = torch.tensor([5.0, 1.0, 3.0, 1.0, float("nan"), 0.5, 7.0, 3.0], device=dev)
    sel = torch.zeros(5, dtype=torch.int32, device=dev)
    hs.polish_select(E, 5, sel)
    torch.cuda.synchronize()
    assert sel.cpu().tolist() == [5, 1, 3, 2, 7]  # ascending, lower index on ties, NaN last
    x = torch.arange(8 * 26, dtype=torch.float32, device=dev).reshape(8, 26)
    x_sel = torch.zeros(5, 26, device=dev)
    E_sel = torch.zeros(5, device=dev)
    hs.polish_gather(x, E, sel, x_sel, E_sel)
    torch.cuda.synchronize()
    assert torch.equal(x_sel, x[sel.long()]) and torch.equal(E_sel, E[sel.long()])
    x_new = x_sel + 100.0
    E_new = torch.tensor([0.4, 2.0, 0.9, float("nan"), 2.5], device=dev)  # better, worse, better, nan, better
    hs.polish_keep_better(x, E, sel, x_new, E_sel, E_new)
    torch.cuda.synchronize()
    Ec = E.cpu().numpy()
    assert Ec[5] == np.float32(0.4) and Ec[1] == 1.0 and Ec[3] == np.float32(0.9) and Ec[2] == 3.0
    assert Ec[7] == np.float32(2.5)
    assert torch.equal(x[5], x_new[0]) and torch.equal(x[3], x_new[2]) and torch.equal(x[1], x_sel[1])


def test_hybrid_polish_never_raises_E_and_tracks(scene):
    """One frame of the hybrid (k = 8, 5 polish steps): after every polish the
    objectives are elementwise no larger than before it; gbest_E ends below the
    starting pose's E; graph replay equals eager execution."""
    from paper_2005_07068_b300 import tracker as T
    sc, poses = scene
    dev = torch.device("cuda")
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    cam = hs.camera(*[float(v) for v in sc.cam])
    start = torch.from_numpy(poses[3]).to(dev)

    class Probe(T.HybridTracker):
        def _after_render(self, o, x):
            before = self.swarm.E.clone()
            super()._after_render(o, x)
            self.checks.append((before, self.swarm.E.clone()))

    tr = Probe(sc.model_g, cam, P=64, gens=8, seed=11, device=dev)
    tr.checks = []
    tr.run_frame(obs, 0, start, graph=False)
    torch.cuda.synchronize()
    for before, after in tr.checks:
        b, a = before.cpu().numpy(), after.cpu().numpy()
        assert np.all(a <= b)
    assert any(np.any(a.cpu().numpy() < b.cpu().numpy()) for b, a in tr.checks)  # the polish did something
    eager = (tr.swarm.gbest.clone(), tr.swarm.gbest_E.clone())
    E_start = C.run_gpu(sc, debug=False, poses=poses[3:4]).E[0]
    assert float(eager[1][0]) < E_start
    tr2 = T.HybridTracker(sc.model_g, cam, P=64, gens=8, seed=11, device=dev)
    tr2.run_frame(obs, 0, start, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(tr2.swarm.gbest, eager[0]) and torch.equal(tr2.swarm.gbest_E, eager[1])
    REPORT["hybrid_frame_gbest_E"] = float(eager[1][0])
