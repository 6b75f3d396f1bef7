"""Pins of the oracle's smoothed objective E_s and its gradient (CPU).

E_s is the objective the gradient polish descends; its definition lives in
oracle/soft.py.  It is pinned here by things other than itself: the FK it
uses equals the C oracle's FK, its limit as the softness goes to zero is the
hard objective of the C oracle (coverage, depth, sums), and its complex-step
gradient equals FP64 central differences (h = 1e-4 rad / 1e-2 mm).
"""
import numpy as np
import pytest

import oracle
from oracle import soft
from paper_2005_07068_b300 import inputs as I


@pytest.fixture(scope="module")
def scene():
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    m = oracle.Model.from_geometry(g, lo, hi)
    W, H = 80, 60
    cam = oracle.camera_tuple(I.kinect_camera(W, H))
    cam[:2] *= 1.4
    gt = I.ground_truth_pose(7)
    depth, hit, _, _ = oracle.render_pose(m, gt, cam, W, H, boundary=False)
    Od, S = I.kinect_observation(depth, hit, 7)
    rng = np.random.default_rng(1)
    poses = [gt + s * rng.uniform(-1, 1, 26) * I.perturbation_scale() for s in (0.3, 0.6, 1.0)]
    # strictly inside the limits: at a limit the clamp makes central differences one-sided
    margin = np.where(np.arange(26) < 3, 1.0, 0.02)
    return m, cam, Od.astype(np.float64), S, [np.clip(p, lo + margin, hi - margin) for p in poses]


def test_fk_matches_c_oracle(scene):
    m, _, _, _, poses = scene
    rng = np.random.default_rng(2)
    lo, hi = I.search_limits()
    for p in list(poses) + list(I.sample_poses(rng, 5, lo - 0.1, hi + 0.1)):
        f = oracle.fk(m, p)
        q, pR, pC, kc = soft.fk(m, p)
        assert np.abs(pR - f["prim_R"]).max() < 1e-12
        assert np.abs(pC - f["prim_C"]).max() < 1e-9
        assert abs(kc - f["kc"]) < 1e-12
        assert np.array_equal(q, f["q"])


def test_zero_softness_limit_is_the_hard_objective(scene):
    m, cam, Od, S, poses = scene
    for p in poses:
        E, parts = soft.soft_objective(m, p, cam, Od, S, tau=1e-4, tau_mm=1e-4, return_parts=True)
        o = oracle.score_batch(m, p[None], cam, Od, S, per_pixel=True)
        hit = o["hit"][0]
        cov = np.real(parts["coverage"]) > 0.5
        assert (cov != hit).sum() <= 2  # at most a pixel or two exactly on a silhouette
        both = cov & hit & ~o["boundary"][0]
        assert np.abs(np.real(parts["depth"]) - o["depth"][0])[both].max() < 1e-3
        assert abs(E - o["E"][0]) <= 1e-3 * abs(o["E"][0]) + 1e-2
        assert abs(parts["sum_or"] - o["sums"][0, 2]) < 2.5
    # with the working softness only pixels near a silhouette differ from E's decisions
    E_s, parts = soft.soft_objective(m, poses[0], cam, Od, S, return_parts=True)
    o = oracle.score_batch(m, poses[0][None], cam, Od, S, per_pixel=True)
    cov = np.real(parts["coverage"])
    hit = o["hit"][0]
    from scipy.ndimage import binary_dilation, binary_erosion
    edge = binary_dilation(hit, iterations=6) & ~binary_erosion(hit, iterations=6)
    assert np.all(cov[hit & ~edge] > 0.95) and np.all(cov[~hit & ~edge] < 0.05)


def test_complex_step_gradient_equals_central_differences(scene):
    m, cam, Od, S, poses = scene
    for p in poses:
        gc = soft.soft_gradient(m, p, cam, Od, S)
        gf = soft.central_difference(m, p, cam, Od, S)
        scale = np.abs(gc).max()
        assert scale > 1.0
        assert np.abs(gc - gf).max() <= 2e-3 * scale, (np.abs(gc - gf).max(), scale)


def test_clamped_dof_has_zero_gradient(scene):
    m, cam, Od, S, poses = scene
    p = poses[0].copy()
    p[13] = m.hi[13] + 0.2   # beyond its limit: FK clamps it
    p[2] = m.lo[2] - 5.0      # the wrist depth too
    gc = soft.soft_gradient(m, p, cam, Od, S)
    assert gc[13] == 0.0 and gc[2] == 0.0
    assert np.abs(gc).max() > 0.1
