"""Seeded input generators and the oracle's end-to-end tracking behaviour.

The geometry follows Section II.A / Fig. 2 (37 primitives, bone lengths in
[20, 90] mm); trajectories move at most 5 deg / 5 mm per frame; the Kinect
corruption hits its stated fractions exactly.  The oracle's plain PSO lowers
the objective over the generations (Fig. 7, Section V.A) on a tiny frame.
"""
import math

import numpy as np

import oracle
from paper_2005_07068_b300 import inputs as I


def test_geometry_counts_and_lengths():
    g = I.hand_geometry()
    assert g.bones_i.shape == (16, 3) and g.prims_i.shape == (37, 2)
    kinds = g.prims_i[:, 1]
    assert (kinds == I.PRIM_ECONE).sum() == 1 + 2 + 4 * 3  # palm + thumb 2 + fingers 3 each
    assert (kinds == I.PRIM_ELLIPSOID).sum() == 2 + 1 + 3 + 4 * 4
    assert np.all(g.lengths >= 20.0) and np.all(g.lengths <= 90.0)
    assert 20.0 <= g.palm_length <= 90.0
    for b in range(1, 16):
        assert 0 <= g.bones_i[b, 0] < b
    econe = g.prims_f[kinds == I.PRIM_ECONE]
    assert np.all(np.abs(econe[:, 6]) < 1.0) and np.all(econe[:, 3:6] > 0)
    assert I.hand_geometry().prims_f.tobytes() == g.prims_f.tobytes()  # seeded


def test_trajectory_step_bounds():
    tr = I.trajectory(I.CONFIG_SEED_BASE + 2, 30)
    lo, hi = I.search_limits()
    assert tr.shape == (30, 26)
    assert np.all(tr >= lo) and np.all(tr <= hi)
    step = np.abs(np.diff(tr, axis=0))
    assert step[:, :3].max() <= 5.0 + 1e-9
    assert step[:, 3:].max() <= math.radians(5.0) + 1e-12
    assert step.max() > 0


def test_kinect_corruption_fractions():
    H, W = 240, 320
    depth = np.full((H, W), 520.0)
    hit = np.zeros((H, W), bool)
    hit[60:180, 100:220] = True
    d, s = I.kinect_observation(depth, hit, 5)
    assert d.dtype == np.uint16 and s.dtype == np.uint8
    assert (d == 0).sum() >= round(0.05 * H * W) - 5  # the holes (noise never reaches 0)
    flips = (s != hit.astype(np.uint8)).sum()
    assert flips == round(0.02 * H * W)
    bg = ~hit & (d > 0)
    assert abs(float(d[bg].mean()) - 600.0) < 0.5 and 2.0 < float(d[bg].std()) < 4.0


def test_pitched_rows():
    img = np.arange(15, dtype=np.uint16).reshape(3, 5)
    p = I.pitched(img)
    assert p.shape == (3, 8) and np.array_equal(p[:, :5], img)
    assert I.pitched(np.zeros((2, 17), np.uint8)).shape == (2, 32)


def test_oracle_tracking_lowers_cost():
    """Plain PSO, 16 particles x 10 generations on a 64x64 clean frame."""
    W = H = 64
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    model = oracle.Model.from_geometry(g, lo, hi)
    cam = I.kinect_camera(W, H)
    gt = I.ground_truth_pose(I.CONFIG_SEED_BASE + 1)
    depth, hit, _, _ = oracle.render_pose(model, gt, oracle.camera_tuple(cam), W, H, boundary=False)
    Od, S = I.clean_observation(depth, hit)
    rng = np.random.default_rng(0)
    start = np.clip(gt + rng.uniform(-1, 1, 26) * I.perturbation_scale(), lo, hi)
    sw, hist = oracle.track_frame(model, cam, Od.astype(np.float64), S, start, I.perturbation_scale(),
                                  16, 10, 1234, 0)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < hist[0]
