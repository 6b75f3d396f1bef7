"""Pins of the oracle's objective (Section III.A, Eq. 4-5).

Hand-worked 3x3 cases for every branch of the per-pixel rule, the exact
identity of the area term with one minus the Dice coefficient (checked with
scipy's Dice dissimilarity), D = 0 for the noise-free observation of the same
pose, invariance under permutations of background-only pixels, monotonicity
in an added unrendered skin pixel, and the empty-union convention.
"""
import numpy as np
import pytest
from scipy.spatial.distance import dice

import oracle
from paper_2005_07068_b300 import inputs as I
from tests.conftest import golden_path

G = I.hand_geometry()
LO, HI = I.search_limits()
MODEL = oracle.Model.from_geometry(G, LO, HI)
LAM = oracle.DEFAULT_PARAMS[2]


def _cases():
    cases, cur = {}, None
    with open(golden_path("cost_3x3_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "case":
                cur = cases.setdefault(line[1], {})
            else:
                cur[line[0]] = np.array([float(x) for x in line[1:]])
    return cases


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_hand_worked_3x3(name):
    c = CASES[name]
    D, sums, _ = oracle.cost(c["depth"].reshape(3, 3), c["hit"].reshape(3, 3) > 0, c["Od"].reshape(3, 3),
                             c["S"].reshape(3, 3) > 0)
    assert np.array_equal(sums, c["sums"])
    assert D == c["D"][0]


def _scene(seed, W=48, H=40):
    pose = I.ground_truth_pose(seed)
    cam = oracle.camera_tuple(I.kinect_camera(W, H))
    cam[0] = cam[1] = 3.0 * cam[0]  # zoom so the hand fills the ROI
    depth, hit, _, _ = oracle.render_pose(MODEL, pose, cam, W, H, boundary=False)
    return pose, cam, depth, hit


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_cost_zero_at_ground_truth(seed):
    pose, cam, depth, hit = _scene(seed)
    assert hit.sum() > 50
    Od, S = np.where(hit, depth, 0.0), hit.astype(np.uint8)  # exact FP64 render
    r = oracle.score_batch(MODEL, pose[None], cam, Od, S)
    assert r["D"][0] == 0.0
    assert r["E"][0] == oracle.DEFAULT_PARAMS[3] * oracle.kc(np.clip(pose, LO, HI))
    # a perturbed pose scores worse
    p2 = pose.copy()
    p2[0] += 6.0
    r2 = oracle.score_batch(MODEL, p2[None], cam, Od, S)
    assert r2["D"][0] > 0.5


@pytest.mark.parametrize("seed", [6, 7])
def test_area_term_is_one_minus_dice(seed):
    pose, cam, depth, hit = _scene(seed)
    Od, S = I.kinect_observation(depth, hit, seed, plane_mm=600.0)
    p2 = pose.copy()
    p2[3] += 0.05
    d2, h2, _, _ = oracle.render_pose(MODEL, p2, cam, 48, 40, boundary=False)
    D, sums, rm = oracle.cost(d2, h2, Od.astype(np.float64), S)
    area = D - sums[0] / sums[2]
    assert abs(area - LAM * dice(S.ravel() > 0, rm.ravel())) < 1e-12
    # and the union identity: sum(and) + sum(or) = |S| + |r_m|
    assert sums[1] + sums[2] == (S > 0).sum() + rm.sum()


def test_background_permutation_invariance():
    pose, cam, depth, hit = _scene(8)
    Od, S = I.kinect_observation(depth, hit, 8, plane_mm=600.0)
    poses = np.stack([pose, pose + np.r_[4.0, -3.0, 2.0, np.zeros(23)]])
    ref = oracle.score_batch(MODEL, poses, cam, Od.astype(np.float64), S, per_pixel=True)
    bg = (~ref["hit"].any(axis=0)) & (S == 0)
    idx = np.flatnonzero(bg.ravel())
    assert len(idx) > 100
    rng = np.random.default_rng(0)
    Od2, S2 = Od.copy().ravel(), S.copy().ravel()
    perm = rng.permutation(idx)
    Od2[idx] = Od2[perm]
    S2[idx] = S2[perm]
    out = oracle.score_batch(MODEL, poses, cam, Od2.reshape(Od.shape).astype(np.float64), S2.reshape(S.shape))
    assert np.array_equal(out["E"], ref["E"])


def test_unrendered_skin_pixel_monotone():
    pose, cam, depth, hit = _scene(9)
    Od, S = I.clean_observation(depth, hit)
    D0, s0, _ = oracle.cost(depth, hit, Od.astype(np.float64), S)
    v, u = np.argwhere(~hit)[0]
    S2 = S.copy()
    Od2 = Od.astype(np.float64).copy()
    S2[v, u] = 1
    Od2[v, u] = 555.0
    D1, s1, _ = oracle.cost(depth, hit, Od2, S2)
    assert s1[0] == s0[0] + oracle.DEFAULT_PARAMS[1]
    assert s1[1] == s0[1] and s1[2] == s0[2] + 1
    assert D1 > D0


def test_objective_adds_lambda_k_kc():
    pose, cam, depth, hit = _scene(10)
    Od, S = I.clean_observation(depth, hit)
    p = pose.copy()
    p[11], p[15] = -0.2, 0.1  # index crosses the middle finger by 0.3 rad
    p = np.clip(p, LO, HI)
    r = oracle.score_batch(MODEL, p[None], cam, Od.astype(np.float64), S)
    assert abs(r["kc"][0] - oracle.kc(p)) == 0.0 and r["kc"][0] >= 0.3 - 1e-12
    assert r["E"][0] == r["D"][0] + oracle.DEFAULT_PARAMS[3] * r["kc"][0]
