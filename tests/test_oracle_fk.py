"""Pins of the oracle's forward kinematics (Eq. 1-3, Section II.A).

Checked against properties the kinematic tree must have whatever the code:
orthonormal frames, preserved bone lengths, joint angles recovered from the
frames, rigid wrist motion, clamping to Tables 1-2, closed-form finger-tip
positions, and kc(h) on hand-worked angles.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_07068_b300 import inputs as I

G = I.hand_geometry()
LO, HI = I.search_limits()
MODEL = oracle.Model.from_geometry(G, LO, HI)
RNG = np.random.default_rng(1)
POSES = I.sample_poses(RNG, 20, LO, HI)


def _fk(pose):
    r = oracle.fk(MODEL, pose)
    assert r is not None
    return r


@pytest.mark.parametrize("i", range(5))
def test_frames_orthonormal(i):
    r = _fk(POSES[i])
    for R in list(r["bone_R"]) + list(r["prim_R"]):
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12
        assert abs(np.linalg.det(R) - 1.0) < 1e-12


@pytest.mark.parametrize("i", range(5))
def test_bone_lengths_preserved(i):
    r = _fk(POSES[i])
    for b in range(1, 16):
        parent = G.bones_i[b, 0]
        dist = np.linalg.norm(r["bone_p"][b] - r["bone_p"][parent])
        assert abs(dist - np.linalg.norm(G.bones_f[b, :3])) < 1e-9


@pytest.mark.parametrize("i", range(5))
def test_flexion_angles_recovered(i):
    """Between bone k and its child the y axes turn by exactly the PIP/DIP
    angle about the shared x axis."""
    q = _fk(POSES[i])["q"]
    r = _fk(POSES[i])
    for f in range(5):
        for j, dof in ((1, "PIP"), (2, "DIP")):
            b = 1 + 3 * f + j
            Rp, Rc = r["bone_R"][b - 1], r["bone_R"][b]
            assert np.abs(Rp[:, 0] - Rc[:, 0]).max() < 1e-12  # shared x axis
            cosang = float(np.clip(Rp[:, 1] @ Rc[:, 1], -1, 1))
            assert abs(math.acos(cosang) - abs(q[I.dof_index(I.FINGERS[f], dof)])) < 1e-7


def test_straight_and_bent_finger_closed_form():
    pose = np.zeros(26)
    pose[:3] = (0.0, 80.0, 520.0)
    r = _fk(pose)
    for f in range(1, 5):
        L = G.lengths[f]
        mcp = r["bone_p"][1 + 3 * f]
        tip_c = r["prim_C"][9 + 7 * (f - 1) + 6]  # tip sphere centre
        assert abs(np.linalg.norm(tip_c - mcp) - L.sum()) < 1e-9
    # PIP at 90 degrees, DIP straight: right triangle
    pose2 = pose.copy()
    pose2[I.dof_index("index", "PIP")] = math.pi / 2
    r2 = _fk(pose2)
    L = G.lengths[1]
    d = np.linalg.norm(r2["prim_C"][9 + 6] - r2["bone_p"][4])
    assert abs(d - math.hypot(L[0], L[1] + L[2])) < 1e-9


def test_rest_layout_closed_form():
    """Zero angles: the palm frame is the mount diag(1,-1,-1) and each finger
    points along its rest splay."""
    t = np.array([10.0, 90.0, 530.0])
    pose = np.zeros(26)
    pose[:3] = t
    r = _fk(pose)
    mount = np.diag([1.0, -1.0, -1.0])
    for f in range(1, 5):
        b = 1 + 3 * f
        off = G.bones_f[b, :3]
        assert np.abs(r["bone_p"][b] - (t + mount @ off)).max() < 1e-12
        a = G.bones_f[b, 5]  # rest rotation about z
        direction = mount @ np.array([-math.sin(a), math.cos(a), 0.0])
        tip = r["bone_p"][b] + G.lengths[f].sum() * direction
        assert np.abs(r["prim_C"][9 + 7 * (f - 1) + 6] - tip).max() < 1e-9


def test_translation_equivariance():
    p = POSES[0].copy()
    r0 = _fk(p)
    p[:3] += (3.0, -2.0, 4.0)
    r1 = _fk(p)
    assert np.abs(r1["prim_C"] - r0["prim_C"] - np.array([3.0, -2.0, 4.0])).max() < 1e-9
    assert np.abs(r1["prim_R"] - r0["prim_R"]).max() == 0.0


@pytest.mark.parametrize("i", range(4))
def test_wrist_rotation_is_rigid_about_the_wrist(i):
    p0 = POSES[i].copy()
    p1 = p0.copy()
    p1[3:6] = POSES[i + 5][3:6]
    c0 = _fk(p0)["prim_C"]
    c1 = _fk(p1)["prim_C"]
    d0 = np.linalg.norm(c0[:, None] - c0[None], axis=-1)
    d1 = np.linalg.norm(c1[:, None] - c1[None], axis=-1)
    assert np.abs(d0 - d1).max() < 1e-9
    w = p0[:3]
    assert np.abs(np.linalg.norm(c0 - w, axis=1) - np.linalg.norm(c1 - w, axis=1)).max() < 1e-9


def test_clamping_to_limits():
    p = POSES[1].copy()
    p[0] = 1e4
    p[7] = -3.0
    p[12] = 9.0
    r = _fk(p)
    q = r["q"]
    assert np.all(q >= LO) and np.all(q <= HI)
    assert q[0] == HI[0] and q[7] == LO[7] and q[12] == HI[12]
    r2 = _fk(np.clip(p, LO, HI))
    assert np.array_equal(r["prim_C"], r2["prim_C"])


def test_nonfinite_pose_rejected():
    p = POSES[2].copy()
    p[9] = np.nan
    assert oracle.fk(MODEL, p) is None
    p[9] = np.inf
    assert oracle.fk(MODEL, p) is None


def test_kc_hand_worked():
    q = np.zeros(26)
    # index, middle, ring, pinky abduction (rad)
    q[11], q[15], q[19], q[23] = -0.1, 0.05, -0.2, -0.1
    # phi(index,middle) = -0.15 -> 0.15; phi(middle,ring) = 0.25 -> 0;
    # phi(ring,pinky) = -0.1 -> 0.1; total 0.25
    assert abs(oracle.kc(q) - 0.25) < 1e-15
    q[11], q[15], q[19], q[23] = 0.2, 0.1, 0.0, -0.3  # fanned out: no crossing
    assert oracle.kc(q) == 0.0
    q[6:10] = 5.0  # the thumb is not in any pair
    assert oracle.kc(q) == 0.0
