"""Pins of the oracle's interpenetration test and kc variants (the reading of
the kc term of Eq. 5, Section III.A, that tests fingers passing through each
other directly).

Checked against what the definition fixes independently of the code: the
overlap depth of two spheres in closed form and by sampling their common
volume, that every proxy sphere lies inside its primitive (the primitive's own
implicit inequality), the finger numbering of the kinematic tree, invariance
under rigid motion of the hand, monotone growth as one finger is swung into
its neighbour, and the paper's kc for variant 0."""
import math

import numpy as np
import pytest

import oracle
from oracle import collide as K
from paper_2005_07068_b300 import inputs as I

G = I.hand_geometry()
LO, HI = I.search_limits()
MODEL = oracle.Model.from_geometry(G, LO, HI)
RNG = np.random.default_rng(7)
POSES = I.sample_poses(RNG, 12, LO, HI)


def test_two_spheres_closed_form():
    C = np.array([[0.0, 0.0, 0.0], [6.0, 0.0, 0.0]])
    assert K.penetration_of(C, np.array([5.0, 3.0]), np.array([0, 1])) == pytest.approx(2.0, abs=1e-15)
    # apart, same finger, or on the palm: nothing
    assert K.penetration_of(C, np.array([2.0, 3.0]), np.array([0, 1])) == 0.0
    assert K.penetration_of(C, np.array([5.0, 3.0]), np.array([1, 1])) == 0.0
    assert K.penetration_of(C, np.array([5.0, 3.0]), np.array([-1, 1])) == 0.0
    # three spheres: pairs add
    C3 = np.array([[0.0, 0.0, 0.0], [6.0, 0.0, 0.0], [0.0, 7.0, 0.0]])
    pen = K.penetration_of(C3, np.array([5.0, 3.0, 4.0]), np.array([0, 1, 2]))
    d13 = 7.0
    d23 = math.hypot(6.0, 7.0)
    assert pen == pytest.approx(2.0 + (5.0 + 4.0 - d13) + max(0.0, 3.0 + 4.0 - d23), abs=1e-12)


@pytest.mark.parametrize("d", [2.0, 5.0, 7.5, 8.5, 10.0])
def test_overlap_sign_by_sampling(d):
    """pen > 0 exactly when the two balls share volume (grid points in both)."""
    r1, r2 = 5.0, 3.0
    g = np.linspace(-6.0, 12.0, 181)
    X, Y, Z = np.meshgrid(g, np.linspace(-6, 6, 121), np.linspace(-6, 6, 121), indexing="ij")
    both = (X ** 2 + Y ** 2 + Z ** 2 < r1 ** 2) & ((X - d) ** 2 + Y ** 2 + Z ** 2 < r2 ** 2)
    pen = K.penetration_of(np.array([[0.0, 0, 0], [d, 0, 0]]), np.array([r1, r2]), np.array([0, 1]))
    assert (pen > 0) == bool(both.any())
    if pen > 0.5:  # the overlap along the centre line has length pen
        on_line = (g ** 2 < r1 ** 2) & ((g - d) ** 2 < r2 ** 2)
        step = g[1] - g[0]
        assert abs(on_line.sum() * step - pen) <= 2 * step


def test_fingers_of_the_tree():
    f = K.fingers(MODEL.bones_i)
    assert f[0] == -1
    assert list(f[1:]) == [i for i in range(5) for _ in range(3)]


def test_proxies_inside_their_primitives():
    """Every proxy sphere lies in its primitive's solid (local implicit form)."""
    fk = oracle.fk(MODEL, POSES[0])
    C, r, f, fixed = K.proxies(MODEL, fk)
    n_ell = int((MODEL.prims_i[:, 1] == K.PRIM_ELLIPSOID).sum())
    n_cone = MODEL.np_ - n_ell
    assert len(r) == n_ell + 3 * n_cone
    dirs = RNG.normal(size=(200, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    i = 0
    for k in range(MODEL.np_):
        kind = int(MODEL.prims_i[k, 1])
        d = MODEL.prims_f[k, 3:]
        R, c = fk["prim_R"][k], fk["prim_C"][k]
        for _ in range(1 if kind == K.PRIM_ELLIPSOID else 3):
            pts = C[i] + 0.999 * r[i] * dirs
            loc = (pts - c) @ R  # local coordinates
            if kind == K.PRIM_ELLIPSOID:
                val = (loc[:, 0] / d[0]) ** 2 + (loc[:, 1] / d[1]) ** 2 + (loc[:, 2] / d[2]) ** 2
                assert val.max() <= 1.0
            else:
                ax, az, hl, kap = d
                y = loc[:, 1]
                s = 1.0 + kap * y / hl
                assert np.abs(y).max() <= hl
                assert ((loc[:, 0] / (ax * s)) ** 2 + (loc[:, 2] / (az * s)) ** 2).max() <= 1.0
            i += 1


def test_knuckles_fixed_to_the_palm_are_left_out():
    """The proxies centred at the finger roots' origins keep their mutual
    distances in every pose (checked), and their pairs are left out: straight,
    spread fingers do not penetrate."""
    lo, hi = LO.copy(), HI.copy()
    C0 = None
    for p in POSES[:4]:
        C, r, f, fixed = K.proxies(MODEL, oracle.fk(MODEL, p))
        assert fixed.sum() == 4  # the knuckle spheres of index to pinky (the thumb has no root sphere)
        D = np.linalg.norm(C[fixed][:, None] - C[fixed][None], axis=2)
        if C0 is not None:
            assert np.abs(D - C0).max() < 1e-9
        C0 = D
    p = POSES[0].copy()
    p[6:] = 0.0
    p[[11, 15, 19, 23]] = [math.radians(15), 0.0, math.radians(-15), math.radians(-25)]
    assert K.penetration(MODEL, p) == 0.0


@pytest.mark.parametrize("i", range(4))
def test_rigid_motion_invariance(i):
    p = POSES[i].copy()
    base = K.penetration(MODEL, p)
    q = p.copy()
    q[0:3] = (LO[0:3] + HI[0:3]) / 2 + np.array([7.0, -5.0, 3.0]) * 0.5
    q[3:6] = np.clip(p[3:6] + np.array([0.1, -0.2, 0.3]), LO[3:6], HI[3:6])
    assert K.penetration(MODEL, q) == pytest.approx(base, abs=1e-9)


def test_swinging_a_finger_into_its_neighbour():
    """Index abduction toward the middle finger (MCP_z of the index decreasing
    toward the ulnar side) never lowers the penetration, and past contact it
    rises; spreading the fingers apart removes it."""
    p = I.sample_poses(np.random.default_rng(3), 1, LO, HI)[0]
    p[6:] = 0.0  # straight fingers
    p[[11, 15, 19, 23]] = [math.radians(15), 0.0, math.radians(-15), math.radians(-25)]
    spread = K.penetration(MODEL, p)
    assert spread == 0.0
    vals = []
    for a in np.linspace(math.radians(15), math.radians(-15), 13):
        q = p.copy()
        q[11] = a
        vals.append(K.penetration(MODEL, q))
    assert all(b >= a - 1e-12 for a, b in zip(vals, vals[1:]))
    assert vals[-1] > vals[0] + 1.0
    assert spread == pytest.approx(vals[0])


@pytest.mark.parametrize("i", range(6))
def test_variants(i):
    p = POSES[i]
    k0 = oracle.kc(np.clip(p, LO, HI))
    pen = K.penetration(MODEL, p)
    assert K.kc_variant(MODEL, p, 0, 0.05) == pytest.approx(k0, abs=1e-15)
    assert K.kc_variant(MODEL, p, 2, 1.0) == pytest.approx(pen, abs=1e-12)
    assert K.kc_variant(MODEL, p, 1, 0.05) == pytest.approx(k0 + 0.05 * pen, abs=1e-12)


def _penetrating_pose(seed, swing):
    """Nearly straight fingers (every flexion 0.05 rad, strictly inside its
    limits, so that the clamp is not at a corner) with the index swung by
    `swing` rad toward the middle finger, the palm and wrist from a seeded
    sample: the index and middle proxies interpenetrate."""
    p = I.sample_poses(np.random.default_rng(seed), 1, LO, HI)[0]
    p[6:] = 0.05
    p[[11, 15, 19, 23]] = [swing, 0.0, math.radians(-15), math.radians(-25)]
    assert np.all(p > LO) and np.all(p < HI)
    return p


def _min_threshold_gap(p):
    """Smallest | r_i + r_j - d_ij | over the counted pairs: how far the pose
    is from a kink of pen (where one pair starts or stops touching)."""
    C, r, f, fixed = K.proxies(MODEL, oracle.fk(MODEL, p))
    gaps = [abs(r[i] + r[j] - np.linalg.norm(C[i] - C[j]))
            for i in range(len(r)) for j in range(i + 1, len(r))
            if f[i] >= 0 and f[j] >= 0 and f[i] != f[j] and not (fixed[i] and fixed[j])]
    return min(gaps)


@pytest.mark.parametrize("seed,swing", [(11, -0.12), (12, -0.18), (13, -0.24)])
def test_penetration_gradient_against_central_differences(seed, swing):
    """The complex-step gradient of kc + w pen (variant 1) against FP64 central
    differences of the real function (h = 1e-6), at poses away from any kink;
    the wrist translation does not move the proxies relative to each other, so
    its three components are zero."""
    p = _penetrating_pose(seed, swing)
    assert K.penetration(MODEL, p) > 0.5
    assert _min_threshold_gap(p) > 1e-3
    w = 0.05
    g = K.kc_variant_gradient(MODEL, p, 1, w)
    fd = np.zeros(26)
    for k in range(26):
        a, b = p.copy(), p.copy()
        a[k] += 1e-6
        b[k] -= 1e-6
        fd[k] = (K.kc_variant(MODEL, a, 1, w) - K.kc_variant(MODEL, b, 1, w)) / 2e-6
    assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(g).max()), np.abs(g - fd).max()
    assert np.all(g[:3] == 0.0)
    assert np.abs(g).max() > 0.01  # the term does move the fingers


def test_variant_gradients_reduce_to_the_abduction_ordering():
    """Variant 0's gradient is the abduction ordering's in closed form: for each
    pair (a, b) of adjacent non-thumb fingers with q_b > q_a, -1 on q_a and +1 on
    q_b; variant 2 carries no part of it."""
    p = POSES[1].copy()
    p[[11, 15, 19, 23]] = [-0.1, 0.05, -0.3, -0.1]  # (11,15) and (19,23) ordered the wrong way
    assert np.all(p > LO) and np.all(p < HI)
    g0 = K.kc_variant_gradient(MODEL, p, 0, 0.0)
    want = np.zeros(26)
    for a, b in ((11, 15), (15, 19), (19, 23)):
        if p[b] > p[a]:
            want[a] -= 1.0
            want[b] += 1.0
    assert np.array_equal(g0, want)
    g1 = K.kc_variant_gradient(MODEL, p, 1, 0.05)
    g2 = K.kc_variant_gradient(MODEL, p, 2, 0.05)
    assert np.abs(g1 - (g0 + g2)).max() <= 1e-12
