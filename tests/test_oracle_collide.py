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
