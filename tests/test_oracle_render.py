"""Pins of the oracle's depth rendering r_d (Section III.A; primitives of
Section II.A and Fig. 2).

Closed forms: silhouettes of a sphere / axis-aligned ellipsoid on the optical
axis are discs / ellipses whose pixel counts are lattice-point counts; a
side-on truncated cone has a closed-form front-surface depth; a cylinder seen
end-on shows its near cap at constant depth.  Brute force: a dense march along
each ray with an implicit inside-test (no ray-quadric algebra), refined by
bisection, on 8x8 ROIs of the full hand.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_07068_b300 import inputs as I

EYE = np.eye(3)


def _single(kind, dims, R, C, cam, W, H):
    pi = np.array([[0, kind]], np.int32)
    pf = np.array([[0.0, 0.0, 0.0, *dims]])
    return oracle.render(pi, pf, np.asarray(R, float)[None], np.asarray(C, float)[None], cam, W, H)


def _lattice_ellipse(W, H, cx, cy, ru, rv):
    u = np.arange(W) + 0.5 - cx
    v = np.arange(H) + 0.5 - cy
    q = (u[None, :] / ru) ** 2 + (v[:, None] / rv) ** 2
    assert np.abs(q - 1.0).min() > 1e-6  # no lattice point on the boundary
    return int((q <= 1.0).sum())


@pytest.mark.parametrize("z0,r,f", [(500.0, 40.0, 500.0), (620.0, 25.0, 700.0), (450.0, 9.0, 2100.0)])
def test_sphere_silhouette_is_lattice_disc(z0, r, f):
    W = H = 128
    cam = np.array([f, f, 64.0, 64.0])
    depth, hit, _, _ = _single(0, (r, r, r, 0.0), EYE, (0.0, 0.0, z0), cam, W, H)
    R = f * r / math.sqrt(z0 * z0 - r * r)
    assert hit.sum() == _lattice_ellipse(W, H, 64.0, 64.0, R, R)
    assert depth[hit].min() >= z0 - r - 1e-9 and depth[hit].max() <= z0 + 1e-9
    # every hit point lies on the sphere, where the ray enters it
    v, u = np.nonzero(hit)
    d = np.stack([(u + 0.5 - 64.0) / f, (v + 0.5 - 64.0) / f, np.ones(len(u))], axis=1)
    p = depth[v, u][:, None] * d - np.array([0.0, 0.0, z0])
    assert np.abs(np.linalg.norm(p, axis=1) - r).max() < 1e-9
    assert np.all((p * d).sum(axis=1) < 0.0)


@pytest.mark.parametrize("axes,z0,f", [((30.0, 15.0, 20.0), 500.0, 600.0), ((12.0, 40.0, 9.0), 560.0, 800.0)])
def test_axis_aligned_ellipsoid_silhouette(axes, z0, f):
    a, b, c = axes
    W = H = 128
    cam = np.array([f, f, 64.0, 64.0])
    depth, hit, _, _ = _single(0, (a, b, c, 0.0), EYE, (0.0, 0.0, z0), cam, W, H)
    k = math.sqrt(z0 * z0 - c * c)
    assert hit.sum() == _lattice_ellipse(W, H, 64.0, 64.0, f * a / k, f * b / k)


@pytest.mark.parametrize("kappa", [0.0, 0.12, -0.2])
def test_side_on_cone_front_depth(kappa):
    """Cone axis along camera x through (0, 0, z0): on the image row through the
    axis the first hit is the front of the side surface,
    t = (z0 - rm) / (1 + rm kappa a / hl), a = (u + 0.5 - cx) / f."""
    z0, rm, hl, f = 520.0, 10.0, 30.0, 900.0
    W, H = 160, 64
    cam = np.array([f, f, 80.0, 32.5])  # row 32 passes through the axis
    R = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, -1.0]])  # local y -> camera x
    depth, hit, _, _ = _single(1, (rm, rm, hl, kappa), R, (0.0, 0.0, z0), cam, W, H)
    for u in range(40, 121):
        a = (u + 0.5 - 80.0) / f
        t = (z0 - rm) / (1.0 + rm * kappa * a / hl)
        assert abs(t * a) < hl - 2.0
        assert hit[32, u] and abs(depth[32, u] - t) < 1e-9
    if kappa == 0.0:  # cylinder: rows hit in the middle column
        rows = hit[:, 80].sum()
        lim = rm / math.sqrt(z0 * z0 - rm * rm) * f
        vv = np.arange(H) + 0.5 - 32.5
        assert rows == int((np.abs(vv) <= lim).sum())


def test_end_on_cylinder_shows_near_cap():
    z0, r, hl, f = 560.0, 12.0, 25.0, 800.0
    W = H = 64
    cam = np.array([f, f, 32.0, 32.0])
    R = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])  # local y -> camera z
    pi = np.array([[0, 1]], np.int32)
    pf = np.array([[0.0, 0.0, 0.0, r, r, hl, 0.0]])
    depth, hit, _, _ = oracle.render(pi, pf, R[None], np.array([[0.0, 0.0, z0]]), cam, W, H)
    rad = f * r / (z0 - hl)
    assert hit.sum() == _lattice_ellipse(W, H, 32.0, 32.0, rad, rad)
    assert np.abs(depth[hit] - (z0 - hl)).max() < 1e-9
    t, surf = oracle.intersect(1, (r, r, hl, 0.0), R, (0.0, 0.0, z0), (0.0, 0.0, 1.0))
    assert surf == 1 and abs(t - (z0 - hl)) < 1e-12


# ---- brute force on 8x8 ROIs of the whole hand ----------------------------

def _inside(pts, kinds, dims, R, C):
    """pts [N,3] camera points -> bool [N] inside any primitive (implicit test)."""
    inside = np.zeros(len(pts), bool)
    for k in range(len(kinds)):
        loc = (pts - C[k]) @ R[k]  # R^T (p - C), row vectors
        if kinds[k] == 0:
            s = (loc[:, 0] / dims[k, 0]) ** 2 + (loc[:, 1] / dims[k, 1]) ** 2 + (loc[:, 2] / dims[k, 2]) ** 2
            inside |= s <= 1.0
        else:
            ax, az, hl, kap = dims[k]
            w = 1.0 + kap * loc[:, 1] / hl
            s = (loc[:, 0] / ax) ** 2 + (loc[:, 2] / az) ** 2
            inside |= (np.abs(loc[:, 1]) <= hl) & (s <= w * w)
    return inside


def _march(d, kinds, dims, R, C, t0=350.0, t1=760.0, dt=0.02):
    ts = np.arange(t0, t1, dt)
    ins = _inside(ts[:, None] * d[None, :], kinds, dims, R, C)
    if not ins.any():
        return 0.0
    j = int(np.argmax(ins))
    assert j > 0
    a, b = ts[j - 1], ts[j]
    for _ in range(60):
        m = 0.5 * (a + b)
        if _inside((m * d)[None, :], kinds, dims, R, C)[0]:
            b = m
        else:
            a = m
    return b


@pytest.mark.parametrize("seed,cam", [(11, (20.0, 20.0, 4.0, 4.0)), (12, (20.0, 20.0, 4.0, 4.0)),
                                      (13, (180.0, 180.0, 4.0, 4.0))])
def test_hand_8x8_brute_force(seed, cam):
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    model = oracle.Model.from_geometry(g, lo, hi)
    pose = I.ground_truth_pose(seed)
    cam = np.array(cam)
    f = oracle.fk(model, pose)
    if cam[0] > 100:  # zoom onto the palm centre
        c = f["prim_C"][0]
        cam[2] = 4.0 - cam[0] * c[0] / c[2]
        cam[3] = 4.0 - cam[1] * c[1] / c[2]
    depth, hit, _, bnd = oracle.render(model.prims_i, model.prims_f, f["prim_R"], f["prim_C"], cam, 8, 8)
    kinds = model.prims_i[:, 1]
    dims = model.prims_f[:, 3:]
    n_hit = 0
    for v in range(8):
        for u in range(8):
            if bnd[v, u]:
                continue
            d = np.array([(u + 0.5 - cam[2]) / cam[0], (v + 0.5 - cam[3]) / cam[1], 1.0])
            tb = _march(d, kinds, dims, f["prim_R"], f["prim_C"])
            assert (tb > 0) == hit[v, u], (u, v)
            if hit[v, u]:
                n_hit += 1
                assert abs(tb - depth[v, u]) < 1e-6, (u, v, tb, depth[v, u])
    assert n_hit >= 4
