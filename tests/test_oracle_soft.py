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


# ---- single primitives at the working softness, against closed forms of their geometry ----
# A sphere of radius r centred on the optical axis at depth Z (rotation I) and a
# cylinder of radius r, half-length hl, lying along the camera x axis at depth Z.
# The closed forms below come from the geometry (the tangent cone of a sphere,
# the ray-cylinder intersection in the plane of the axis), not from the
# oracle's general ray-quadric expressions.

F_PX = 262.5
SPHERE_R, SPHERE_Z = 10.0, 500.0


def _sphere_terms(a, b, tau=soft.TAU_PX):
    dims = np.array([SPHERE_R, SPHERE_R, SPHERE_R, 0.0])
    return soft.primitive_terms(0, dims, np.eye(3), np.array([0.0, 0.0, SPHERE_Z]), np.asarray(a, float),
                                np.asarray(b, float), F_PX, F_PX, tau)


def _sphere_closed_form(a, b, tau):
    """Delta, |grad_pixel Delta| and the soft near root for the ray (a, b, 1),
    from |t e - C|^2 = r^2 with e = (a, b, 1): the quadratic |e|^2 t^2 - 2 Z t +
    Z^2 - r^2 = 0 scaled by 1 / r^2 has Delta = (Z^2 - |e|^2 (Z^2 - r^2)) / r^4."""
    r, Z = SPHERE_R, SPHERE_Z
    e2 = a * a + b * b + 1.0
    D = (Z * Z - e2 * (Z * Z - r * r)) / r ** 4
    N = 2.0 * np.hypot(a, b) * (Z * Z - r * r) / (r ** 4 * F_PX)  # d Delta / d(pixel) along the radius
    Dp = 0.5 * (D + np.sqrt(D * D + (tau * N) ** 2))
    t = ((Z * Z - r * r) / r ** 2) / (Z / r ** 2 + np.sqrt(Dp))
    return D, N, t


def test_sphere_silhouette_distance_and_soft_depth():
    """The silhouette of the sphere is the circle of radius f r / sqrt(Z^2 - r^2)
    pixels: there delta = 0 and delta falls by one per pixel outward (first-order
    signed distance); inside, Delta, its pixel gradient and the soft near root
    (the soft positive part of Delta in the root) equal the closed forms, and far
    inside the soft root is the exact near intersection."""
    r, Z = SPHERE_R, SPHERE_Z
    rho = F_PX * r / np.sqrt(Z * Z - r * r)  # silhouette radius, pixels
    eps = np.array([-0.5, -0.25, -1e-3, 0.0, 1e-3, 0.25, 0.5])  # pixels outward from the silhouette
    a = (rho + eps) / F_PX
    D, delta, t, ok, extra = _sphere_terms(a, np.zeros_like(a))
    assert extra is None
    assert abs(delta[3]) < 1e-9 * rho
    # first order: delta = -eps + O(eps^2 / rho)
    assert np.all(np.abs(delta + eps) <= 2.0 * eps * eps / rho + 1e-9)
    # inside, at several radii and directions: the closed forms
    for frac, ang in ((0.0, 0.0), (0.3, 0.7), (0.8, 2.0), (0.97, 4.0)):
        aa, bb = frac * rho / F_PX * np.cos(ang), frac * rho / F_PX * np.sin(ang)
        D, delta, t, ok, _ = _sphere_terms(np.array([aa]), np.array([bb]))
        Dc, Nc, tc = _sphere_closed_form(aa, bb, soft.TAU_PX)
        assert bool(ok[0])
        # (B^2 - A C cancels about four digits of its terms: relative 1e-9 is rounding)
        assert np.isclose(D[0], Dc, rtol=1e-9)
        if frac > 0:
            assert np.isclose(delta[0], Dc / Nc, rtol=1e-9)
        assert np.isclose(t[0], tc, rtol=1e-10)
    # well inside, the soft root is the exact near hit (|e|^2 t^2 - 2 Z t + Z^2 - r^2 = 0)
    aa = 0.3 * rho / F_PX
    _, _, t, _, _ = _sphere_terms(np.array([aa]), np.array([0.0]))
    e2 = aa * aa + 1.0
    t_exact = (Z - np.sqrt(Z * Z - e2 * (Z * Z - r * r))) / e2
    assert abs(t[0] - t_exact) < 1e-2  # mm: the soft positive part's share this far inside (4.5e-3 here)
    # at zero softness the root is exact to rounding
    _, _, t0, _, _ = _sphere_terms(np.array([aa]), np.array([0.0]), tau=0.0)
    assert np.isclose(t0[0], t_exact, rtol=1e-10)


def test_sphere_soft_root_at_the_silhouette():
    """On the silhouette Delta = 0, so the soft positive part is tau |grad Delta| / 2
    and the depth is the root with that in place of Delta: a closed form in tau."""
    r, Z = SPHERE_R, SPHERE_Z
    rho = F_PX * r / np.sqrt(Z * Z - r * r)
    for tau in (0.25, 0.5, 1.0):
        a = rho / F_PX
        _, _, t, _, _ = _sphere_terms(np.array([a]), np.array([0.0]), tau=tau)
        N = 2.0 * a * (Z * Z - r * r) / (r ** 4 * F_PX)
        t_c = ((Z * Z - r * r) / r ** 2) / (Z / r ** 2 + np.sqrt(0.5 * tau * N))
        assert np.isclose(t[0], t_c, rtol=1e-10), tau


def test_cylinder_end_cut_distance():
    """A cylinder (kappa = 0) along the camera x axis: for rays in the plane of
    its axis (b = 0) the near hit is at depth Z - r and its axial coordinate is
    Y = (Z - r) a / h_l, so the end cut's distance is (1 - |Y|) L pixels with L
    the projected half-length f h_l / Z; it is zero where the ray meets the end
    of the front surface, a = h_l / (Z - r)."""
    r, hl, Z = 8.0, 30.0, 450.0
    R = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, -1.0]])  # local y (the axis) along camera x
    dims = np.array([r, r, hl, 0.0])
    a_end = hl / (Z - r)
    a = np.array([0.0, 0.25, 0.5, 0.9, 1.0, 1.02]) * a_end
    D, delta, t, ok, (delta_y, fade) = soft.primitive_terms(1, dims, R, np.array([0.0, 0.0, Z]), a,
                                                            np.zeros_like(a), F_PX, F_PX, soft.TAU_PX)
    L = F_PX * hl / Z
    assert np.allclose(t, Z - r, rtol=1e-13)
    assert np.allclose(delta_y, (1.0 - (Z - r) * np.abs(a) / hl) * L, rtol=1e-10, atol=1e-9)
    assert abs(delta_y[4]) < 1e-9
    # the fade by the angle to a surface generator: the axial ray (a = 0) is perpendicular to the
    # generators, sin^2 = 1, which leaves 1 / (1 + (0.06 tau)^4); the others are within 1e-6 of it
    assert np.isclose(fade[0], 1.0 / (1.0 + (0.06 * soft.TAU_PX) ** 4), rtol=1e-14)
    assert np.all(np.abs(fade - fade[0]) < 1e-6)
