"""Smoothed objective E_s and its gradient, FP64 (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path).  It shares no code with the CUDA path.

The hard objective E (Eq. 4-5, Section III.A) is piecewise constant in the
pose wherever a pixel changes state at a silhouette or a depth threshold, so
its gradient carries no silhouette information and finite differences of it
are meaningless.  E_s replaces each hard decision by a smooth one and
otherwise follows E term by term (reading R1):

* coverage of pixel p by primitive j: sigma(delta_j / tau), where delta_j is
  the signed distance in pixels to j's silhouette, taken to first order from
  the ray-quadric discriminant Delta_j: delta_j = Delta_j / |grad_pixel Delta_j|
  (positive inside); union coverage c = 1 - prod_j (1 - sigma_j);
* depth: the near root of the ray-quadric equation A t^2 + 2 B t + C = 0
  (t the camera-ray parameter, = depth), written as t = C / (-B + sqrt(Delta+))
  with the soft positive part Delta+ = (Delta + sqrt(Delta^2 +
  (tau |grad Delta|)^2)) / 2 in place of max(Delta, 0), so that the depth is
  smooth across the silhouette (the exact root has an infinite slope there).
  With Delta+ = Delta this is the near root; unlike (-B - sqrt(Delta+)) / A it
  stays bounded as A -> 0 (a ray nearly parallel to a cone's surface).  A
  visible near root needs A > 0 and B < 0, which the primitive must satisfy.
  The depth's offset s = t - t0 from the primitive's centre depth t0 is then
  clamped smoothly to its bounding radius R (largest semi-axis, or for a cone
  the half-diagonal sqrt(h_l^2 + r_max^2)): identity for |s| <= R, and
  sign(s) R (2 - exp(1 - |s| / R)) beyond (C1, at most 2R).  A real hit is
  never clamped; near-miss rays of a cone seen nearly end-on otherwise get
  depths metres away.  The cone's end cut below uses the same clamped
  offsets (of the root and of the closest approach);
  a cone's coverage is further multiplied by sigma(delta_Y / tau), its end
  cut |Y| <= 1 softened with delta_Y = (1 - |Y_e|) L pixels.  L is the
  projected half-length of the axis in pixels (the distance between the
  projections of C - h_l y and C + h_l y, over two), at least the cone's
  largest radius in pixels at its centre depth.  Y_e = Y* + w (Y_root - Y*)
  blends the axial coordinate of the root (exact, but ill-conditioned near a
  grazing silhouette, where the root slides along the ray as 1 / A) with
  that of the ray's closest approach to the axis, t* = -B/A (smooth there),
  by w = sigma(delta / tau - 2): the root well inside the silhouette, the
  closest approach near and outside it; both at their clamped offsets.
  A cone seen within a few degrees of a surface generator fades out: with
  a = A / |h|^2 (the squared sine of that angle) its coverage is also
  multiplied by a^4 / (a^4 + a0^4), a0 = 0.06 tau (tau in pixels; at
  tau = 0.5: half at ~10 degrees, 1e-6 at ~2, and no fade as tau -> 0).
  There every quantity above is ill-conditioned (the quadratic degenerates,
  A -> 0), and the joint sphere at the cone's near end hides all of it but a
  thin crescent.  Cone caps are not part of E_s (the
  model's joint spheres cover every cone end);
* soft nearest surface: the primitives are composited front to back in order
  of depth, alpha_j = sigma_j, T_j = prod over nearer k of (1 - alpha_k),
  z~ = sum_j T_j alpha_j z_j / c (c = sum_j T_j alpha_j); continuous where two
  surfaces swap order, since they do so at equal depth;
* the depth difference |O_d - z~| becomes the soft absolute value
  sqrt((O_d - z~)^2 + tau_mm^2), the d_M clamp a soft minimum and the r_m
  threshold a sigmoid, all of width tau_mm;
* per pixel, with valid = S and O_d > 0:
  t_hit = valid ? smin(diff, d_M) : (S ? 0 : d_M),  t_miss = valid ? d_M : 0,
  t = c t_hit + (1 - c) t_miss,  r_m = c (valid ? sigmoid((d_m - diff)/tau_mm) : 1),
  sum_and += S r_m,  sum_or += S + (1 - S) r_m;
* D_s = sum_t / sum_or + lambda (1 - 2 sum_and / (sum_and + sum_or)),
  E_s = D_s + lambda_k kc(h) (Eq. 4-5; kc keeps its hinge).

As tau and tau_mm -> 0, E_s -> E.  The gradient is obtained by the
complex step, dE/dx_k = Im E_s(x + i h e_k) / h with h = 1e-30, which is
exact to rounding for the analytic functions used here (every branch is
decided on real parts).  Pinned in tests by FP64 central differences and by
the tau -> 0 limit against the hard oracle.
"""
from __future__ import annotations

import numpy as np

from .oracle import DEFAULT_PARAMS, Model

TAU_PX = 0.5     # silhouette softness, pixels
TAU_MM = 0.5     # softness of the d_M clamp and of the d_m test, mm
MOUNT = np.diag([1.0, -1.0, -1.0])


def _re(x):
    return np.real(x)


def _rot_x(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[1, 0 * c, 0 * c], [0 * c, c, -s], [0 * c, s, c]])


def _rot_y(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, 0 * c, s], [0 * c, 1 + 0 * c, 0 * c], [-s, 0 * c, c]])


def _rot_z(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s, 0 * c], [s, c, 0 * c], [0 * c, 0 * c, 1 + 0 * c]])


def fk(model: Model, pose):
    """Forward kinematics (Eq. 1-3, Section II.A; Tables 1-2) on real or complex
    poses: clamp (decided on the real part), palm Mount Rz Ry Rx at the wrist,
    bone b = parent T(offset) Rest Rz(q_dz) Rx(q_dx), primitive frames.
    Returns (q, prim_R [np, 3, 3], prim_C [np, 3], kc)."""
    pose = np.asarray(pose)
    lo, hi = model.lo, model.hi
    q = np.where(_re(pose) < lo, lo, np.where(_re(pose) > hi, hi, pose))
    nb = model.bones_i.shape[0]
    R = [None] * nb
    O = [None] * nb
    R[0] = MOUNT @ _rot_z(q[5]) @ _rot_y(q[4]) @ _rot_x(q[3])
    O[0] = np.array([q[0], q[1], q[2]])
    for k in range(1, nb):
        parent, dz, dx = (int(v) for v in model.bones_i[k])
        f = model.bones_f[k]
        O[k] = O[parent] + R[parent] @ f[:3]
        rest = _rot_z(f[5]) @ _rot_y(f[4]) @ _rot_x(f[3])
        R[k] = R[parent] @ rest @ _rot_z(q[dz] if dz >= 0 else 0.0) @ _rot_x(q[dx] if dx >= 0 else 0.0)
    npr = model.prims_i.shape[0]
    pR = np.array([R[int(model.prims_i[j, 0])] for j in range(npr)])
    pC = np.array([R[int(model.prims_i[j, 0])] @ model.prims_f[j, :3] + O[int(model.prims_i[j, 0])]
                   for j in range(npr)])
    kc = 0.0
    for a, b in ((11, 15), (15, 19), (19, 23)):  # -min(phi, 0) over adjacent non-thumb fingers
        phi = q[a] - q[b]
        kc = kc + (-phi if _re(phi) < 0 else 0.0)
    return q, pR, pC, kc


def _sigmoid(x):
    with np.errstate(all="ignore"):
        pos = 1.0 / (1.0 + np.exp(-x))
        ex = np.exp(x)
        neg = ex / (1.0 + ex)
    return np.where(_re(x) >= 0, pos, neg)


def _smin(x, y, tau):
    """Soft minimum -tau log(exp(-x/tau) + exp(-y/tau)), evaluated stably."""
    m = np.minimum(_re(x), _re(y))
    with np.errstate(all="ignore"):
        return m - tau * np.log(np.exp(-(x - m) / tau) + np.exp(-(y - m) / tau))


def _clamp_offset(s, R):
    """Identity for |s| <= R, sign(s) R (2 - exp(1 - |s| / R)) beyond (C1, |.| < 2R)."""
    a = np.where(_re(s) >= 0, s, -s)
    sgn = np.where(_re(s) >= 0, 1.0, -1.0)
    with np.errstate(all="ignore"):
        return np.where(_re(a) <= R, s, sgn * R * (2.0 - np.exp(1.0 - a / R)))


def primitive_terms(kind, dims, R, C, a, b, fx, fy, tau=TAU_PX):
    """Per-pixel terms of one primitive for rays d = (a, b, 1) over the pixel grid:
    (Delta, delta_px, z, ok, None for an ellipsoid or (delta_y_px, fade) for a cone)."""
    # local frame: ray from the camera o + t e, o = R^T (0 - C), e = R^T d
    o = -(R.T @ C)
    e = [R[0, i] * a + R[1, i] * b + R[2, i] for i in range(3)]
    eu = [R[0, i] / fx for i in range(3)]  # d e / d u (pixel column)
    ev = [R[1, i] / fy for i in range(3)]  # d e / d v (pixel row)
    if kind == 0:
        sc = [dims[0], dims[1], dims[2]]
        Q = [1.0, 1.0, 1.0]
        qv = [0.0, 0.0, 0.0]
    else:
        ax, az, hl, kap = dims[0], dims[1], dims[2], dims[3]
        sc = [ax, hl, az]
        Q = [1.0, -kap * kap, 1.0]
        qv = [0.0, -kap, 0.0]
    os_ = [o[i] / sc[i] for i in range(3)]
    es = [e[i] / sc[i] for i in range(3)]
    esu = [eu[i] / sc[i] for i in range(3)]
    esv = [ev[i] / sc[i] for i in range(3)]
    A = sum(Q[i] * es[i] * es[i] for i in range(3))
    B = sum(Q[i] * os_[i] * es[i] + qv[i] * es[i] for i in range(3))
    Cq = sum(Q[i] * os_[i] * os_[i] + 2.0 * qv[i] * os_[i] for i in range(3)) - 1.0
    Au = sum(2.0 * Q[i] * es[i] * esu[i] for i in range(3))
    Av = sum(2.0 * Q[i] * es[i] * esv[i] for i in range(3))
    Bu = sum(Q[i] * os_[i] * esu[i] + qv[i] * esu[i] for i in range(3))
    Bv = sum(Q[i] * os_[i] * esv[i] + qv[i] * esv[i] for i in range(3))
    Dl = B * B - A * Cq
    Du = 2.0 * B * Bu - Au * Cq
    Dv = 2.0 * B * Bv - Av * Cq
    with np.errstate(all="ignore"):
        N = np.sqrt(Du * Du + Dv * Dv)
        N = np.where(_re(N) > 1e-300, N, 1e-300)
        delta = Dl / N
        tn = tau * N
        Dp = 0.5 * (Dl + np.sqrt(Dl * Dl + tn * tn))  # soft positive part of Delta
        r = np.sqrt(Dp)
        t = Cq / (-B + r)  # the near root (B < 0), without cancellation
        if kind == 0:
            Rb = max(dims[0], dims[1], dims[2])
        else:
            Rb = np.sqrt(dims[2] ** 2 + (max(dims[0], dims[1]) * (1.0 + abs(dims[3]))) ** 2)
        t0 = C[2]
        t = t0 + _clamp_offset(t - t0, Rb)
    ok = (_re(A) > 0) & (_re(B) < 0) & (_re(t) > 0)
    if kind == 0:
        return Dl, delta, t, ok, None
    ax, az, hl, kap = dims[0], dims[1], dims[2], dims[3]
    ends = [C + sgn * hl * R[:, 1] for sgn in (-1.0, 1.0)]  # axis end points (camera frame)
    du = fx * (ends[1][0] / ends[1][2] - ends[0][0] / ends[0][2])
    dv = fy * (ends[1][1] / ends[1][2] - ends[0][1] / ends[0][2])
    half_len = 0.5 * np.sqrt(du * du + dv * dv)
    r_px = max(ax, az) * (1.0 + abs(kap)) * fx / C[2]
    L = half_len if _re(half_len) > _re(r_px) else r_px
    with np.errstate(all="ignore"):
        a_rel = A / (es[0] * es[0] + es[1] * es[1] + es[2] * es[2])  # squared sine to the generator
        a4 = a_rel ** 4
        fade = a4 / (a4 + (0.06 * tau) ** 4)
        y_root = os_[1] + t * es[1]
        y_near = os_[1] + (t0 + _clamp_offset(-B / A - t0, Rb)) * es[1]
        Y = y_near + _sigmoid(delta / tau - 2.0) * (y_root - y_near)
        absY = np.where(_re(Y) >= 0, Y, -Y)
        delta_y = (1.0 - absY) * L  # pixels to the cone's end along its projected axis
    return Dl, delta, t, ok, (delta_y, fade)


def soft_objective(model: Model, pose, cam, Od, S, params=DEFAULT_PARAMS, *, tau=TAU_PX, tau_mm=TAU_MM,
                   return_parts=False):
    """E_s of one pose (real or complex) against observation (Od [H, W] mm, S [H, W])."""
    d_m, d_M, lam, lam_k = params
    fx, fy, cx, cy = cam
    Od = np.asarray(Od, np.float64)
    S = np.asarray(S) != 0
    H, W = Od.shape
    a = ((np.arange(W) + 0.5 - cx) / fx)[None, :] * np.ones((H, 1))
    b = ((np.arange(H) + 0.5 - cy) / fy)[:, None] * np.ones((1, W))
    _, pR, pC, kc = fk(model, pose)
    cplx = np.iscomplexobj(pR) or np.iscomplexobj(pC)
    dt = complex if cplx else float
    npr = model.prims_i.shape[0]
    alpha = np.zeros((npr, H, W), dt)
    z = np.zeros((npr, H, W), dt)
    for j in range(npr):
        kind = int(model.prims_i[j, 1])
        _, delta, t, ok, delta_y = primitive_terms(kind, model.prims_f[j, 3:7], pR[j], pC[j], a, b, fx, fy, tau)
        sig = _sigmoid(delta / tau)
        if delta_y is not None:
            dy, fade = delta_y
            sig = sig * _sigmoid(dy / tau) * fade
        alpha[j] = np.where(ok, sig, 0.0)
        z[j] = np.where(ok, t, 1e30)  # primitives that do not count sort last
    # front-to-back compositing in order of depth (decided on real parts)
    order = np.argsort(_re(z), axis=0, kind="stable")
    al = np.take_along_axis(alpha, order, axis=0)
    zz = np.take_along_axis(z, order, axis=0)
    T = np.cumprod(np.concatenate([np.ones((1, H, W), dt), 1.0 - al[:-1]], axis=0), axis=0)
    wgt = T * al
    c = wgt.sum(axis=0)
    with np.errstate(all="ignore"):
        zt = np.where(_re(c) > 0, (wgt * np.where(_re(al) > 0, zz, 0.0)).sum(axis=0) / np.where(_re(c) > 0, c, 1.0),
                      0.0)
    valid = S & (Od > 0)
    diff = np.sqrt((Od - zt) ** 2 + tau_mm * tau_mm)  # soft |O_d - z~|
    t_hit = np.where(valid, _smin(diff, d_M, tau_mm), np.where(S, 0.0, d_M))
    t_miss = np.where(valid, d_M, 0.0)
    m = np.where(valid, _sigmoid((d_m - diff) / tau_mm), 1.0)
    t_px = c * t_hit + (1.0 - c) * t_miss
    r_m = c * m
    s_t = t_px.sum()
    s_and = (S * r_m).sum()
    s_or = (S + (~S) * r_m).sum()
    if _re(s_or) == 0:
        D = lam + 0.0 * s_t
    else:
        D = s_t / s_or + lam * (1.0 - 2.0 * s_and / (s_and + s_or))
    E = D + lam_k * kc
    if return_parts:
        return E, dict(sum_t=s_t, sum_and=s_and, sum_or=s_or, coverage=c, depth=zt, kc=kc, t=t_px, r_m=r_m)
    return E


def soft_gradient(model: Model, pose, cam, Od, S, params=DEFAULT_PARAMS, *, h=1e-30, **kw) -> np.ndarray:
    """dE_s/dpose [26] by the complex step (one complex evaluation per DOF)."""
    pose = np.asarray(pose, np.float64)
    g = np.zeros(pose.shape[0])
    for k in range(pose.shape[0]):
        pc = pose.astype(complex)
        pc[k] += 1j * h
        g[k] = np.imag(soft_objective(model, pc, cam, Od, S, params, **kw)) / h
    return g


def central_difference(model: Model, pose, cam, Od, S, params=DEFAULT_PARAMS, *, h_rad=1e-4, h_mm=1e-2,
                       **kw) -> np.ndarray:
    """FP64 central differences of E_s: h = 1e-2 mm for the wrist translation,
    1e-4 rad for every angle."""
    pose = np.asarray(pose, np.float64)
    g = np.zeros(pose.shape[0])
    for k in range(pose.shape[0]):
        h = h_mm if k < 3 else h_rad
        p1, p0 = pose.copy(), pose.copy()
        p1[k] += h
        p0[k] -= h
        g[k] = (soft_objective(model, p1, cam, Od, S, params, **kw)
                - soft_objective(model, p0, cam, Od, S, params, **kw)) / (2 * h)
    return g
