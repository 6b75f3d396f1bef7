"""FP64 interpenetration test of a hand pose and the kc variants built on it.
Test infrastructure only: the test-suite may import it, the product path
never does.

Section III.A adds lambda_k kc(h) to E (Eq. 5) to rule out implausible poses
such as two fingers passing through each other; its kc only orders the
abduction angles of the three adjacent pairs of non-thumb fingers.  The
variants test interpenetration directly (the reading, stated once here and
implemented independently on the GPU):

* collision proxies are inscribed spheres of the model's primitives: one per
  ellipsoid (its centre, its smallest semi-axis), three per truncated cone, on
  its axis at local y = -hl/2, 0, +hl/2, each the largest sphere about that
  point inside the cone of circular section rho (1 + kappa y / hl),
  rho = min(ax, az) (which the elliptic cone contains): the smaller of the
  distance to its slanted side, rho (1 + kappa y / hl) / sqrt(1 + (rho kappa /
  hl)^2), and the distance to its end plane, hl - |y|;
* a primitive's finger is the child of the palm bone on its bone's path to the
  palm (numbered in bone order); palm primitives take no part;
* a proxy centred at the origin of a bone attached to the palm (a knuckle
  sphere) is fixed to the palm whatever the pose; pairs of two such proxies
  are left out, since their distance is a constant of the model;
* pen(h) = sum over the remaining pairs of proxies on different fingers of
  max(0, r_i + r_j - |c_i - c_j|), in mm;
* variant 0: the paper's kc; 1: kc + w pen; 2: w pen (w in rad per mm).

Everything is a plain loop over the definition.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

PRIM_ELLIPSOID, PRIM_ECONE = 0, 1


def fingers(bones_i) -> np.ndarray:
    """Finger number of every bone (-1 for the palm, bone 0)."""
    parent = np.asarray(bones_i)[:, 0]
    f = np.full(len(parent), -1, int)
    n = 0
    for b in range(1, len(parent)):
        if parent[b] == 0:
            f[b] = n
            n += 1
        else:
            f[b] = f[parent[b]]
    return f


def proxies(model: O.Model, fk: dict):
    """Centres (camera frame, mm) [n, 3], radii [n], fingers [n] and the
    fixed-to-the-palm flags [n] of the collision proxies of the pose whose FK
    is `fk` (oracle.fk)."""
    fb = fingers(model.bones_i)
    parent = model.bones_i[:, 0]
    C, r, f, fixed = [], [], [], []
    for k in range(model.np_):
        bone, kind = int(model.prims_i[k, 0]), int(model.prims_i[k, 1])
        d = model.prims_f[k, 3:]
        R, c = fk["prim_R"][k], fk["prim_C"][k]
        if kind == PRIM_ELLIPSOID:
            C.append(c)
            r.append(min(d[0], d[1], d[2]))
            f.append(fb[bone])
            fixed.append(bone > 0 and parent[bone] == 0 and not np.any(model.prims_f[k, :3]))
        else:
            ax, az, hl, kap = d
            rho = min(ax, az)
            for y in (-hl / 2, 0.0, hl / 2):
                C.append(c + R @ np.array([0.0, y, 0.0]))
                side = rho * (1.0 + kap * y / hl) / np.sqrt(1.0 + (rho * kap / hl) ** 2)
                r.append(min(side, hl - abs(y)))
                f.append(fb[bone])
                cen = model.prims_f[k, :3] + np.array([0.0, y, 0.0])
                fixed.append(bone > 0 and parent[bone] == 0 and not np.any(cen))
    return np.array(C), np.array(r), np.array(f), np.array(fixed, bool)


def penetration_of(C, r, f, fixed=None):
    """sum over pairs on different fingers (both >= 0), not both fixed to the
    palm, of max(0, r_i + r_j - d_ij).  Centres may be complex (the complex
    step below): the max is then decided on the real part."""
    pen = 0.0
    n = len(r)
    if fixed is None:
        fixed = np.zeros(n, bool)
    for i in range(n):
        for j in range(i + 1, n):
            if f[i] < 0 or f[j] < 0 or f[i] == f[j] or (fixed[i] and fixed[j]):
                continue
            d = np.sqrt(np.sum((C[i] - C[j]) ** 2))
            v = r[i] + r[j] - d
            if np.real(v) > 0.0:
                pen = pen + v
    return pen if np.iscomplexobj(pen) else float(pen)


def penetration(model: O.Model, pose) -> float:
    fk = O.fk(model, pose)
    return penetration_of(*proxies(model, fk))


def kc_variant_gradient(model: O.Model, pose, variant: int, w: float, h: float = 1e-30) -> np.ndarray:
    """d kc_variant / d pose [26] by the complex step: the pose is perturbed
    by i h in one dimension at a time and carried through the FK of
    oracle.soft (which takes complex poses), the proxies and the sum above;
    the imaginary part over h is the derivative (no cancellation, exact to
    rounding where the function is smooth)."""
    from . import soft as OS

    pose = np.asarray(pose, np.float64)
    g = np.zeros(pose.shape[0])
    for k in range(pose.shape[0]):
        pc = pose.astype(complex)
        pc[k] += 1j * h
        _, pR, pC, kc = OS.fk(model, pc)
        val = 0.0 if variant == 2 else kc
        if variant != 0:
            val = val + w * penetration_of(*proxies(model, {"prim_R": pR, "prim_C": pC}))
        g[k] = np.imag(val) / h
    return g


def kc_variant(model: O.Model, pose, variant: int, w: float) -> float:
    """kc of Eq. 5 under the given variant (on the clamped pose, as oracle.fk)."""
    fk = O.fk(model, pose)
    k = fk["kc"]
    if variant == 0:
        return k
    pen = penetration_of(*proxies(model, fk))
    return (k if variant == 1 else 0.0) + w * pen
