"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds data only: the paper's joint-limit tables, a seeded hand
geometry descriptor, seeded poses and trajectories, the camera intrinsics and
the Kinect-style corruption of an already rendered depth image.  It contains
none of the method's arithmetic (no kinematics, no ray casting, no cost, no
swarm update), so both sides can consume its output without sharing code.

Conventions (units mm and rad):

* Pose ``h`` (Eq. 1-3): ``[x, y, z, tx, ty, tz]`` for the wrist (Eq. 2),
  followed by ``(MP_x, MP_z, PIP, DIP)`` (Eq. 1) for thumb, index, middle,
  ring and pinky.  Index ``6 + 4 f + j`` addresses finger ``f`` joint ``j``.
* Geometry descriptor: 16 bones (palm + 3 per finger) and 37 primitives
  (Section II.A and Fig. 2: palm = elliptic cylinder capped by two
  ellipsoids; every finger = 3 truncated cones + 4 spheres; the thumb's
  largest phalanx is an ellipsoid).  The thumb keeps 3 spheres (its root
  sphere is covered by the ellipsoid), so 3 + 6 + 4 * 7 = 37.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

N_DOF = 26
N_BONES = 16
N_PRIMS = 37

# primitive kinds
PRIM_ELLIPSOID = 0  # dims = (sx, sy, sz, unused): semi-axes along local x, y, z
PRIM_ECONE = 1      # dims = (ax, az, hl, kappa): capped elliptic truncated cone
                    # along local y, |y| <= hl, section semi-axes scaled by
                    # (1 + kappa * y / hl); kappa = 0 is an elliptic cylinder

FINGERS = ("thumb", "index", "middle", "ring", "pinky")
JOINTS = ("MPx", "MPz", "PIP", "DIP")

# Table 1 (finger angle limits, degrees) and Table 2 (wrist limits, metres and
# degrees), transcribed as printed in the paper (Section II.A).
TABLE1_DEG = {
    "thumb":  ((0, 90), (-15, 60), (0, 50), (-15, 70)),
    "index":  ((0, 90), (-15, 15), (0, 100), (0, 60)),
    "middle": ((0, 90), (-10, 10), (0, 100), (0, 60)),
    "ring":   ((0, 90), (-30, 0), (0, 100), (0, 60)),
    "pinky":  ((0, 90), (-45, 0), (0, 100), (0, 60)),
}
TABLE2 = {  # x_c, y_c, z_c in metres; angles in degrees
    "x_m": (-0.9, 0.9), "y_m": (-0.68, 0.68), "z_m": (0.5, 1.5),
    "tx_deg": (-30, 120), "ty_deg": (-70, 75), "tz_deg": (-35, 20),
}

# the view box that keeps synthetic hands inside the ROI and in front of the
# 600 mm background plane; intersected with Table 2 for the search space
VIEW_BOX = {
    "x_mm": (-60.0, 60.0), "y_mm": (40.0, 120.0), "z_mm": (500.0, 540.0),
    "tx_deg": (-15.0, 40.0), "ty_deg": (-30.0, 30.0), "tz_deg": (-35.0, 20.0),
}

GEOMETRY_SEED = 20050706
CONFIG_SEED_BASE = 2005070680  # configuration k uses CONFIG_SEED_BASE + k


def dof_index(finger: str, joint: str) -> int:
    return 6 + 4 * FINGERS.index(finger) + JOINTS.index(joint)


def paper_joint_limits() -> tuple[np.ndarray, np.ndarray]:
    """Tables 1-2 as (lo, hi) float64 arrays in mm / rad."""
    lo = np.zeros(N_DOF)
    hi = np.zeros(N_DOF)
    for i, key in enumerate(("x_m", "y_m", "z_m")):
        lo[i], hi[i] = (v * 1000.0 for v in TABLE2[key])
    for i, key in enumerate(("tx_deg", "ty_deg", "tz_deg")):
        lo[3 + i], hi[3 + i] = (math.radians(v) for v in TABLE2[key])
    for f in FINGERS:
        for j, (a, b) in enumerate(TABLE1_DEG[f]):
            k = 6 + 4 * FINGERS.index(f) + j
            lo[k], hi[k] = math.radians(a), math.radians(b)
    return lo, hi


def search_limits() -> tuple[np.ndarray, np.ndarray]:
    """Tables 1-2 intersected with the view box (the PSO search space)."""
    lo, hi = paper_joint_limits()
    box = [VIEW_BOX["x_mm"], VIEW_BOX["y_mm"], VIEW_BOX["z_mm"]]
    box += [tuple(math.radians(v) for v in VIEW_BOX[k]) for k in ("tx_deg", "ty_deg", "tz_deg")]
    for i, (a, b) in enumerate(box):
        lo[i] = max(lo[i], a)
        hi[i] = min(hi[i], b)
    return lo, hi


@dataclass
class HandGeometry:
    """Flat arrays describing the kinematic tree and the primitives.

    bones_i[b] = (parent, dof_z, dof_x)   (-1 = none; bone 0 is the palm/root)
    bones_f[b] = (off_x, off_y, off_z, rest_x, rest_y, rest_z): offset of the
                 bone origin in the parent frame (mm) and a fixed rest rotation
                 given as angles (rad) of Rz(rest_z) Ry(rest_y) Rx(rest_x)
    prims_i[k] = (bone, kind)
    prims_f[k] = (c_x, c_y, c_z, d0, d1, d2, d3): centre in the bone frame and
                 the kind's dims; primitives are axis-aligned with their bone
    """
    bones_i: np.ndarray  # int32 [16, 3]
    bones_f: np.ndarray  # float64 [16, 6]
    prims_i: np.ndarray  # int32 [37, 2]
    prims_f: np.ndarray  # float64 [37, 7]
    lengths: np.ndarray  # float64 [5, 3] phalanx lengths, for tests
    palm_length: float


def hand_geometry(seed: int = GEOMETRY_SEED) -> HandGeometry:
    """Seeded 16-bone / 37-primitive hand; bone lengths lie in [20, 90] mm."""
    rng = np.random.default_rng(seed)
    # on a 1/64 mm grid, so the palm cylinder's cap planes (centre +- half
    # length) coincide exactly with the end ellipsoids in float32 as well
    palm_len = round(float(rng.uniform(75.0, 90.0)) * 64.0) / 64.0
    scale = {"index": 1.0, "middle": 1.06, "ring": 0.98, "pinky": 0.82}
    lengths = np.zeros((5, 3))
    lengths[0] = [rng.uniform(40, 50), rng.uniform(28, 36), rng.uniform(22, 28)]
    for f in FINGERS[1:]:
        raw = [rng.uniform(38, 50), rng.uniform(22, 32), rng.uniform(20, 26)]
        lengths[FINGERS.index(f)] = np.clip(np.array(raw) * scale[f], 20.0, 90.0)
    base_r = {"thumb": 10.0, "index": 9.0, "middle": 9.3, "ring": 8.7, "pinky": 7.5}
    taper = (1.0, 0.88, 0.78, 0.70)  # joint radii at MCP, PIP, DIP, tip

    bones_i = np.full((N_BONES, 3), -1, np.int32)
    bones_f = np.zeros((N_BONES, 6))
    mcp_x = {"index": -25.0, "middle": -8.0, "ring": 9.0, "pinky": 25.0}
    mcp_dy = {"index": -2.0, "middle": 0.0, "ring": -3.0, "pinky": -10.0}
    splay = {"index": 0.10, "middle": 0.0, "ring": -0.08, "pinky": -0.18}
    for fi, f in enumerate(FINGERS):
        b1 = 1 + 3 * fi
        bones_i[b1] = (0, dof_index(f, "MPz"), dof_index(f, "MPx"))
        if f == "thumb":
            bones_f[b1] = (-30.0, 18.0, 8.0, 0.0, 0.6, 0.85)
        else:
            bones_f[b1] = (mcp_x[f], palm_len + mcp_dy[f], 0.0, 0.0, 0.0, splay[f])
        bones_i[b1 + 1] = (b1, -1, dof_index(f, "PIP"))
        bones_f[b1 + 1] = (0.0, lengths[fi, 0], 0.0, 0.0, 0.0, 0.0)
        bones_i[b1 + 2] = (b1 + 1, -1, dof_index(f, "DIP"))
        bones_f[b1 + 2] = (0.0, lengths[fi, 1], 0.0, 0.0, 0.0, 0.0)

    prims_i = np.zeros((N_PRIMS, 2), np.int32)
    prims_f = np.zeros((N_PRIMS, 7))
    k = 0

    def add(bone, kind, centre, dims):
        nonlocal k
        prims_i[k] = (bone, kind)
        prims_f[k, :3] = centre
        prims_f[k, 3:] = dims
        k += 1

    def cone(bone, length, r0, r1):
        add(bone, PRIM_ECONE, (0.0, length / 2, 0.0),
            ((r0 + r1) / 2, (r0 + r1) / 2, length / 2, (r1 - r0) / (r1 + r0)))

    def sphere(bone, y, r):
        add(bone, PRIM_ELLIPSOID, (0.0, y, 0.0), (r, r, r, 0.0))

    y0, y1 = 14.0, palm_len - 8.0
    add(0, PRIM_ECONE, (0.0, (y0 + y1) / 2, 0.0), (38.0, 13.0, (y1 - y0) / 2, 0.0))
    add(0, PRIM_ELLIPSOID, (0.0, y0, 0.0), (38.0, 12.0, 13.0, 0.0))
    add(0, PRIM_ELLIPSOID, (0.0, y1, 0.0), (38.0, 10.0, 13.0, 0.0))
    for fi, f in enumerate(FINGERS):
        r = [base_r[f] * t for t in taper]
        b1 = 1 + 3 * fi
        L = lengths[fi]
        if f == "thumb":
            add(b1, PRIM_ELLIPSOID, (0.0, L[0] / 2, 0.0), (11.0, L[0] / 2, 10.0, 0.0))
        else:
            sphere(b1, 0.0, r[0])
            cone(b1, L[0], r[0], r[1])
        sphere(b1 + 1, 0.0, r[1])
        cone(b1 + 1, L[1], r[1], r[2])
        sphere(b1 + 2, 0.0, r[2])
        cone(b1 + 2, L[2], r[2], r[3])
        sphere(b1 + 2, L[2], r[3])
    assert k == N_PRIMS
    return HandGeometry(bones_i, bones_f, prims_i, prims_f, lengths, palm_len)


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float


def kinect_camera(W: int, H: int) -> Camera:
    """Kinect-v1-like pinhole scaled to the ROI width: f = 525 W / 640."""
    f = 525.0 * W / 640.0
    return Camera(f, f, W / 2.0, H / 2.0)


def sample_poses(rng: np.random.Generator, n: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """n poses uniform within [lo, hi] (float64 [n, 26])."""
    return lo + rng.random((n, N_DOF)) * (hi - lo)


def ground_truth_pose(seed: int) -> np.ndarray:
    """One pose uniform within the search limits (Tables 1-2 and the view box)."""
    lo, hi = search_limits()
    return sample_poses(np.random.default_rng(seed), 1, lo, hi)[0]


def trajectory(seed: int, n_frames: int, max_deg: float = 5.0, max_mm: float = 5.0) -> np.ndarray:
    """Smooth seeded trajectory [n_frames, 26]: a base pose plus 3 sinusoids per
    DOF, amplitudes scaled so |step| <= max_deg per frame for angles and
    max_mm for translations, then clipped to the search limits."""
    rng = np.random.default_rng(seed)
    lo, hi = search_limits()
    mid_lo = lo + 0.25 * (hi - lo)
    mid_hi = hi - 0.25 * (hi - lo)
    base = sample_poses(rng, 1, mid_lo, mid_hi)[0]
    omega = rng.uniform(0.05, 0.3, (3, N_DOF))
    phase = rng.uniform(0.0, 2 * math.pi, (3, N_DOF))
    weight = rng.uniform(0.2, 1.0, (3, N_DOF))
    limit = np.full(N_DOF, math.radians(max_deg))
    limit[:3] = max_mm
    # |d/df sum_k A_k sin(w_k f + p_k)| <= sum_k A_k w_k; the per-frame step of a
    # sum of sinusoids is bounded by the same sum, so scale it to `limit`
    amp = weight * (limit / (weight * omega).sum(axis=0))
    span = 0.25 * (hi - lo)
    amp = np.minimum(amp, span / 3.0)
    f = np.arange(n_frames)[:, None, None]
    traj = base + (amp * np.sin(omega * f + phase)).sum(axis=1)
    return np.clip(traj, lo, hi)


def batch_workload(seed: int, n_seq: int = 64, side=(48, 256), particles=(32, 64, 128, 256)
                   ) -> tuple[list[tuple[int, int]], list[int], list[int]]:
    """Many independent sequences at once: per sequence a square ROI whose side
    is uniform in [side[0], side[1]] px, a particle count drawn uniformly from
    `particles`, and a trajectory seed.  Each ROI is the Kinect view scaled to
    its width (kinect_camera), so the hand covers the same fraction of every ROI."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side[0], side[1] + 1, n_seq)
    P = rng.choice(np.asarray(particles), n_seq)
    seeds = rng.integers(1, 2**31 - 1, n_seq)
    return [(int(s), int(s)) for s in sides], [int(p) for p in P], [int(v) for v in seeds]


def perturbation_scale() -> np.ndarray:
    """Half-widths of the tracking init box: 10 mm per translation, 10 deg per angle."""
    s = np.full(N_DOF, math.radians(10.0))
    s[:3] = 10.0
    return s


def kinect_observation(depth: np.ndarray, hit: np.ndarray, seed: int, *, plane_mm: float = 600.0,
                       sigma_mm: float = 3.0, hole_frac: float = 0.05, flip_frac: float = 0.02
                       ) -> tuple[np.ndarray, np.ndarray]:
    """Corrupt a clean rendered depth image like a Kinect v1 frame.

    depth/hit: clean render of the ground-truth pose (mm, bool).  The hand is
    composited in front of a plane at plane_mm; the skin mask is where the hand
    is visible; then N(0, sigma) noise, rounding to uint16 mm, hole_frac of the
    pixels zeroed (a uniform random set) and flip_frac of the mask flipped.
    Returns (uint16 depth [H, W], uint8 skin [H, W]).
    """
    rng = np.random.default_rng(seed)
    H, W = depth.shape
    visible = hit & (depth < plane_mm)
    d = np.where(visible, depth, plane_mm)
    d = d + rng.normal(0.0, sigma_mm, d.shape)
    d = np.clip(np.rint(d), 0, 65535).astype(np.uint16)
    n = H * W
    holes = rng.choice(n, int(round(hole_frac * n)), replace=False)
    d.reshape(-1)[holes] = 0
    skin = visible.astype(np.uint8)
    flips = rng.choice(n, int(round(flip_frac * n)), replace=False)
    skin.reshape(-1)[flips] ^= 1
    return d, skin


def clean_observation(depth: np.ndarray, hit: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Noise-free observation: float32 depth of the render, skin = silhouette."""
    d = np.where(hit, depth, 0.0).astype(np.float32)
    return d, hit.astype(np.uint8)


def pitched(img: np.ndarray, align_bytes: int = 16) -> np.ndarray:
    """Copy a 2-D image into rows padded to a multiple of align_bytes; returns the
    padded [H, pitch_elems] array (the ROI is its [:, :W] view)."""
    H, W = img.shape
    esz = img.dtype.itemsize
    pitch = -(-W * esz // align_bytes) * align_bytes // esz
    out = np.zeros((H, pitch), img.dtype)
    out[:, :W] = img
    return out
