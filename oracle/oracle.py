"""ctypes binding of the FP64 oracle (hs_oracle.c).  Test infrastructure only.

All arrays are numpy float64 / int32 / uint8, C-contiguous.  The hand model
arrives as the flat arrays of a geometry descriptor (bones_i, bones_f,
prims_i, prims_f) plus joint limits (lo, hi); the camera as (fx, fy, cx, cy).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_u32 = ctypes.POINTER(ctypes.c_uint32)


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [_u32, _u32, _u32]
        L.or_uniform.argtypes = [ctypes.c_uint32]
        L.or_uniform.restype = ctypes.c_double
        L.or_clamp_pose.argtypes = [_d, _d, _d, _d]
        L.or_kc.argtypes = [_d]
        L.or_kc.restype = ctypes.c_double
        L.or_fk.argtypes = [ctypes.c_int, _i32, _d, ctypes.c_int, _i32, _d, _d, _d, _d, _d, _d, _d, _d,
                            _d, _d]
        L.or_intersect.argtypes = [ctypes.c_int, _d, _d, _d, _d, ctypes.POINTER(ctypes.c_int)]
        L.or_intersect.restype = ctypes.c_double
        L.or_render.argtypes = [ctypes.c_int, _i32, _d, _d, _d, _d, ctypes.c_int, ctypes.c_int, _d, _u8,
                                _i32, _u8, ctypes.c_double, ctypes.c_double]
        L.or_cost.argtypes = [ctypes.c_int, ctypes.c_int, _d, _u8, _d, _u8, _d, _d, _u8]
        L.or_cost.restype = ctypes.c_double
        L.or_score_batch.argtypes = [ctypes.c_int, _d, ctypes.c_int, _i32, _d, ctypes.c_int, _i32, _d, _d,
                                     _d, _d, ctypes.c_int, ctypes.c_int, _d, _u8, _d, _d, _d, _d, _d, _d,
                                     _u8, _u8, _u8, ctypes.c_double, ctypes.c_double]
        L.or_pso_w.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_pso_w.restype = ctypes.c_double
        L.or_pso_update.argtypes = [_d] * 6 + [ctypes.c_double] * 3 + [_d] * 4
        L.or_pso_step.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _d, _d, _d, _d, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_int, ctypes.c_int]
        L.or_pso_init.argtypes = [ctypes.c_int, _d, _d, _d, _d, ctypes.c_uint64, ctypes.c_uint32, _d, _d,
                                  _d, _d, _d, _d]
        L.or_mean_joint_error_deg.argtypes = [_d, _d]
        L.or_mean_joint_error_deg.restype = ctypes.c_double
        _LIB = L
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _b(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


# constants of Section III.A (after Eq. 5) with d_m, d_M in mm
DEFAULT_PARAMS = (10.0, 40.0, 20.0, 10.0)  # d_m, d_M, lambda, lambda_k
PSO_C1, PSO_C2 = 2.8, 1.3                   # Section III.B


@dataclass
class Model:
    bones_i: np.ndarray
    bones_f: np.ndarray
    prims_i: np.ndarray
    prims_f: np.ndarray
    lo: np.ndarray
    hi: np.ndarray

    @classmethod
    def from_geometry(cls, g, lo, hi) -> "Model":
        return cls(_i(g.bones_i), _f64(g.bones_f), _i(g.prims_i), _f64(g.prims_f), _f64(lo), _f64(hi))

    @property
    def nb(self):
        return self.bones_i.shape[0]

    @property
    def np_(self):
        return self.prims_i.shape[0]


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, _u32), _p(k, _u32), _p(out, _u32))
    return out


def uniform(u: int) -> float:
    return lib().or_uniform(ctypes.c_uint32(u))


def kc(q) -> float:
    q = _f64(q)
    return lib().or_kc(_p(q, _d))


def fk(model: Model, pose):
    """Returns dict(q, bone_R [nb,3,3], bone_p [nb,3], prim_R [np,3,3], prim_C [np,3], kc) or None."""
    pose = _f64(pose)
    q = np.zeros(26)
    bR = np.zeros((model.nb, 3, 3))
    bp = np.zeros((model.nb, 3))
    pR = np.zeros((model.np_, 3, 3))
    pC = np.zeros((model.np_, 3))
    k = ctypes.c_double(0.0)
    rc = lib().or_fk(model.nb, _p(model.bones_i, _i32), _p(model.bones_f, _d), model.np_,
                     _p(model.prims_i, _i32), _p(model.prims_f, _d), _p(model.lo, _d), _p(model.hi, _d),
                     _p(pose, _d), _p(q, _d), _p(bR, _d), _p(bp, _d), _p(pR, _d), _p(pC, _d),
                     ctypes.byref(k))
    if rc != 0:
        return None
    return dict(q=q, bone_R=bR, bone_p=bp, prim_R=pR, prim_C=pC, kc=k.value)


def intersect(kind: int, dims, R, C, d):
    dims = _f64(dims)
    R = _f64(R)
    C = _f64(C)
    d = _f64(d)
    s = ctypes.c_int(-1)
    t = lib().or_intersect(kind, _p(dims, _d), _p(R, _d), _p(C, _d), _p(d, _d), ctypes.byref(s))
    return t, s.value


def render(prims_i, prims_f, prim_R, prim_C, cam, W, H, *, jitter=2e-3, tie_mm=1e-3, boundary=True):
    """Render camera-space primitives.  Returns (depth, hit, prim_id, boundary)."""
    prims_i = _i(prims_i)
    prims_f = _f64(prims_f)
    pR = _f64(prim_R)
    pC = _f64(prim_C)
    cam = _f64(cam)
    depth = np.zeros((H, W))
    hit = np.zeros((H, W), np.uint8)
    pid = np.zeros((H, W), np.int32)
    bnd = np.zeros((H, W), np.uint8) if boundary else None
    lib().or_render(prims_i.shape[0], _p(prims_i, _i32), _p(prims_f, _d), _p(pR, _d), _p(pC, _d),
                    _p(cam, _d), W, H, _p(depth, _d), _p(hit, _u8), _p(pid, _i32), _p(bnd, _u8),
                    jitter, tie_mm)
    return depth, hit.astype(bool), pid, (bnd.astype(bool) if boundary else None)


def render_pose(model: Model, pose, cam, W, H, **kw):
    f = fk(model, pose)
    return render(model.prims_i, model.prims_f, f["prim_R"], f["prim_C"], cam, W, H, **kw)


def cost(depth, hit, Od, S, params=DEFAULT_PARAMS):
    """Eq. 4 by reading R1.  Returns (D, sums(3,), r_m)."""
    depth = _f64(depth)
    H, W = depth.shape
    hit = _b(hit)
    Od = _f64(Od)
    S = _b(S)
    prm = _f64(params)
    sums = np.zeros(3)
    rm = np.zeros((H, W), np.uint8)
    D = lib().or_cost(W, H, _p(depth, _d), _p(hit, _u8), _p(Od, _d), _p(S, _u8), _p(prm, _d),
                      _p(sums, _d), _p(rm, _u8))
    return D, sums, rm.astype(bool)


def score_batch(model: Model, poses, cam, Od, S, params=DEFAULT_PARAMS, *, per_pixel=False,
                jitter=2e-3, tie_mm=1e-3):
    """E, D, kc, sums for P poses; with per_pixel also depth/hit/rm/boundary [P,H,W]."""
    poses = _f64(np.atleast_2d(poses))
    P = poses.shape[0]
    Od = _f64(Od)
    H, W = Od.shape
    S = _b(S)
    cam = _f64(cam)
    prm = _f64(params)
    E = np.zeros(P)
    D = np.zeros(P)
    kcv = np.zeros(P)
    sums = np.zeros((P, 3))
    depth = np.zeros((P, H, W)) if per_pixel else None
    hit = np.zeros((P, H, W), np.uint8) if per_pixel else None
    rm = np.zeros((P, H, W), np.uint8) if per_pixel else None
    bnd = np.zeros((P, H, W), np.uint8) if per_pixel else None
    lib().or_score_batch(P, _p(poses, _d), model.nb, _p(model.bones_i, _i32), _p(model.bones_f, _d),
                         model.np_, _p(model.prims_i, _i32), _p(model.prims_f, _d), _p(model.lo, _d),
                         _p(model.hi, _d), _p(cam, _d), W, H, _p(Od, _d), _p(S, _u8), _p(prm, _d),
                         _p(E, _d), _p(D, _d), _p(kcv, _d), _p(sums, _d), _p(depth, _d), _p(hit, _u8),
                         _p(rm, _u8), _p(bnd, _u8), jitter, tie_mm)
    out = dict(E=E, D=D, kc=kcv, sums=sums)
    if per_pixel:
        out.update(depth=depth, hit=hit.astype(bool), rm=rm.astype(bool), boundary=bnd.astype(bool))
    return out


def pso_w(c1=PSO_C1, c2=PSO_C2) -> float:
    return lib().or_pso_w(c1, c2)


def pso_update(x, v, pbest, gbest, r1, r2, lo, hi, c1=PSO_C1, c2=PSO_C2, w=None):
    x, v, pbest, gbest, r1, r2, lo, hi = map(_f64, (x, v, pbest, gbest, r1, r2, lo, hi))
    if w is None:
        w = pso_w(c1, c2)
    xo = np.zeros(26)
    vo = np.zeros(26)
    lib().or_pso_update(_p(x, _d), _p(v, _d), _p(pbest, _d), _p(gbest, _d), _p(r1, _d), _p(r2, _d),
                        c1, c2, w, _p(lo, _d), _p(hi, _d), _p(xo, _d), _p(vo, _d))
    return xo, vo


class Swarm:
    """FP64 swarm state: x, v, pbest [P,26], pbest_E [P], gbest [26], gbest_E."""

    def __init__(self, x, v, pbest, pbest_E, gbest, gbest_E):
        self.x, self.v, self.pbest = _f64(x).copy(), _f64(v).copy(), _f64(pbest).copy()
        self.pbest_E = _f64(pbest_E).copy()
        self.gbest = _f64(gbest).copy()
        self.gbest_E = float(gbest_E)

    def copy(self) -> "Swarm":
        return Swarm(self.x, self.v, self.pbest, self.pbest_E, self.gbest, self.gbest_E)


def pso_init(P, seed_pose, scale, lo, hi, seed, frame) -> Swarm:
    seed_pose, scale, lo, hi = map(_f64, (seed_pose, scale, lo, hi))
    x = np.zeros((P, 26))
    v = np.zeros((P, 26))
    pb = np.zeros((P, 26))
    pbE = np.zeros(P)
    gb = np.zeros(26)
    gE = ctypes.c_double(0)
    lib().or_pso_init(P, _p(seed_pose, _d), _p(scale, _d), _p(lo, _d), _p(hi, _d), seed, frame,
                      _p(x, _d), _p(v, _d), _p(pb, _d), _p(pbE, _d), _p(gb, _d), ctypes.byref(gE))
    return Swarm(x, v, pb, pbE, gb, gE.value)


def pso_step(sw: Swarm, E, lo, hi, seed, frame, gen, mutate_every=3, n_mutate=None,
             c1=PSO_C1, c2=PSO_C2) -> Swarm:
    """One generation (in a copy of sw)."""
    s = sw.copy()
    P = s.x.shape[0]
    if n_mutate is None:
        n_mutate = P // 2
    E = _f64(E)
    lo, hi = _f64(lo), _f64(hi)
    gE = ctypes.c_double(s.gbest_E)
    lib().or_pso_step(P, _p(s.x, _d), _p(s.v, _d), _p(s.pbest, _d), _p(s.pbest_E, _d), _p(s.gbest, _d),
                      ctypes.byref(gE), _p(E, _d), _p(lo, _d), _p(hi, _d), c1, c2, seed, frame, gen,
                      mutate_every, n_mutate)
    s.gbest_E = gE.value
    return s


def mean_joint_error_deg(a, b) -> float:
    a, b = _f64(a), _f64(b)
    return lib().or_mean_joint_error_deg(_p(a, _d), _p(b, _d))


def camera_tuple(cam) -> np.ndarray:
    return np.array([cam.fx, cam.fy, cam.cx, cam.cy], np.float64)


def track_frame(model: Model, cam, Od, S, seed_pose, scale, P, gens, seed, frame,
                params=DEFAULT_PARAMS, mutate_every=3):
    """Plain PSO on one frame (Section III.B): init around seed_pose, then `gens`
    generations of score + step.  Returns (swarm, history of gbest_E)."""
    sw = pso_init(P, seed_pose, scale, model.lo, model.hi, seed, frame)
    hist = []
    for g in range(1, gens + 1):
        r = score_batch(model, sw.x, camera_tuple(cam), Od, S, params)
        sw = pso_step(sw, r["E"], model.lo, model.hi, seed, frame, g, mutate_every)
        hist.append(sw.gbest_E)
    return sw, hist


def threads_used() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
