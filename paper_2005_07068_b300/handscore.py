"""Thin ctypes binding of libhandscore.so (include/handscore.h).

Argument marshalling only: every step of the scoring path runs in the CUDA
kernels of the library.  Device memory comes from torch tensors; the stream
is torch's current stream unless one is given.  If the shared library is
missing this module raises at first use; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhandscore.so")

HS_OK, HS_ERR_ARG, HS_ERR_ALIGN, HS_ERR_SIZE, HS_ERR_TIMEOUT, HS_ERR_NOT_IMPL, HS_ERR_CUDA = 0, -1, -2, -3, -4, -5, -6
HS_DEV_NONFINITE_POSE, HS_DEV_TMA_TIMEOUT, HS_DEV_BARRIER_TIMEOUT = 0x1, 0x2, 0x4
HS_KC_ABDUCTION, HS_KC_ABD_PEN, HS_KC_PEN = 0, 1, 2
MAX_PROXIES = 128
HS_PRIM_ELLIPSOID, HS_PRIM_ECONE = 0, 1
HS_DEPTH_U16, HS_DEPTH_F32 = 0, 1
NDOF = 26


class HsBoneDesc(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int32), ("dof_z", ctypes.c_int32), ("dof_x", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("offset", ctypes.c_float * 3), ("rest", ctypes.c_float * 3)]


class HsPrimDesc(ctypes.Structure):
    _fields_ = [("bone", ctypes.c_int32), ("kind", ctypes.c_int32), ("center", ctypes.c_float * 3),
                ("dims", ctypes.c_float * 4)]


class HsModelDesc(ctypes.Structure):
    _fields_ = [("n_bones", ctypes.c_int32), ("n_prims", ctypes.c_int32),
                ("bones", ctypes.POINTER(HsBoneDesc)), ("prims", ctypes.POINTER(HsPrimDesc)),
                ("lo", ctypes.c_float * NDOF), ("hi", ctypes.c_float * NDOF)]


class HsKcParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("pen_weight", ctypes.c_float)]


class HsCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class HsObs(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("skin", ctypes.c_void_p), ("W", ctypes.c_int32),
                ("H", ctypes.c_int32), ("depth_pitch", ctypes.c_int32), ("skin_pitch", ctypes.c_int32),
                ("depth_type", ctypes.c_int32), ("stats", ctypes.c_void_p)]


class HsScoreParams(ctypes.Structure):
    _fields_ = [("d_m", ctypes.c_float), ("d_M", ctypes.c_float), ("lambda_", ctypes.c_float),
                ("lambda_k", ctypes.c_float), ("variant", ctypes.c_int32), ("ctas_per_particle", ctypes.c_int32)]


# render kernels (same results, different work layout); AUTO picks by particles per call
(RENDER_AUTO, RENDER_UNITS, RENDER_TILES_32x16, RENDER_TILES_32x32, RENDER_TILES_64x32, RENDER_TILES_64x64,
 RENDER_STRIPS_8x16, RENDER_STRIPS_8x32, RENDER_PERSISTENT_8x16, RENDER_PERSISTENT_8x32) = range(10)
RENDER_VARIANTS = {"auto": RENDER_AUTO, "units": RENDER_UNITS, "tiles32x16": RENDER_TILES_32x16,
                   "tiles32x32": RENDER_TILES_32x32, "tiles64x32": RENDER_TILES_64x32,
                   "tiles64x64": RENDER_TILES_64x64, "strips8x16": RENDER_STRIPS_8x16,
                   "strips8x32": RENDER_STRIPS_8x32, "persistent8x16": RENDER_PERSISTENT_8x16,
                   "persistent8x32": RENDER_PERSISTENT_8x32}


class HsSwarm(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("x", "v", "pbest", "pbest_E", "gbest", "gbest_E", "E")]


class HsPsoParams(ctypes.Structure):
    _fields_ = [("c1", ctypes.c_float), ("c2", ctypes.c_float), ("mutate_every", ctypes.c_int32),
                ("n_mutate", ctypes.c_int32), ("e_stop", ctypes.c_float)]


class HsSoftParams(ctypes.Structure):
    _fields_ = [("tau_px", ctypes.c_float), ("tau_mm", ctypes.c_float), ("ctas_per_particle", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


SOFT_ADJ = 13  # per-primitive adjoint: M (9), C (3), cone length in pixels (1)


class HsSwarmDesc(ctypes.Structure):
    _fields_ = [("obs", HsObs), ("cam", HsCamera), ("P", ctypes.c_int32), ("n_mutate", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_vp = ctypes.c_void_p
_SIGS = {
    "hs_version": ([], ctypes.c_int),
    "hs_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "hs_model_create": ([ctypes.POINTER(HsModelDesc), ctypes.POINTER(_vp)], ctypes.c_int),
    "hs_model_destroy": ([_vp], ctypes.c_int),
    "hs_model_set_kc": ([_vp, ctypes.POINTER(HsKcParams)], ctypes.c_int),
    "hs_workspace_size": ([ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hs_workspace_reset": ([_vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "hs_obs_prepare": ([ctypes.POINTER(HsObs), _vp], ctypes.c_int),
    "pose_fk": ([_vp, _vp, ctypes.c_int, ctypes.POINTER(HsCamera), _vp, _vp, _vp], ctypes.c_int),
    "render_score_batch": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), _vp, _vp, ctypes.c_int,
                            ctypes.POINTER(HsScoreParams), _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp, _vp],
                           ctypes.c_int),
    "pso_init": ([_vp, ctypes.POINTER(HsSwarm), ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_float),
                  ctypes.c_uint64, ctypes.c_uint32, _vp], ctypes.c_int),
    "pso_step": ([_vp, ctypes.POINTER(HsSwarm), ctypes.c_int, ctypes.POINTER(HsPsoParams), ctypes.c_uint64,
                  ctypes.c_uint32, ctypes.c_uint32, _vp], ctypes.c_int),
    "hs_get_device_status": ([ctypes.POINTER(ctypes.c_uint32), ctypes.c_int], ctypes.c_int),
    "pso_step_fk": ([_vp, ctypes.POINTER(HsSwarm), _vp, ctypes.c_int, ctypes.POINTER(HsPsoParams), ctypes.c_uint64,
                     ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(HsCamera), _vp, _vp, _vp], ctypes.c_int),
    "render_score_batch_noalloc": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), _vp, _vp, ctypes.c_int,
                                    ctypes.POINTER(HsScoreParams), _vp, _vp, _vp], ctypes.c_int),
    "hs_render_variant": ([ctypes.POINTER(HsScoreParams), ctypes.c_int], ctypes.c_int),
    "render_score_batch_autotune": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), _vp, _vp, ctypes.c_int,
                                     ctypes.POINTER(HsScoreParams), _vp, ctypes.c_size_t, _vp, ctypes.c_int, _vp, _vp],
                                    ctypes.c_int),
    "render_score_multi_autotune": ([_vp, _vp, _vp, _vp, ctypes.POINTER(HsScoreParams), _vp, ctypes.c_size_t, _vp,
                                     ctypes.c_int, _vp, _vp], ctypes.c_int),
    "soft_score": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), _vp, _vp, ctypes.c_int,
                    ctypes.POINTER(HsScoreParams), ctypes.POINTER(HsSoftParams), _vp, ctypes.c_size_t, _vp, _vp, _vp],
                   ctypes.c_int),
    "soft_score_backward": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), _vp, ctypes.c_int,
                             ctypes.POINTER(HsScoreParams), ctypes.POINTER(HsSoftParams), _vp, _vp, _vp],
                            ctypes.c_int),
    "pose_grad": ([_vp, _vp, ctypes.c_int, ctypes.POINTER(HsCamera), ctypes.POINTER(HsScoreParams), _vp, _vp, _vp,
                   _vp, _vp], ctypes.c_int),
    "polish_select": ([_vp, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "polish_gather": ([_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "polish_step": ([_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp],
                    ctypes.c_int),
    "polish_keep_better": ([_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "hs_batch_buffer_size": ([ctypes.POINTER(HsSwarmDesc), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
                             ctypes.c_int),
    "hs_batch_create": ([_vp, ctypes.POINTER(HsSwarmDesc), ctypes.c_int, _vp, ctypes.c_size_t, _vp,
                         ctypes.POINTER(_vp)], ctypes.c_int),
    "hs_batch_destroy": ([_vp], ctypes.c_int),
    "hs_batch_particles": ([_vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "hs_obs_prepare_multi": ([_vp, _vp], ctypes.c_int),
    "pose_fk_multi": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "render_score_multi": ([_vp, _vp, _vp, _vp, ctypes.POINTER(HsScoreParams), _vp, ctypes.c_size_t, _vp, _vp, _vp],
                           ctypes.c_int),
    "pso_init_multi": ([_vp, _vp, ctypes.POINTER(HsSwarm), _vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32,
                        _vp], ctypes.c_int),
    "pso_step_fk_multi": ([_vp, _vp, ctypes.POINTER(HsSwarm), _vp, ctypes.POINTER(HsPsoParams), ctypes.c_uint32,
                           ctypes.c_uint32, _vp, _vp, _vp], ctypes.c_int),
    "hs_frame_workspace_size": ([ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hs_frame_capacity": ([ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "track_frame": ([_vp, ctypes.POINTER(HsObs), ctypes.POINTER(HsCamera), ctypes.POINTER(HsSwarm), _vp, ctypes.c_int,
                     ctypes.c_int, ctypes.POINTER(HsScoreParams), ctypes.POINTER(HsPsoParams), _vp,
                     ctypes.POINTER(ctypes.c_float), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _vp,
                     ctypes.c_size_t, _vp, _vp, _vp], ctypes.c_int),
    "hs_frame_multi_workspace_size": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hs_frame_multi_capacity": ([_vp, _vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "track_frame_multi": ([_vp, _vp, ctypes.POINTER(HsSwarm), _vp, ctypes.c_int, ctypes.POINTER(HsScoreParams),
                           ctypes.POINTER(HsPsoParams), _vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32,
                           ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp, _vp], ctypes.c_int),
}
NOALLOC_SCRATCH_BYTES = 256 * 1024
MAX_PRIMS = 64
MAX_PARTICLES = 65535
FUSED_MAX_PARTICLES = 4096
FRAME_MAX_PARTICLES = 1024

_LIB = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2005_07068_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


class HandscoreError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {lib().hs_status_string(status).decode()} ({status})")
        self.status = status


def _check(fn: str, status: int) -> None:
    if status != HS_OK:
        raise HandscoreError(fn, status)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---- model ------------------------------------------------------------------------

class Model:
    """A validated hand model (host object; passed to kernels by value)."""

    def __init__(self, bones_i, bones_f, prims_i, prims_f, lo, hi):
        nb, npr = len(bones_i), len(prims_i)
        self._bones = (HsBoneDesc * nb)()
        for b in range(nb):
            B = self._bones[b]
            B.parent, B.dof_z, B.dof_x = (int(v) for v in bones_i[b])
            B.offset[:] = [float(v) for v in bones_f[b][:3]]
            B.rest[:] = [float(v) for v in bones_f[b][3:6]]
        self._prims = (HsPrimDesc * npr)()
        for k in range(npr):
            Pd = self._prims[k]
            Pd.bone, Pd.kind = (int(v) for v in prims_i[k])
            Pd.center[:] = [float(v) for v in prims_f[k][:3]]
            Pd.dims[:] = [float(v) for v in prims_f[k][3:7]]
        d = HsModelDesc()
        d.n_bones, d.n_prims = nb, npr
        d.bones = ctypes.cast(self._bones, ctypes.POINTER(HsBoneDesc))
        d.prims = ctypes.cast(self._prims, ctypes.POINTER(HsPrimDesc))
        d.lo[:] = [float(v) for v in lo]
        d.hi[:] = [float(v) for v in hi]
        h = _vp()
        _check("hs_model_create", lib().hs_model_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_prims = npr
        self.lo = np.asarray(lo, np.float32)
        self.hi = np.asarray(hi, np.float32)

    @classmethod
    def from_geometry(cls, g, lo, hi) -> "Model":
        return cls(g.bones_i, g.bones_f, g.prims_i, g.prims_f, lo, hi)

    def set_kc(self, variant: int = HS_KC_ABDUCTION, pen_weight: float = 0.0) -> "Model":
        """Select the kc variant: the paper's abduction ordering, that plus
        pen_weight x the interpenetration of different fingers (mm), or the
        interpenetration term alone."""
        _check("hs_model_set_kc", lib().hs_model_set_kc(self.handle, ctypes.byref(HsKcParams(variant, pen_weight))))
        self.kc_variant, self.pen_weight = variant, pen_weight
        return self

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _LIB is not None:
            _LIB.hs_model_destroy(h)
            self.handle = None


def camera(fx, fy, cx, cy) -> HsCamera:
    return HsCamera(fx, fy, cx, cy)


def render_variant(params: HsScoreParams, P: int) -> str:
    """Name of the render kernel a call over P particles runs with these parameters."""
    v = lib().hs_render_variant(ctypes.byref(params), int(P))
    _check("hs_render_variant", min(v, 0))
    return {i: n for n, i in RENDER_VARIANTS.items()}[v]


def score_params(d_m=10.0, d_M=40.0, lam=20.0, lam_k=10.0, variant=RENDER_AUTO, ctas_per_particle=0
                 ) -> HsScoreParams:
    """Eq. 4-5 constants (Section III.A: 1 cm, 4 cm, 20, 10) in mm, and the render's
    launch shape (kernel variant, CTAs per particle; neither changes results)."""
    return HsScoreParams(d_m, d_M, lam, lam_k, int(variant), int(ctas_per_particle))


def pso_params(c1=2.8, c2=1.3, mutate_every=3, n_mutate=None, P=None, e_stop=0.0) -> HsPsoParams:
    """Section III.B constants; n_mutate defaults to half the swarm; e_stop > 0
    (batch steps only) stops a swarm once its best E falls below it."""
    if n_mutate is None:
        n_mutate = (P or 0) // 2
    return HsPsoParams(c1, c2, mutate_every, n_mutate, e_stop)


# ---- observation ----------------------------------------------------------------------

@dataclass
class Obs:
    """Device observation: depth [H, pitch] (uint16 or float32, row pitch a multiple of
    16 bytes), skin [H, pitch] uint8, ROI W x H, and a 2-word stats buffer."""
    depth: torch.Tensor
    skin: torch.Tensor
    W: int
    H: int
    stats: torch.Tensor

    def struct(self) -> HsObs:
        dt = HS_DEPTH_F32 if self.depth.dtype == torch.float32 else HS_DEPTH_U16
        return HsObs(_ptr(self.depth), _ptr(self.skin), self.W, self.H,
                     self.depth.stride(0) * self.depth.element_size(), self.skin.stride(0), dt, _ptr(self.stats))

    @classmethod
    def from_numpy(cls, depth: np.ndarray, skin: np.ndarray, device="cuda") -> "Obs":
        from .inputs import pitched
        H, W = depth.shape
        d = torch.from_numpy(pitched(depth)).to(device)
        s = torch.from_numpy(pitched(skin.astype(np.uint8))).to(device)
        return cls(d, s, W, H, torch.zeros(2, dtype=torch.int32, device=device))


def hs_obs_prepare(obs: Obs, stream=None) -> None:
    st = obs.struct()
    _check("hs_obs_prepare", lib().hs_obs_prepare(ctypes.byref(st), _stream(stream)))


def workspace_size(P: int) -> int:
    n = ctypes.c_size_t(0)
    _check("hs_workspace_size", lib().hs_workspace_size(P, ctypes.byref(n)))
    return n.value


def new_workspace(P: int, device="cuda") -> torch.Tensor:
    """A zeroed workspace tensor (uint8) for render_score_batch."""
    return torch.zeros(max(workspace_size(P), 16), dtype=torch.uint8, device=device)


def hs_workspace_reset(ws: torch.Tensor, stream=None) -> None:
    _check("hs_workspace_reset", lib().hs_workspace_reset(_ptr(ws), ws.numel(), _stream(stream)))


# ---- the hot path ------------------------------------------------------------------------

def pose_fk(model: Model, poses: torch.Tensor, cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor,
            stream=None) -> None:
    """poses [P, 26] f32 -> prims [P, n_prims, 16] f32 records, kc [P]."""
    P = poses.shape[0]
    _check("pose_fk", lib().pose_fk(model.handle, _ptr(poses), P, ctypes.byref(cam), _ptr(prims), _ptr(kc),
                                    _stream(stream)))


def render_score_batch(model: Model, obs: Obs, cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor,
                       params: HsScoreParams, ws: torch.Tensor, E: torch.Tensor, parts: torch.Tensor | None = None,
                       dbg_depth: torch.Tensor | None = None, dbg_mask: torch.Tensor | None = None,
                       stream=None) -> None:
    """Fused render + Eq. 4-5: E [P]; parts [P, 4] int32 view of HsParts (optional);
    dbg_depth [P, H, W] f32 and dbg_mask [P, H, W] uint8 (optional)."""
    P = kc.shape[0]
    st = obs.struct()
    _check("render_score_batch",
           lib().render_score_batch(model.handle, ctypes.byref(st), ctypes.byref(cam), _ptr(prims), _ptr(kc), P,
                                    ctypes.byref(params), _ptr(ws), ws.numel(), _ptr(E), _ptr(parts),
                                    _ptr(dbg_depth), _ptr(dbg_mask), _stream(stream)))


def render_score_batch_noalloc(model: Model, obs: Obs, cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor,
                               params: HsScoreParams, E: torch.Tensor, parts: torch.Tensor | None = None,
                               stream=None) -> None:
    """render_score_batch without a caller workspace: for callers that cannot
    allocate device memory.  The scratch is a fixed array inside the library
    (one per GPU, NOALLOC_SCRATCH_BYTES); calls that overlap on the GPU race."""
    P = kc.shape[0]
    st = obs.struct()
    _check("render_score_batch_noalloc",
           lib().render_score_batch_noalloc(model.handle, ctypes.byref(st), ctypes.byref(cam), _ptr(prims),
                                            _ptr(kc), P, ctypes.byref(params), _ptr(E), _ptr(parts),
                                            _stream(stream)))


@dataclass
class Swarm:
    """Device swarm state (float32): x, v, pbest [P, 26]; pbest_E [P]; gbest [26];
    gbest_E [1]; E [P]."""
    x: torch.Tensor
    v: torch.Tensor
    pbest: torch.Tensor
    pbest_E: torch.Tensor
    gbest: torch.Tensor
    gbest_E: torch.Tensor
    E: torch.Tensor

    @classmethod
    def empty(cls, P: int, device="cuda") -> "Swarm":
        f = dict(dtype=torch.float32, device=device)
        return cls(torch.zeros(P, NDOF, **f), torch.zeros(P, NDOF, **f), torch.zeros(P, NDOF, **f),
                   torch.zeros(P, **f), torch.zeros(NDOF, **f), torch.zeros(1, **f), torch.zeros(P, **f))

    @property
    def P(self) -> int:
        return self.x.shape[0]

    def struct(self) -> HsSwarm:
        return HsSwarm(*(_ptr(t) for t in (self.x, self.v, self.pbest, self.pbest_E, self.gbest, self.gbest_E,
                                           self.E)))


def pso_init(model: Model, sw: Swarm, seed_pose: torch.Tensor, scale, seed: int, frame: int, stream=None) -> None:
    st = sw.struct()
    sc = (ctypes.c_float * NDOF)(*[float(v) for v in scale])
    _check("pso_init", lib().pso_init(model.handle, ctypes.byref(st), sw.P, _ptr(seed_pose), sc,
                                      ctypes.c_uint64(seed), frame, _stream(stream)))


def pso_step(model: Model, sw: Swarm, params: HsPsoParams, seed: int, frame: int, gen: int, stream=None) -> None:
    st = sw.struct()
    _check("pso_step", lib().pso_step(model.handle, ctypes.byref(st), sw.P, ctypes.byref(params),
                                      ctypes.c_uint64(seed), frame, gen, _stream(stream)))


def pso_step_fk(model: Model, sw: Swarm, x_next: torch.Tensor, params: HsPsoParams, seed: int, frame: int, gen: int,
                cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor, stream=None) -> None:
    """pso_step then pose_fk of the new positions, in one launch; the new
    positions go to x_next (sw.x is only read)."""
    st = sw.struct()
    _check("pso_step_fk", lib().pso_step_fk(model.handle, ctypes.byref(st), _ptr(x_next), sw.P, ctypes.byref(params),
                                            ctypes.c_uint64(seed), frame, gen, ctypes.byref(cam), _ptr(prims),
                                            _ptr(kc), _stream(stream)))


# ---- a whole tracking frame in one launch ---------------------------------------------

def new_frame_workspace(P: int, device="cuda") -> torch.Tensor:
    """Zeroed workspace of track_frame for P particles: a control block and
    three generations of per-particle sums, which every call leaves zeroed."""
    n = ctypes.c_size_t()
    _check("hs_frame_workspace_size", lib().hs_frame_workspace_size(P, ctypes.byref(n)))
    return torch.zeros((n.value + 15) // 16 * 4, dtype=torch.int32, device=device)


def frame_capacity() -> int:
    """CTAs of track_frame the current device keeps resident at once."""
    n = ctypes.c_int()
    _check("hs_frame_capacity", lib().hs_frame_capacity(ctypes.byref(n)))
    return n.value


def track_frame(model: Model, obs: Obs, cam: HsCamera, sw: Swarm, x_next: torch.Tensor, gens: int,
                score: HsScoreParams, pso: HsPsoParams, seed_pose: torch.Tensor, scale, seed: int, frame: int,
                ctas: int, ws: torch.Tensor, kc: torch.Tensor, prims: torch.Tensor | None = None,
                stream=None) -> None:
    """One whole frame (obs totals, init around seed_pose, gens x (score, step)) in
    one cooperative launch of `ctas` CTAs (0: automatic), dealt evenly to the
    particles for the whole frame; identical to the step-by-step calls.
    Generation g writes positions to (sw.x, x_next)[g & 1]."""
    st = sw.struct()
    sc = (ctypes.c_float * NDOF)(*[float(v) for v in np.asarray(scale, np.float32)])
    _check("track_frame", lib().track_frame(model.handle, ctypes.byref(obs.struct()), ctypes.byref(cam),
                                            ctypes.byref(st), _ptr(x_next), sw.P, gens, ctypes.byref(score),
                                            ctypes.byref(pso), _ptr(seed_pose), sc, ctypes.c_uint64(seed), frame,
                                            ctas, _ptr(ws), ws.numel() * ws.element_size(),
                                            _ptr(prims), _ptr(kc), _stream(stream)))


# ---- the smoothed objective E_s and its gradient ------------------------------------

def soft_params(tau_px: float = 0.5, tau_mm: float = 0.5, ctas_per_particle: int = 0) -> HsSoftParams:
    return HsSoftParams(tau_px, tau_mm, int(ctas_per_particle), 0)


def soft_score(model: Model, obs: Obs, cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor, params: HsScoreParams,
               soft: HsSoftParams, ws: torch.Tensor, E_s: torch.Tensor, sums: torch.Tensor | None = None,
               stream=None) -> None:
    """E_s [P] of the records prims [P, n_prims, 16]; sums [P, 3] for the backward pass."""
    st = obs.struct()
    _check("soft_score", lib().soft_score(model.handle, ctypes.byref(st), ctypes.byref(cam), _ptr(prims), _ptr(kc),
                                          kc.shape[0], ctypes.byref(params), ctypes.byref(soft), _ptr(ws), ws.numel(),
                                          _ptr(E_s), _ptr(sums), _stream(stream)))


def soft_score_backward(model: Model, obs: Obs, cam: HsCamera, prims: torch.Tensor, params: HsScoreParams,
                        soft: HsSoftParams, sums: torch.Tensor, adj: torch.Tensor, stream=None) -> None:
    """Adds dE_s/d(records) to adj [P, n_prims, SOFT_ADJ] int64 (fixed point 2^-40, zero on entry)."""
    st = obs.struct()
    _check("soft_score_backward",
           lib().soft_score_backward(model.handle, ctypes.byref(st), ctypes.byref(cam), _ptr(prims), prims.shape[0],
                                     ctypes.byref(params), ctypes.byref(soft), _ptr(sums), _ptr(adj), _stream(stream)))


def pose_grad(model: Model, poses: torch.Tensor, cam: HsCamera, params: HsScoreParams, prims: torch.Tensor,
              kc: torch.Tensor, adj: torch.Tensor, grad: torch.Tensor, stream=None) -> None:
    """grad [P, 26] = dE_s/dpose from the record adjoints (adj is cleared)."""
    _check("pose_grad", lib().pose_grad(model.handle, _ptr(poses), poses.shape[0], ctypes.byref(cam),
                                        ctypes.byref(params), _ptr(prims), _ptr(kc), _ptr(adj), _ptr(grad),
                                        _stream(stream)))


# ---- gradient polish of the best particles ---------------------------------------------

def polish_select(E: torch.Tensor, k: int, sel: torch.Tensor, stream=None) -> None:
    """sel [k] int32 <- indices of the k lowest E (lower index on ties, NaN last)."""
    _check("polish_select", lib().polish_select(_ptr(E), E.shape[0], int(k), _ptr(sel), _stream(stream)))


def polish_gather(x: torch.Tensor, E: torch.Tensor, sel: torch.Tensor, x_sel: torch.Tensor, E_sel: torch.Tensor,
                  stream=None) -> None:
    _check("polish_gather", lib().polish_gather(_ptr(x), _ptr(E), _ptr(sel), sel.shape[0], _ptr(x_sel), _ptr(E_sel),
                                                _stream(stream)))


def polish_step(model: Model, x_sel: torch.Tensor, grad: torch.Tensor, eta: float, scale, stream=None) -> None:
    sc = (ctypes.c_float * NDOF)(*[float(v) for v in scale])
    _check("polish_step", lib().polish_step(model.handle, _ptr(x_sel), _ptr(grad), x_sel.shape[0], float(eta), sc,
                                            _stream(stream)))


def polish_keep_better(x: torch.Tensor, E: torch.Tensor, sel: torch.Tensor, x_sel: torch.Tensor, E_old: torch.Tensor,
                       E_new: torch.Tensor, stream=None) -> None:
    _check("polish_keep_better", lib().polish_keep_better(_ptr(x), _ptr(E), _ptr(sel), sel.shape[0], _ptr(x_sel),
                                                          _ptr(E_old), _ptr(E_new), _stream(stream)))


# ---- batches of independent swarms ---------------------------------------------------

class Batch:
    """S independent swarms (sequences) scored and stepped together, one launch per
    kernel: each with its own observation, camera, particle count and Philox key.
    Particle arrays are concatenated over the swarms; gbest is [S, 26], gbest_E [S]."""

    def __init__(self, model: Model, obs: list, cams: list, P: list, seeds: list, n_mutate: list | None = None,
                 device="cuda", stream=None):
        S = len(obs)
        if not (len(cams) == len(P) == len(seeds) == S):
            raise ValueError("one observation, camera, particle count and seed per swarm")
        if n_mutate is None:
            n_mutate = [p // 2 for p in P]
        descs = (HsSwarmDesc * S)()
        for s in range(S):
            descs[s] = HsSwarmDesc(obs[s].struct(), cams[s], int(P[s]), int(n_mutate[s]), ctypes.c_uint64(seeds[s]))
        n = ctypes.c_size_t(0)
        _check("hs_batch_buffer_size", lib().hs_batch_buffer_size(descs, S, ctypes.byref(n)))
        self.buffer = torch.zeros(n.value, dtype=torch.uint8, device=device)
        h = _vp()
        _check("hs_batch_create", lib().hs_batch_create(model.handle, descs, S, _ptr(self.buffer), n.value,
                                                        _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.obs = list(obs)  # the bound buffers stay alive with the batch
        self.S = S
        self.P = [int(p) for p in P]
        self.offsets = np.concatenate([[0], np.cumsum(self.P)]).astype(np.int64)
        self.P_total = int(self.offsets[-1])

    def set_kc(self, variant: int = HS_KC_ABDUCTION, pen_weight: float = 0.0) -> "Model":
        """Select the kc variant: the paper's abduction ordering, that plus
        pen_weight x the interpenetration of different fingers (mm), or the
        interpenetration term alone."""
        _check("hs_model_set_kc", lib().hs_model_set_kc(self.handle, ctypes.byref(HsKcParams(variant, pen_weight))))
        self.kc_variant, self.pen_weight = variant, pen_weight
        return self

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _LIB is not None:
            _LIB.hs_batch_destroy(h)
            self.handle = None


def hs_obs_prepare_multi(batch: Batch, stream=None) -> None:
    _check("hs_obs_prepare_multi", lib().hs_obs_prepare_multi(batch.handle, _stream(stream)))


def pose_fk_multi(model: Model, batch: Batch, poses: torch.Tensor, prims: torch.Tensor, kc: torch.Tensor,
                  stream=None) -> None:
    """poses [P_total, 26] -> prims [P_total, n_prims, 16], kc [P_total], each with its swarm's camera."""
    _check("pose_fk_multi", lib().pose_fk_multi(model.handle, batch.handle, _ptr(poses), _ptr(prims), _ptr(kc),
                                                _stream(stream)))


def render_score_multi(model: Model, batch: Batch, prims: torch.Tensor, kc: torch.Tensor, params: HsScoreParams,
                       ws: torch.Tensor, E: torch.Tensor, parts: torch.Tensor | None = None, stream=None) -> None:
    """E [P_total]: every particle scored against its own swarm's observation."""
    _check("render_score_multi",
           lib().render_score_multi(model.handle, batch.handle, _ptr(prims), _ptr(kc), ctypes.byref(params),
                                    _ptr(ws), ws.numel(), _ptr(E), _ptr(parts), _stream(stream)))


def pso_init_multi(model: Model, batch: Batch, sw: Swarm, seed_poses: torch.Tensor, scale, frame: int,
                   stream=None) -> None:
    """seed_poses [S, 26] device; sw holds [P_total] particle arrays, gbest [S, 26], gbest_E [S]."""
    st = sw.struct()
    sc = (ctypes.c_float * NDOF)(*[float(v) for v in scale])
    _check("pso_init_multi", lib().pso_init_multi(model.handle, batch.handle, ctypes.byref(st), _ptr(seed_poses), sc,
                                                  frame, _stream(stream)))


def pso_step_fk_multi(model: Model, batch: Batch, sw: Swarm, x_next: torch.Tensor, params: HsPsoParams, frame: int,
                      gen: int, prims: torch.Tensor, kc: torch.Tensor, stream=None) -> None:
    st = sw.struct()
    _check("pso_step_fk_multi",
           lib().pso_step_fk_multi(model.handle, batch.handle, ctypes.byref(st), _ptr(x_next), ctypes.byref(params),
                                   frame, gen, _ptr(prims), _ptr(kc), _stream(stream)))


def batch_swarm(batch: Batch, device="cuda") -> Swarm:
    """Zeroed swarm state for a batch: [P_total] particle arrays, [S] global bests."""
    f = dict(dtype=torch.float32, device=device)
    Pt, S = batch.P_total, batch.S
    return Swarm(torch.zeros(Pt, NDOF, **f), torch.zeros(Pt, NDOF, **f), torch.zeros(Pt, NDOF, **f),
                 torch.zeros(Pt, **f), torch.zeros(S, NDOF, **f), torch.zeros(S, **f), torch.zeros(Pt, **f))


def new_frame_multi_workspace(batch: Batch, device="cuda") -> torch.Tensor:
    """Zeroed workspace of track_frame_multi for a batch: a control block and a
    count per swarm, which every call leaves zeroed, then two generations of E."""
    n = ctypes.c_size_t()
    _check("hs_frame_multi_workspace_size", lib().hs_frame_multi_workspace_size(batch.handle, ctypes.byref(n)))
    return torch.zeros((n.value + 15) // 16 * 4, dtype=torch.int32, device=device)


def frame_multi_capacity(batch: Batch | None = None, model: Model | None = None) -> int:
    """CTAs of track_frame_multi the current device keeps resident at once for
    this batch (None: for any batch) and model (None: any model with the
    paper's kc; a kc variant with the interpenetration test leaves room for
    fewer)."""
    n = ctypes.c_int()
    _check("hs_frame_multi_capacity",
           lib().hs_frame_multi_capacity(model.handle if model is not None else None,
                                         batch.handle if batch is not None else None, ctypes.byref(n)))
    return n.value


def track_frame_multi(model: Model, batch: Batch, sw: Swarm, x_next: torch.Tensor, gens: int, score: HsScoreParams,
                      pso: HsPsoParams, seed_poses: torch.Tensor, scale, frame: int, ctas: int, ws: torch.Tensor,
                      prims: torch.Tensor, kc: torch.Tensor, stream=None) -> None:
    """A whole frame of every swarm of the batch (obs totals, init around
    seed_poses [S, 26], gens x (score, step)) in one cooperative launch of
    `ctas` CTAs (0: the capacity) taking per-particle tasks; identical to the
    step-by-step batch calls.  Step g writes positions to (sw.x, x_next)[g & 1]."""
    st = sw.struct()
    sc = (ctypes.c_float * NDOF)(*[float(v) for v in np.asarray(scale, np.float32)])
    _check("track_frame_multi",
           lib().track_frame_multi(model.handle, batch.handle, ctypes.byref(st), _ptr(x_next), gens,
                                   ctypes.byref(score), ctypes.byref(pso), _ptr(seed_poses), sc, frame, ctas,
                                   _ptr(ws), ws.numel() * ws.element_size(), _ptr(prims), _ptr(kc),
                                   _stream(stream)))


TUNE_CTAS = (0, 1, 2, 3, 4, 6, 8, 16, 32)  # 0: the automatic choice


def _tune_table(times) -> dict:
    names = {i: n for n, i in RENDER_VARIANTS.items()}
    out = {}
    for v in range(1, len(RENDER_VARIANTS)):
        for c, k in enumerate(TUNE_CTAS):
            t = times[v * len(TUNE_CTAS) + c]
            if t >= 0:
                out[f"{names[v]}/k{k}"] = float(t)
    return out


def render_score_batch_autotune(model: Model, obs: Obs, cam: HsCamera, prims: torch.Tensor, kc: torch.Tensor,
                                params: HsScoreParams, ws: torch.Tensor, E: torch.Tensor, reps: int = 5,
                                stream=None) -> tuple[HsScoreParams, dict]:
    """The fastest render launch shape for these inputs: (params with variant and
    CTAs per particle set, {candidate: microseconds per call})."""
    out = HsScoreParams(*[getattr(params, f) for f, _ in HsScoreParams._fields_])
    times = (ctypes.c_float * (len(RENDER_VARIANTS) * len(TUNE_CTAS)))()
    st = obs.struct()
    _check("render_score_batch_autotune",
           lib().render_score_batch_autotune(model.handle, ctypes.byref(st), ctypes.byref(cam), _ptr(prims), _ptr(kc),
                                             kc.shape[0], ctypes.byref(out), _ptr(ws), ws.numel(), _ptr(E), reps,
                                             times, _stream(stream)))
    return out, _tune_table(times)


def render_score_multi_autotune(model: Model, batch: "Batch", prims: torch.Tensor, kc: torch.Tensor,
                                params: HsScoreParams, ws: torch.Tensor, E: torch.Tensor, reps: int = 5,
                                stream=None) -> tuple[HsScoreParams, dict]:
    out = HsScoreParams(*[getattr(params, f) for f, _ in HsScoreParams._fields_])
    times = (ctypes.c_float * (len(RENDER_VARIANTS) * len(TUNE_CTAS)))()
    _check("render_score_multi_autotune",
           lib().render_score_multi_autotune(model.handle, batch.handle, _ptr(prims), _ptr(kc), ctypes.byref(out),
                                             _ptr(ws), ws.numel(), _ptr(E), reps, times, _stream(stream)))
    return out, _tune_table(times)


def hs_get_device_status(clear: bool = False) -> int:
    v = ctypes.c_uint32(0)
    _check("hs_get_device_status", lib().hs_get_device_status(ctypes.byref(v), int(clear)))
    return v.value


def version() -> int:
    return lib().hs_version()
