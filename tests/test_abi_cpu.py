"""The C-ABI boundary on CPU: the library loads, exports every function that
include/handscore.h declares, its structs have the C layout, and invalid calls
are rejected on the host before anything reaches a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "handscore.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert {"pose_fk", "render_score_batch", "pso_step", "pso_init", "hs_obs_prepare"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", hs.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = hs.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "handscore.h"
#define S(t) printf(#t " %zu\\n", sizeof(t));
#define O(t, f) printf(#t "." #f " %zu\\n", offsetof(t, f));
int main(void) {
  S(HsBoneDesc) S(HsPrimDesc) S(HsModelDesc) S(HsCamera) S(HsObs) S(HsScoreParams) S(HsParts)
  S(HsPrim) S(HsSwarm) S(HsPsoParams) S(HsSwarmDesc)
  O(HsSwarmDesc, cam) O(HsSwarmDesc, P) O(HsSwarmDesc, seed)
  O(HsModelDesc, bones) O(HsModelDesc, lo) O(HsModelDesc, hi) O(HsObs, stats) O(HsObs, depth_type)
  O(HsBoneDesc, rest) O(HsPrimDesc, dims) O(HsSwarm, E)
  printf("HS_NOALLOC_SCRATCH_BYTES %d\\n", (int)HS_NOALLOC_SCRATCH_BYTES);
  printf("HS_FUSED_MAX_PARTICLES %d\\n", (int)HS_FUSED_MAX_PARTICLES);
  printf("HS_MAX_PARTICLES %d\\n", (int)HS_MAX_PARTICLES);
  printf("HS_MAX_PRIMS %d\\n", (int)HS_MAX_PRIMS);
  printf("HS_FRAME_MAX_PARTICLES %d\\n", (int)HS_FRAME_MAX_PARTICLES);
  printf("HS_TUNE_CTAS %d\\n", (int)HS_TUNE_CTAS);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = dict(ln.rsplit(" ", 1) for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    py = {
        "HsBoneDesc": ctypes.sizeof(hs.HsBoneDesc), "HsPrimDesc": ctypes.sizeof(hs.HsPrimDesc),
        "HsModelDesc": ctypes.sizeof(hs.HsModelDesc), "HsCamera": ctypes.sizeof(hs.HsCamera),
        "HsObs": ctypes.sizeof(hs.HsObs), "HsScoreParams": ctypes.sizeof(hs.HsScoreParams),
        "HsParts": 16, "HsPrim": 64, "HsSwarm": ctypes.sizeof(hs.HsSwarm),
        "HsPsoParams": ctypes.sizeof(hs.HsPsoParams), "HsSwarmDesc": ctypes.sizeof(hs.HsSwarmDesc),
        "HsSwarmDesc.cam": hs.HsSwarmDesc.cam.offset, "HsSwarmDesc.P": hs.HsSwarmDesc.P.offset,
        "HsSwarmDesc.seed": hs.HsSwarmDesc.seed.offset,
        "HsModelDesc.bones": hs.HsModelDesc.bones.offset, "HsModelDesc.lo": hs.HsModelDesc.lo.offset,
        "HsModelDesc.hi": hs.HsModelDesc.hi.offset, "HsObs.stats": hs.HsObs.stats.offset,
        "HsObs.depth_type": hs.HsObs.depth_type.offset, "HsBoneDesc.rest": hs.HsBoneDesc.rest.offset,
        "HsPrimDesc.dims": hs.HsPrimDesc.dims.offset, "HsSwarm.E": hs.HsSwarm.E.offset,
        # constants the binding repeats
        "HS_NOALLOC_SCRATCH_BYTES": hs.NOALLOC_SCRATCH_BYTES, "HS_FUSED_MAX_PARTICLES": hs.FUSED_MAX_PARTICLES,
        "HS_MAX_PARTICLES": hs.MAX_PARTICLES, "HS_FRAME_MAX_PARTICLES": hs.FRAME_MAX_PARTICLES,
        "HS_MAX_PRIMS": hs.MAX_PRIMS, "HS_TUNE_CTAS": len(hs.TUNE_CTAS),
    }
    for k, v in py.items():
        assert int(got[k]) == v, k


def _model():
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    return hs.Model.from_geometry(g, lo, hi)


def test_model_validation():
    m = _model()
    assert m.handle
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    bad_parent = g.bones_i.copy()
    bad_parent[5, 0] = 7
    with pytest.raises(hs.HandscoreError) as e:
        hs.Model(bad_parent, g.bones_f, g.prims_i, g.prims_f, lo, hi)
    assert e.value.status == hs.HS_ERR_ARG
    bad_kappa = g.prims_f.copy()
    bad_kappa[0, 6] = 1.0
    with pytest.raises(hs.HandscoreError):
        hs.Model(g.bones_i, g.bones_f, g.prims_i, bad_kappa, lo, hi)
    bad_dim = g.prims_f.copy()
    bad_dim[3, 3] = 0.0
    with pytest.raises(hs.HandscoreError):
        hs.Model(g.bones_i, g.bones_f, g.prims_i, bad_dim, lo, hi)
    with pytest.raises(hs.HandscoreError):
        hs.Model(g.bones_i, g.bones_f, g.prims_i, g.prims_f, hi, lo)  # lo > hi
    L = hs.lib()
    assert L.hs_model_create(None, None) == hs.HS_ERR_ARG


def test_model_chain_depth_limit():
    """Bone chains up to HS_MAX_DEPTH (7) below the palm are accepted, deeper
    ones are refused with HS_ERR_SIZE (FK composes each bone's path from the
    palm in one pass, from a table of at most 8 ancestors)."""
    g = I.hand_geometry()
    lo, hi = I.search_limits()
    for depth, ok in ((7, True), (8, False)):
        bi = np.zeros((depth + 1, 3), np.int32)
        bi[:, 1:] = -1           # no degrees of freedom
        bi[1:, 0] = np.arange(depth)  # bone b hangs from bone b - 1
        bf = np.zeros((depth + 1, 6), np.float32)
        bf[1:, 1] = 10.0         # 10 mm along y per bone
        pi = np.array([[depth, g.prims_i[0, 1]]], np.int32)
        pf = g.prims_f[:1].copy()
        if ok:
            assert hs.Model(bi, bf, pi, pf, lo, hi).handle
        else:
            with pytest.raises(hs.HandscoreError) as e:
                hs.Model(bi, bf, pi, pf, lo, hi)
            assert e.value.status == hs.HS_ERR_SIZE


def test_workspace_size():
    n = hs.workspace_size(64)
    assert n >= 64 * 16
    with pytest.raises(hs.HandscoreError):
        hs.workspace_size(-1)
    with pytest.raises(hs.HandscoreError):
        hs.workspace_size(1 << 20)
    assert hs.lib().hs_workspace_size(4, None) == hs.HS_ERR_ARG


FAKE = 0x10000  # a 16-byte aligned address that validation never dereferences


def _obs(**kw):
    o = hs.HsObs(FAKE, FAKE, 320, 240, 640, 320, hs.HS_DEPTH_U16, FAKE)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("kw,code", [
    (dict(depth_pitch=600), hs.HS_ERR_ALIGN),       # not a multiple of 16
    (dict(depth_pitch=320), hs.HS_ERR_SIZE),        # shorter than a row
    (dict(skin=FAKE + 4), hs.HS_ERR_ALIGN),         # misaligned base
    (dict(W=0), hs.HS_ERR_SIZE),
    (dict(H=9000), hs.HS_ERR_SIZE),
    (dict(depth_type=7), hs.HS_ERR_ARG),
    (dict(stats=None), hs.HS_ERR_ARG),
])
def test_render_score_rejects_bad_observation(kw, code):
    m = _model()
    L = hs.lib()
    cam = hs.camera(262.5, 262.5, 160, 120)
    prm = hs.score_params()
    o = _obs(**kw)
    rc = L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(prm),
                              FAKE, 1 << 20, FAKE, None, None, None, None)
    assert rc == code
    assert L.hs_obs_prepare(ctypes.byref(o), None) == code


def test_other_host_checks():
    m = _model()
    L = hs.lib()
    cam = hs.camera(262.5, 262.5, 160, 120)
    prm = hs.score_params()
    o = _obs()
    # workspace too small
    assert L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(prm),
                                FAKE, 16, FAKE, None, None, None, None) == hs.HS_ERR_SIZE
    # d_M beyond the fixed-point range
    big = hs.score_params(d_M=200.0)
    assert L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(big),
                                FAKE, 1 << 20, FAKE, None, None, None, None) == hs.HS_ERR_ARG
    # only one of the two debug outputs
    assert L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(prm),
                                FAKE, 1 << 20, FAKE, None, FAKE, None, None) == hs.HS_ERR_ARG
    bad_cam = hs.camera(0.0, 262.5, 160, 120)
    assert L.pose_fk(m.handle, FAKE, 4, ctypes.byref(bad_cam), FAKE, FAKE, None) == hs.HS_ERR_ARG
    assert L.pose_fk(m.handle, FAKE, 4, ctypes.byref(cam), FAKE + 8, FAKE, None) == hs.HS_ERR_ALIGN
    assert L.pose_fk(m.handle, FAKE, -1, ctypes.byref(cam), FAKE, FAKE, None) == hs.HS_ERR_SIZE
    assert L.pose_fk(m.handle, FAKE, 0, ctypes.byref(cam), FAKE, FAKE, None) == hs.HS_OK  # P = 0: no-op
    sw = hs.HsSwarm(FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    pp = hs.pso_params(P=64)
    assert L.pso_step(m.handle, ctypes.byref(sw), 5000, ctypes.byref(pp), 1, 0, 1, None) == hs.HS_ERR_SIZE
    low = hs.pso_params(c1=1.0, c2=1.0, P=64)  # psi <= 4: constriction undefined
    assert L.pso_step(m.handle, ctypes.byref(sw), 64, ctypes.byref(low), 1, 0, 1, None) == hs.HS_ERR_ARG
    sw.E = None
    assert L.pso_step(m.handle, ctypes.byref(sw), 64, ctypes.byref(pp), 1, 0, 1, None) == hs.HS_ERR_ARG
    scale = (ctypes.c_float * 26)(*([1.0] * 25 + [-1.0]))
    sw.E = FAKE
    assert L.pso_init(m.handle, ctypes.byref(sw), 64, FAKE, scale, 1, 0, None) == hs.HS_ERR_ARG
    assert L.hs_get_device_status(None, 0) == hs.HS_ERR_ARG
    sw.E = FAKE
    assert L.pso_step_fk(m.handle, ctypes.byref(sw), FAKE, 64, ctypes.byref(pp), 1, 0, 1, ctypes.byref(cam), FAKE,
                         FAKE, None) == hs.HS_ERR_ARG  # x_next aliases x
    assert L.pso_step_fk(m.handle, ctypes.byref(sw), FAKE + 4096, 5000, ctypes.byref(pp), 1, 0, 1, ctypes.byref(cam),
                         FAKE, FAKE, None) == hs.HS_ERR_SIZE
    assert hs.lib().hs_status_string(-3) == b"size out of range"
    # gradient polish and the smoothed objective: host checks
    assert L.polish_select(FAKE, 8, 9, FAKE, None) == hs.HS_ERR_SIZE   # k > P
    assert L.polish_select(FAKE, 8, 0, FAKE, None) == hs.HS_ERR_SIZE
    assert L.polish_select(None, 8, 4, FAKE, None) == hs.HS_ERR_ARG
    assert L.polish_gather(FAKE, FAKE, FAKE, 300, FAKE, FAKE, None) == hs.HS_ERR_SIZE
    bad_scale = (ctypes.c_float * 26)(*([1.0] * 25 + [0.0]))
    assert L.polish_step(m.handle, FAKE, FAKE, 4, 0.1, bad_scale, None) == hs.HS_ERR_ARG
    ok_scale = (ctypes.c_float * 26)(*([1.0] * 26))
    assert L.polish_step(m.handle, FAKE, FAKE, 4, -1.0, ok_scale, None) == hs.HS_ERR_ARG
    sp = hs.soft_params()
    bad_sp = hs.soft_params(tau_px=0.0)
    assert L.soft_score(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 4, ctypes.byref(prm),
                        ctypes.byref(bad_sp), FAKE, 1 << 20, FAKE, None, None) == hs.HS_ERR_ARG
    assert L.soft_score(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 4, ctypes.byref(prm),
                        ctypes.byref(sp), FAKE, 16, FAKE, None, None) == hs.HS_ERR_SIZE
    assert L.soft_score_backward(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, 4, ctypes.byref(prm),
                                 ctypes.byref(sp), None, FAKE, None) == hs.HS_ERR_ARG
    assert L.pose_grad(m.handle, FAKE, 4, ctypes.byref(cam), ctypes.byref(prm), FAKE + 8, FAKE, FAKE, FAKE,
                       None) == hs.HS_ERR_ALIGN
    # render launch shape: variant and CTAs per particle are validated; autotuning needs params and reps >= 1
    bad_v = hs.score_params(variant=len(hs.RENDER_VARIANTS))  # one past the last kernel
    assert L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(bad_v),
                                FAKE, 1 << 20, FAKE, None, None, None, None) == hs.HS_ERR_ARG
    bad_k = hs.score_params(ctas_per_particle=65)
    assert L.render_score_batch(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, ctypes.byref(bad_k),
                                FAKE, 1 << 20, FAKE, None, None, None, None) == hs.HS_ERR_ARG
    assert L.hs_render_variant(ctypes.byref(prm), 64) == hs.RENDER_UNITS
    assert L.hs_render_variant(ctypes.byref(prm), 5000) == hs.RENDER_TILES_64x32
    assert L.hs_render_variant(ctypes.byref(bad_v), 64) == hs.HS_ERR_ARG
    assert L.render_score_batch_autotune(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64, None, FAKE,
                                         1 << 20, FAKE, 3, None, None) == hs.HS_ERR_ARG
    assert L.render_score_batch_autotune(m.handle, ctypes.byref(o), ctypes.byref(cam), FAKE, FAKE, 64,
                                         ctypes.byref(prm), FAKE, 1 << 20, FAKE, 0, None, None) == hs.HS_ERR_ARG


def _descs(P, **obs_kw):
    S = len(P)
    d = (hs.HsSwarmDesc * S)()
    for s in range(S):
        d[s] = hs.HsSwarmDesc(_obs(**obs_kw), hs.camera(262.5, 262.5, 160, 120), P[s], P[s] // 2, 7 + s)
    return d


def test_batch_host_checks():
    m = _model()
    L = hs.lib()
    n = ctypes.c_size_t(0)
    assert L.hs_batch_buffer_size(_descs([32, 64, 128]), 3, ctypes.byref(n)) == hs.HS_OK
    assert n.value >= 3 * 256 + 224 * 4  # views with two TMA descriptors each, then the swarm table
    assert L.hs_batch_buffer_size(_descs([32]), 0, ctypes.byref(n)) == hs.HS_ERR_SIZE
    assert L.hs_batch_buffer_size(_descs([0]), 1, ctypes.byref(n)) == hs.HS_ERR_SIZE
    assert L.hs_batch_buffer_size(_descs([5000]), 1, ctypes.byref(n)) == hs.HS_ERR_SIZE  # above the fused step
    assert L.hs_batch_buffer_size(_descs([1024] * 64), 64, ctypes.byref(n)) == hs.HS_ERR_SIZE  # > 65535 in total
    assert L.hs_batch_buffer_size(None, 1, ctypes.byref(n)) == hs.HS_ERR_ARG
    h = ctypes.c_void_p()
    good = _descs([32, 64])
    L.hs_batch_buffer_size(good, 2, ctypes.byref(n))
    need = n.value
    assert L.hs_batch_create(m.handle, good, 2, FAKE, need - 256, None, ctypes.byref(h)) == hs.HS_ERR_SIZE
    assert L.hs_batch_create(m.handle, good, 2, FAKE + 16, need, None, ctypes.byref(h)) == hs.HS_ERR_ALIGN
    assert L.hs_batch_create(m.handle, _descs([32, 64], depth_pitch=600), 2, FAKE, need, None,
                             ctypes.byref(h)) == hs.HS_ERR_ALIGN
    assert L.hs_batch_create(m.handle, _descs([32, 64], stats=None), 2, FAKE, need, None,
                             ctypes.byref(h)) == hs.HS_ERR_ARG
    bad_mut = _descs([32, 64])
    bad_mut[1].n_mutate = 65
    assert L.hs_batch_create(m.handle, bad_mut, 2, FAKE, need, None, ctypes.byref(h)) == hs.HS_ERR_ARG
    bad_cam = _descs([32, 64])
    bad_cam[0].cam.fx = 0.0
    assert L.hs_batch_create(m.handle, bad_cam, 2, FAKE, need, None, ctypes.byref(h)) == hs.HS_ERR_ARG
    assert L.hs_batch_create(m.handle, good, 2, FAKE, need, None, None) == hs.HS_ERR_ARG
    # the batch-wide calls reject a missing batch
    prm = hs.score_params()
    assert L.render_score_multi(m.handle, None, FAKE, FAKE, ctypes.byref(prm), FAKE, 1 << 20, FAKE, None,
                                None) == hs.HS_ERR_ARG
    assert L.pose_fk_multi(m.handle, None, FAKE, FAKE, FAKE, None) == hs.HS_ERR_ARG
    assert L.hs_obs_prepare_multi(None, None) == hs.HS_ERR_ARG
    assert L.hs_batch_destroy(None) == hs.HS_ERR_ARG
    # the batch frame: no batch, no workspace size, no frame
    assert L.hs_frame_multi_workspace_size(None, ctypes.byref(n)) == hs.HS_ERR_ARG
    assert L.hs_frame_multi_capacity(None, None, None) == hs.HS_ERR_ARG
    sw = hs.HsSwarm(FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    scale = (ctypes.c_float * 26)(*([1.0] * 26))
    pp = hs.pso_params()
    assert L.track_frame_multi(m.handle, None, ctypes.byref(sw), FAKE + 4096, 40, ctypes.byref(prm), ctypes.byref(pp),
                               FAKE, scale, 0, 0, FAKE, 1 << 20, FAKE, FAKE, None) == hs.HS_ERR_ARG


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_valid_call_without_gpu_reports_cuda_error():
    m = _model()
    cam = hs.camera(262.5, 262.5, 160, 120)
    rc = hs.lib().pose_fk(m.handle, FAKE, 4, ctypes.byref(cam), FAKE, FAKE, None)
    assert rc == hs.HS_ERR_CUDA


def test_python_binding_requires_device_tensors():
    with pytest.raises(ValueError):
        hs._ptr(torch.zeros(4))
    assert np.float32(hs.score_params().d_M) == 40.0


def test_track_frame_host_checks():
    """track_frame refuses bad arguments on the host, before any CUDA call
    (the capacity check, which needs the device, comes after these)."""
    m = _model()
    L = hs.lib()
    cam = hs.camera(262.5, 262.5, 160, 120)
    prm = hs.score_params()
    pp = hs.pso_params(P=64)
    o = _obs()
    sw = hs.HsSwarm(FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    scale = (ctypes.c_float * 26)(*([1.0] * 26))
    need = ctypes.c_size_t()
    assert L.hs_frame_workspace_size(64, ctypes.byref(need)) == hs.HS_OK
    assert need.value == 128 + 3 * 32 * 64  # control block and three slots of per-particle sums
    assert L.hs_frame_workspace_size(0, ctypes.byref(need)) == hs.HS_ERR_SIZE
    assert L.hs_frame_workspace_size(hs.FRAME_MAX_PARTICLES + 1, ctypes.byref(need)) == hs.HS_ERR_SIZE

    def call(x_next=FAKE + 4096, P=64, gens=40, ctas=0, ws=FAKE, ws_bytes=1 << 20, kc=FAKE, pso=pp, sc=scale, s=sw):
        return L.track_frame(m.handle, ctypes.byref(o), ctypes.byref(cam), ctypes.byref(s), x_next, P, gens,
                             ctypes.byref(prm), ctypes.byref(pso), FAKE, sc, 1, 0, ctas, ws, ws_bytes, None, kc, None)

    assert call(x_next=FAKE) == hs.HS_ERR_ARG            # positions must be double-buffered
    assert call(gens=-1) == hs.HS_ERR_ARG
    assert call(ctas=-1) == hs.HS_ERR_ARG
    assert call(kc=None) == hs.HS_ERR_ARG
    assert call(P=0) == hs.HS_ERR_SIZE
    assert call(P=hs.FRAME_MAX_PARTICLES + 1) == hs.HS_ERR_SIZE
    assert call(ws=None) == hs.HS_ERR_ARG
    assert call(ws=FAKE + 8) == hs.HS_ERR_ALIGN
    assert call(ws_bytes=128) == hs.HS_ERR_SIZE  # smaller than 64 particles need
    assert call(pso=hs.pso_params(c1=1.0, c2=1.0, P=64)) == hs.HS_ERR_ARG   # psi <= 4
    assert call(pso=hs.pso_params(P=64, n_mutate=65)) == hs.HS_ERR_ARG      # more mutants than particles
    assert call(sc=(ctypes.c_float * 26)(*([1.0] * 25 + [-1.0]))) == hs.HS_ERR_ARG
    bad = hs.HsSwarm(FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, None)  # no E
    assert call(s=bad) == hs.HS_ERR_ARG
