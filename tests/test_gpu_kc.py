"""GPU: the kc variants of Eq. 5 -- the paper's abduction ordering, and the
interpenetration test of different fingers -- against the FP64 oracle
(oracle.collide), through pose_fk, the score, and a tracked frame.

Tolerance of pen (derived, not tuned): each penetrating pair contributes
r_i + r_j - |c_i - c_j| with FP32 proxy centres ~1e-4 mm off (the FK centre
bound of the parity tests) and a 2^-20 mm fixed-point rounding; a few dozen
pairs penetrate at most, so 1e-3 mm + 1e-5 relative bounds the sum."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import collide as K
from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import tracker as T
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

PEN_ABS_MM, PEN_REL = 1e-3, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)


def _poses(n, seed):
    """Seeded poses within the limits, half of them with fingers swung into
    their neighbours (penetrating)."""
    lo, hi = I.search_limits()
    P = I.sample_poses(np.random.default_rng(seed), n, lo, hi)
    for i in range(0, n, 2):
        P[i, [11, 15, 19, 23]] = np.clip(P[i, [11, 15, 19, 23]] + np.array([-0.3, 0.25, -0.2, 0.3]),
                                         lo[[11, 15, 19, 23]], hi[[11, 15, 19, 23]])
    return P.astype(np.float32)


def _gpu_kc(model_g, poses, cam):
    P = poses.shape[0]
    prims = torch.zeros(P, model_g.n_prims, 16, device="cuda")
    kc = torch.zeros(P, device="cuda")
    hs.pose_fk(model_g, torch.from_numpy(poses).cuda(), cam, prims, kc)
    torch.cuda.synchronize()
    return kc.cpu().numpy()


@pytest.mark.parametrize("variant,w", [(hs.HS_KC_ABDUCTION, 0.0), (hs.HS_KC_ABD_PEN, 0.05), (hs.HS_KC_PEN, 1.0)])
def test_pose_fk_kc_against_oracle(variant, w):
    g = C.geometry_f32()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    mo = oracle.Model.from_geometry(g, lo.astype(np.float64), hi.astype(np.float64))
    mg = hs.Model.from_geometry(g, lo, hi).set_kc(variant, w)
    cam = hs.camera(*[float(v) for v in oracle.camera_tuple(I.kinect_camera(320, 240))])
    poses = _poses(48, 901)
    got = _gpu_kc(mg, poses, cam)
    ref = np.array([K.kc_variant(mo, p.astype(np.float64), variant, w) for p in poses])
    pen = np.array([K.penetration(mo, p.astype(np.float64)) for p in poses])
    tol = 1e-6 + w * (PEN_ABS_MM + PEN_REL * pen)
    assert np.all(np.abs(got - ref) <= tol), np.abs(got - ref).max()
    if variant != hs.HS_KC_ABDUCTION:
        assert (pen > 1.0).sum() >= 10  # the test poses do penetrate
    assert hs.hs_get_device_status(clear=True) == 0


def test_score_with_penetration_term():
    """E = D + lambda_k kc with the variant's kc, against the oracle's D (its E
    with the paper's kc) plus lambda_k times the variant's kc."""
    sc = C.make_scene(96, 80, 24, 902, noisy=True, f32=False, spread=3.0)
    w = 0.05
    sc.model_g.set_kc(hs.HS_KC_ABD_PEN, w)
    try:
        gr = C.run_gpu(sc, debug=False)
    finally:
        sc.model_g.set_kc(hs.HS_KC_ABDUCTION, 0.0)
    ref = oracle.score_batch(sc.model_o, sc.poses.astype(np.float64), sc.cam.astype(np.float64),
                             sc.Od.astype(np.float64), sc.S)["E"]
    lam_k = float(hs.score_params().lambda_k)
    k0 = np.array([oracle.kc(np.clip(p.astype(np.float64), sc.model_o.lo, sc.model_o.hi)) for p in sc.poses])
    kv = np.array([K.kc_variant(sc.model_o, p.astype(np.float64), hs.HS_KC_ABD_PEN, w) for p in sc.poses])
    E_ref = ref + lam_k * (kv - k0)
    tol = C.E_REL_TOL * np.abs(E_ref) + C.E_ABS_TOL + lam_k * w * PEN_ABS_MM
    assert np.all(np.abs(gr.E - E_ref) <= tol), np.abs(gr.E - E_ref).max()


def test_frame_equals_step_by_step_with_penetration_term():
    """The fixed-point penetration sum does not depend on how many threads
    share the pairs: a tracked frame with the variant is the same, bit for
    bit, through the one-launch frame kernel and the step-by-step calls."""
    sc = C.make_scene(128, 96, 32, 903, noisy=True, f32=False, spread=2.0)
    sc.model_g.set_kc(hs.HS_KC_ABD_PEN, 0.05)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    start = torch.from_numpy(sc.poses[-1]).cuda()
    out = []
    for tr in (T.Tracker(sc.model_g, cam, P=32, gens=6, seed=5),
               T.FrameTracker(sc.model_g, cam, P=32, gens=6, seed=5, ctas=70)):
        tr.run_frame(obs, 0, start, graph=False)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy().copy() for t in (tr.swarm.x, tr.swarm.gbest, tr.swarm.gbest_E, tr.kc, tr.prims)])
    sc.model_g.set_kc(hs.HS_KC_ABDUCTION, 0.0)
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def _inside_poses(n, seed):
    """Seeded poses strictly inside the limits, most of them with the index
    swung into the middle finger (penetrating), none within 1e-3 mm of a kink
    of pen (a pair just touching) or with two abduction angles equal."""
    lo, hi = I.search_limits()
    rng = np.random.default_rng(seed)
    out = []
    g = C.geometry_f32()
    mo = oracle.Model.from_geometry(g, lo, hi)
    while len(out) < n:
        p = I.sample_poses(rng, 1, lo + 0.02, hi - 0.02)[0]
        p[11] = rng.uniform(-0.25, -0.05)
        p[15] = rng.uniform(-0.05, 0.15)
        C_, r, f, fixed = K.proxies(mo, oracle.fk(mo, p))
        gaps = [abs(r[i] + r[j] - np.linalg.norm(C_[i] - C_[j])) for i in range(len(r)) for j in range(i + 1, len(r))
                if f[i] >= 0 and f[j] >= 0 and f[i] != f[j] and not (fixed[i] and fixed[j])]
        if min(gaps) > 1e-3 and len(set(np.round(p[[11, 15, 19, 23]], 6))) == 4:
            out.append(p.astype(np.float32))
    return np.array(out)


@pytest.mark.parametrize("variant,w", [(hs.HS_KC_ABDUCTION, 0.0), (hs.HS_KC_ABD_PEN, 0.05), (hs.HS_KC_PEN, 1.0)])
def test_gradient_of_the_kc_variants(variant, w):
    """pose_grad with a zero render adjoint is lambda_k d kc / d pose alone:
    against lambda_k times the oracle's complex-step gradient of the variant's
    kc.  Tolerance (derived): the proxy centres carry the FK's FP32 error
    (~1e-4 mm) over distances of a few mm, so each pair's unit vector is good
    to ~1e-4 and the tangents to ~1e-6: 1e-3 of the largest component, and
    the direction to a cosine of 1 - 1e-6."""
    g = C.geometry_f32()
    lo, hi = (a.astype(np.float32) for a in I.search_limits())
    mo = oracle.Model.from_geometry(g, lo.astype(np.float64), hi.astype(np.float64))
    mg = hs.Model.from_geometry(g, lo, hi).set_kc(variant, w)
    cam = hs.camera(*[float(v) for v in oracle.camera_tuple(I.kinect_camera(320, 240))])
    poses = _inside_poses(12, 905 + variant)
    P = poses.shape[0]
    prims = torch.zeros(P, mg.n_prims, 16, device="cuda")
    kc = torch.zeros(P, device="cuda")
    adj = torch.zeros(P, mg.n_prims, hs.SOFT_ADJ, dtype=torch.int64, device="cuda")
    grad = torch.zeros(P, 26, device="cuda")
    prm = hs.score_params()
    hs.pose_grad(mg, torch.from_numpy(poses).cuda(), cam, prm, prims, kc, adj, grad)
    torch.cuda.synchronize()
    got = grad.cpu().numpy().astype(np.float64)
    lam_k = float(prm.lambda_k)
    pens = []
    for k in range(P):
        want = lam_k * K.kc_variant_gradient(mo, poses[k].astype(np.float64), variant, w)
        scale = max(np.abs(want).max(), lam_k)
        assert np.abs(got[k] - want).max() <= 1e-3 * scale, (k, np.abs(got[k] - want).max(), scale)
        if np.linalg.norm(want) > 0:
            cos = got[k] @ want / (np.linalg.norm(got[k]) * np.linalg.norm(want))
            assert cos >= 1 - 1e-6, (k, cos)
        pens.append(K.penetration(mo, poses[k].astype(np.float64)))
    if variant != hs.HS_KC_ABDUCTION:
        assert sum(p > 0.5 for p in pens) >= 4  # the term is exercised
    assert hs.hs_get_device_status(clear=True) == 0
