"""GPU: a whole tracking frame in one cooperative launch (track_frame).

The frame kernel runs the same arithmetic as the step-by-step path (the unit
renderer, form_E, swarm_update, fk_particle), so a frame must equal, bit for
bit, hs_obs_prepare + pso_init + pose_fk + gens x (render_score_batch,
pso_step_fk): every swarm array, the final records and kc, and the
observation totals -- for every number of CTAs per particle.  The
step-by-step path itself is checked against the FP64 oracle in
test_gpu_parity.py; here its first generation is also checked against the
oracle's scores of the same initial swarm."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import tracker as T
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

# (W, H, P, seed, kw): tiny FP32, ragged uint16, Kinect scale, and a swarm
# pushed partly out of the ROI
SCENES = [
    (64, 64, 16, 711, dict()),
    (77, 45, 7, 712, dict(noisy=True, f32=False)),
    (320, 240, 64, 713, dict(noisy=True, f32=False)),
    (128, 96, 33, 714, dict(noisy=True, shift=(70.0, 0.0), spread=2.0)),
]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)


def _state(tr):
    sw = tr.swarm
    return dict(x=sw.x, v=sw.v, pbest=sw.pbest, pbest_E=sw.pbest_E, gbest=sw.gbest, gbest_E=sw.gbest_E, E=sw.E,
                prims=tr.prims, kc=tr.kc)


def _counter_words(P):
    """int32 words of the frame workspace that every call leaves zeroed (the
    control block and three slots of per-particle sums)."""
    return (128 + 3 * 32 * P) // 4


def _run(tr, obs, frames, start):
    out = []
    for f in range(frames):
        tr.run_frame(obs, f, start if f == 0 else None, graph=False)
        torch.cuda.synchronize()
        st = {k: v.cpu().numpy().copy() for k, v in _state(tr).items()}
        st["stats"] = obs.stats.cpu().numpy().copy()
        out.append(st)
    return out


@pytest.mark.parametrize("scene", range(len(SCENES)))
@pytest.mark.parametrize("gens", [7, 4])
def test_frame_equals_step_by_step(scene, gens):
    """Two frames (mutation after generations 3 and 6 when gens = 7; an even
    count leaves the positions in the first buffer) at several grid sizes: one
    CTA per particle, sizes that are no multiple of P (uneven deals), the
    device's capacity and the automatic choice."""
    W, H, P, seed, kw = SCENES[scene]
    sc = C.make_scene(W, H, P, seed, **kw)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    start = torch.from_numpy(sc.poses[-1]).cuda()
    ref = _run(T.Tracker(sc.model_g, cam, P=P, gens=gens, seed=seed), obs, 2, start)
    ft = T.FrameTracker(sc.model_g, cam, P=P, gens=gens, seed=seed)
    cand = ft.candidates()
    cap = hs.frame_capacity()
    assert cand and cand[0] == P and cand[-1] == cap
    sizes = sorted({P, 2 * P + 1, 3 * P - 1, cap} & set(range(P, cap + 1))) + [0]
    for n in sizes:
        ft = T.FrameTracker(sc.model_g, cam, P=P, gens=gens, seed=seed, ctas=n)
        got = _run(ft, obs, 2, start)
        for f in range(2):
            for k in ref[f]:
                assert np.array_equal(got[f][k], ref[f][k], equal_nan=True), (n, f, k)
        # the counters and sums are left zeroed for the next frame
        assert int(ft.fws[:_counter_words(P)].abs().sum()) == 0, n
    assert hs.hs_get_device_status(clear=True) == 0
    # the search made progress
    assert ref[-1]["gbest_E"][0] <= ref[0]["gbest_E"][0]


def test_frame_at_the_capacity_limit():
    """As many particles as the device keeps resident at one CTA each (the
    largest grid a frame may have), on a small ROI: still the step-by-step
    result, and a grid one CTA larger is refused without a launch."""
    cap = hs.frame_capacity()
    P = min(cap, hs.FRAME_MAX_PARTICLES)
    sc = C.make_scene(64, 48, 2, 717, noisy=True, f32=False)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    start = torch.from_numpy(sc.gt).cuda()
    ref = _run(T.Tracker(sc.model_g, cam, P=P, gens=3, seed=9), obs, 1, start)
    ft = T.FrameTracker(sc.model_g, cam, P=P, gens=3, seed=9, ctas=P)
    got = _run(ft, obs, 1, start)
    for k in ref[0]:
        assert np.array_equal(got[0][k], ref[0][k], equal_nan=True), k
    if P < hs.FRAME_MAX_PARTICLES:
        big = T.FrameTracker(sc.model_g, cam, P=P + 1, gens=3, seed=9, ctas=P + 1)
        with pytest.raises(hs.HandscoreError) as e:
            big.run_frame(obs, 0, start)
        assert e.value.status == hs.HS_ERR_SIZE
    torch.cuda.synchronize()
    assert hs.hs_get_device_status(clear=True) == 0


def test_barrier_time_limit_is_reported():
    """A grid barrier that waits for arrivals that never come (the workspace's
    word for missing arrivals set) runs out after about a second: the frame
    stops with HS_DEV_BARRIER_TIMEOUT and no fault, and the next frame (word
    cleared) equals the step-by-step calls."""
    W, H, P, seed = 64, 48, 8, 718
    sc = C.make_scene(W, H, P, seed, noisy=True, f32=False)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    start = torch.from_numpy(sc.gt).cuda()
    hs.hs_get_device_status(clear=True)
    ft = T.FrameTracker(sc.model_g, cam, P=P, gens=3, seed=seed, ctas=P)
    ft.fws[2] = 1  # one arrival that never comes
    t0 = time.perf_counter()
    ft.run_frame(obs, 0, start)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert hs.hs_get_device_status(clear=True) & hs.HS_DEV_BARRIER_TIMEOUT
    assert 0.5 < waited < 30.0, waited
    assert int(ft.fws[:2].abs().sum()) == 0  # the counters were returned to zero on the way out
    ft.fws[2] = 0
    got = _run(ft, obs, 1, start)
    ref = _run(T.Tracker(sc.model_g, cam, P=P, gens=3, seed=seed), obs, 1, start)
    for k in ref[0]:
        assert np.array_equal(got[0][k], ref[0][k], equal_nan=True), k
    assert hs.hs_get_device_status(clear=True) == 0


def test_first_generation_against_oracle():
    """One generation: E of the initial swarm (the positions the frame kernel
    drew around the seed pose, left in the first position buffer) against the
    FP64 oracle's scores of the same poses."""
    W, H, P, seed = 96, 80, 24, 715
    sc = C.make_scene(W, H, P, seed, noisy=True, f32=False)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    ft = T.FrameTracker(sc.model_g, cam, P=P, gens=1, seed=seed, ctas=2 * P + 3)
    start = torch.from_numpy(sc.gt).cuda()
    ft.run_frame(obs, 0, start)
    torch.cuda.synchronize()
    E = ft.swarm.E.cpu().numpy()
    x0 = ft.x_buf[0].cpu().numpy().astype(np.float64)
    assert np.array_equal(x0[0], np.clip(sc.gt, *I.search_limits()).astype(np.float32))  # particle 0 = seed pose
    ref = oracle.score_batch(sc.model_o, x0, sc.cam.astype(np.float64), sc.Od.astype(np.float64), sc.S)["E"]
    assert np.all(np.abs(E - ref) <= C.E_REL_TOL * np.abs(ref) + C.E_ABS_TOL), np.abs(E - ref).max()


def test_frame_rejects_bad_arguments():
    sc = C.make_scene(64, 48, 8, 716)
    cam = hs.camera(*[float(v) for v in sc.cam])
    obs = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    ft = T.FrameTracker(sc.model_g, cam, P=8, gens=3, seed=1)
    start = torch.from_numpy(sc.gt).cuda()
    for n, status in ((hs.frame_capacity() + 1, hs.HS_ERR_SIZE),  # more CTAs than the device holds
                      (7, hs.HS_ERR_SIZE),                       # fewer CTAs than particles
                      (-1, hs.HS_ERR_ARG)):
        with pytest.raises(hs.HandscoreError) as e:
            hs.track_frame(ft.model, obs, cam, ft.swarm, ft.x_buf[1], 3, ft.score, ft.pso, start, ft.scale, 1, 0,
                           n, ft.fws, ft.kc)
        assert e.value.status == status, n
    with pytest.raises(hs.HandscoreError) as e:  # workspace too small
        hs.track_frame(ft.model, obs, cam, ft.swarm, ft.x_buf[1], 3, ft.score, ft.pso, start, ft.scale, 1, 0, 8,
                       ft.fws[:4], ft.kc)
    assert e.value.status == hs.HS_ERR_SIZE
    with pytest.raises(hs.HandscoreError) as e:  # positions must be double-buffered
        hs.track_frame(ft.model, obs, cam, ft.swarm, ft.swarm.x, 3, ft.score, ft.pso, start, ft.scale, 1, 0, 8,
                       ft.fws, ft.kc)
    assert e.value.status == hs.HS_ERR_ARG
    torch.cuda.synchronize()
    assert hs.hs_get_device_status(clear=True) == 0
