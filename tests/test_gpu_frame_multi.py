"""GPU: a whole frame of every swarm of a batch in one cooperative launch
(track_frame_multi).

The kernel runs the step-by-step batch calls' arithmetic (init_position,
swarm_update, fk_particle, the unit renderer, form_E) per particle task, so a
frame must equal, bit for bit, hs_obs_prepare_multi + pso_init_multi +
pose_fk_multi + gens x (render_score_multi, pso_step_fk_multi): every swarm
array, the final records and kc -- for any grid size, and whatever order the
swarms' generations interleave in.  The step-by-step batch calls are checked
against single swarms (test_gpu_batch.py) and those against the FP64 oracle;
here the first generation is also checked against the oracle directly."""
import time

import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import tracker as T
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

# (W, H, P, seed, kw): ROIs from 31x200 to 256x256 with ragged tails, P from 1
# to 256, float32 and uint16 depth
SWARMS = [
    (48, 48, 32, 601, dict()),
    (67, 53, 17, 602, dict(noisy=True, f32=False)),
    (128, 96, 64, 603, dict(noisy=True)),
    (31, 200, 1, 604, dict(zoom=2.0)),
    (200, 150, 128, 605, dict(noisy=True, f32=False, spread=2.0)),
    (256, 256, 256, 606, dict(f32=False, noisy=True)),
]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)


@pytest.fixture(scope="module")
def scenes():
    return [C.make_scene(W, H, P, seed, **kw) for W, H, P, seed, kw in SWARMS]


def _batch(scenes):
    dev = torch.device("cuda")
    obs = [hs.Obs.from_numpy(sc.Od, sc.S, dev) for sc in scenes]
    cams = [hs.camera(*[float(v) for v in sc.cam]) for sc in scenes]
    seeds = [0x5EED0100 + 29 * s for s in range(len(scenes))]
    return obs, hs.Batch(scenes[0].model_g, obs, cams, [sc.poses.shape[0] for sc in scenes], seeds)


def _run(tr, frames, starts):
    out = []
    for f in range(frames):
        tr.run_frame(f, starts if f == 0 else None, graph=False)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy().copy() for t in tr._state()])
    return out


def _counters_zero(ft, b):
    """The control block (32 words) and the per-swarm counts after it."""
    return int(ft.fws[:32].abs().sum()) == 0 and int(ft.fws[32:32 + b.S].abs().sum()) == 0


def _equal(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("kc_variant", [hs.HS_KC_ABDUCTION, hs.HS_KC_ABD_PEN])
def test_batch_frame_equals_step_by_step(scenes, kc_variant):
    """Two frames x 7 generations (mutation after 3 and 6) of six uneven
    swarms: the whole state equals the step-by-step batch calls' bit for bit,
    with a grid of 5 CTAs (each takes hundreds of tasks), 97 CTAs and the
    device's capacity; the workspace is left zeroed after every frame.  Also
    with the interpenetration term in kc (the model with collision data)."""
    m = scenes[0].model_g
    m.set_kc(kc_variant, 0.05 if kc_variant != hs.HS_KC_ABDUCTION else 0.0)
    try:
        obs, b = _batch(scenes)
        starts = torch.from_numpy(np.stack([sc.poses[-1] for sc in scenes]).astype(np.float32)).cuda()
        ref = _run(T.BatchTracker(m, b, gens=7), 2, starts)
        for ctas in (5, 97, 0):
            ft = T.BatchFrameTracker(m, b, gens=7, ctas=ctas)
            got = _run(ft, 2, starts)
            for f in range(2):
                for k, (x, y) in enumerate(zip(got[f], ref[f])):
                    assert _equal(x, y), (ctas, f, k)
            assert _counters_zero(ft, b), ctas  # the counters return to zero for the next frame
        assert hs.hs_get_device_status(clear=True) == 0
        # the search made progress on every sequence
        assert np.all(ref[-1][6] <= ref[0][6])
    finally:
        m.set_kc(hs.HS_KC_ABDUCTION, 0.0)


@pytest.mark.parametrize("gens", [0, 1, 2])
def test_batch_frame_few_generations(scenes, gens):
    """No generation (the initial swarms and their records), one (a render,
    then the step on it) and two: still the step-by-step result."""
    sub = scenes[:4]
    m = sub[0].model_g
    obs, b = _batch(sub)
    starts = torch.from_numpy(np.stack([sc.gt for sc in sub]).astype(np.float32)).cuda()
    ref = _run(T.BatchTracker(m, b, gens=gens), 1, starts)
    got = _run(T.BatchFrameTracker(m, b, gens=gens, ctas=11), 1, starts)
    for k, (x, y) in enumerate(zip(got[0], ref[0])):
        assert _equal(x, y), (gens, k)
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_frame_first_generation_against_oracle(scenes):
    """One generation: E of each swarm's initial positions (drawn by the
    kernel around the seed poses, left in the first position buffer) against
    the FP64 oracle's scores of the same poses.  E after one generation is the
    objective of those positions (the step moves them afterwards)."""
    sub = [scenes[1], scenes[2]]
    m = sub[0].model_g
    obs, b = _batch(sub)
    starts = np.stack([sc.gt for sc in sub]).astype(np.float32)
    ft = T.BatchFrameTracker(m, b, gens=1, ctas=9)
    ft.run_frame(0, torch.from_numpy(starts).cuda())
    torch.cuda.synchronize()
    E = ft.swarm.E.cpu().numpy()
    x0 = ft.x_buf[0].cpu().numpy().astype(np.float64)
    lim = [a.astype(np.float32) for a in I.search_limits()]
    for s, sc in enumerate(sub):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        assert np.array_equal(x0[lo].astype(np.float32), np.clip(starts[s], *lim))  # particle 0 = seed pose
        # the same poses through the single-swarm calls: the same E bit for bit,
        # and those against the oracle with the full parity protocol
        gr = C.run_gpu(sc, debug=True, poses=x0[lo:hi].astype(np.float32))
        assert _equal(E[lo:hi], gr.E), s
        C.check_parity(sc, gr, C.run_oracle(sc, poses=x0[lo:hi]))
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_frame_wait_time_limit_is_reported(scenes):
    """A per-swarm wait for renders that never come (the workspace's word for
    missing renders set) runs out after about a second: every CTA stops taking
    tasks, HS_DEV_BARRIER_TIMEOUT is set with no fault, the counters return to
    zero, and the next frame (word cleared) equals the step-by-step calls."""
    sub = scenes[:3]
    m = sub[0].model_g
    obs, b = _batch(sub)
    starts = torch.from_numpy(np.stack([sc.gt for sc in sub]).astype(np.float32)).cuda()
    hs.hs_get_device_status(clear=True)
    ft = T.BatchFrameTracker(m, b, gens=3, ctas=6)
    ft.fws[3] = 1  # one render every wait expects that never comes
    t0 = time.perf_counter()
    ft.run_frame(0, starts)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert hs.hs_get_device_status(clear=True) & hs.HS_DEV_BARRIER_TIMEOUT
    assert 0.5 < waited < 30.0, waited
    ft.fws[3] = 0
    assert _counters_zero(ft, b)
    got = _run(ft, 1, starts)
    ref = _run(T.BatchTracker(m, b, gens=3), 1, starts)
    for k, (x, y) in enumerate(zip(got[0], ref[0])):
        assert _equal(x, y), k
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_frame_rejects_bad_arguments(scenes):
    sub = scenes[:2]
    m = sub[0].model_g
    obs, b = _batch(sub)
    ft = T.BatchFrameTracker(m, b, gens=3)
    starts = torch.from_numpy(np.stack([sc.gt for sc in sub]).astype(np.float32)).cuda()

    def call(ctas=0, x_next=None, ws=None, pso=None, gens=3):
        hs.track_frame_multi(m, b, ft.swarm, ft.x_buf[1] if x_next is None else x_next, gens, ft.score,
                             ft.pso if pso is None else pso, starts, ft.scale, 0, ctas,
                             ft.fws if ws is None else ws, ft.prims, ft.kc)

    cap = hs.frame_multi_capacity(b, m)
    assert cap >= hs.frame_multi_capacity(b)  # (None: any model, up to HS_MAX_PRIMS primitives)
    assert cap >= hs.frame_multi_capacity() >= torch.cuda.get_device_properties(0).multi_processor_count
    for kw, status in ((dict(ctas=cap + 1), hs.HS_ERR_SIZE),
                       (dict(ctas=-1), hs.HS_ERR_ARG),
                       (dict(ws=ft.fws[:8]), hs.HS_ERR_SIZE),
                       (dict(x_next=ft.swarm.x), hs.HS_ERR_ARG),
                       (dict(pso=hs.pso_params(e_stop=1.0)), hs.HS_ERR_ARG),
                       (dict(gens=-1), hs.HS_ERR_ARG),
                       (dict(gens=(1 << 31) // b.P_total), hs.HS_ERR_SIZE)):  # beyond the task counter
        with pytest.raises(hs.HandscoreError) as e:
            call(**kw)
        assert e.value.status == status, kw
    # a kc variant keeps the collision data in shared memory: fewer CTAs fit, and the frame takes no more
    m.set_kc(hs.HS_KC_ABD_PEN, 0.05)
    try:
        cap_pen = hs.frame_multi_capacity(b, m)
        assert torch.cuda.get_device_properties(0).multi_processor_count <= cap_pen <= cap
        with pytest.raises(hs.HandscoreError) as e:
            call(ctas=cap_pen + 1)
        assert e.value.status == hs.HS_ERR_SIZE
    finally:
        m.set_kc(hs.HS_KC_ABDUCTION, 0.0)
    torch.cuda.synchronize()
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_frame_autotune_keeps_state(scenes):
    """The grid-size tuner times real grids, picks one of them, and leaves the
    swarms as they were; a frame at the chosen grid still equals the
    step-by-step calls."""
    sub = scenes[:3]
    m = sub[0].model_g
    obs, b = _batch(sub)
    starts = torch.from_numpy(np.stack([sc.gt for sc in sub]).astype(np.float32)).cuda()
    ft = T.BatchFrameTracker(m, b, gens=2)
    before = [t.clone() for t in ft._state()]
    table = ft.autotune(starts, reps=1)
    assert ft.ctas in ft.candidates() and len(table) == len(ft.candidates())
    assert all(v > 0 for v in table.values())
    assert all(torch.equal(x, y) for x, y in zip(before, ft._state()))
    got = _run(ft, 1, starts)
    ref = _run(T.BatchTracker(m, b, gens=2), 1, starts)
    for k, (x, y) in enumerate(zip(got[0], ref[0])):
        assert _equal(x, y), k
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_frame_max_primitive_model():
    """A model with HS_MAX_PRIMS primitives: the frame kernel's shared memory is
    sized for the model's primitives, so this is its largest layout; the frame
    still equals the step-by-step calls bit for bit."""
    g = C.geometry_max_prims()
    sub = [C.make_scene(W, H, P, seed, geometry=g, **kw) for W, H, P, seed, kw in SWARMS[:3]]
    m = sub[0].model_g
    assert m.n_prims == hs.MAX_PRIMS
    obs, b = _batch(sub)
    starts = torch.from_numpy(np.stack([sc.gt for sc in sub]).astype(np.float32)).cuda()
    assert torch.cuda.get_device_properties(0).multi_processor_count <= hs.frame_multi_capacity(b, m)
    ref = _run(T.BatchTracker(m, b, gens=3), 1, starts)
    got = _run(T.BatchFrameTracker(m, b, gens=3), 1, starts)
    for k, (x, y) in enumerate(zip(got[0], ref[0])):
        assert _equal(x, y), k
    assert hs.hs_get_device_status(clear=True) == 0

