"""GPU: per-generation records of tracked frames and checkpoint/resume of the
trackers (a tracker restored from a checkpoint continues bit for bit)."""
import io
import json

import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import runlog as RL
from paper_2005_07068_b300 import tracker as T
from tests import gpu_common as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)


@pytest.fixture(scope="module")
def scene():
    return C.make_scene(96, 80, 32, 911, zoom=1.5, noisy=True, f32=False)


def _tracker(sc, **kw):
    cam = hs.camera(*[float(v) for v in sc.cam])
    return T.Tracker(sc.model_g, cam, P=32, gens=6, seed=5, **kw)


def _obs(sc):
    o = hs.Obs.from_numpy(sc.Od, sc.S, torch.device("cuda"))
    return o


def test_generation_records_of_a_tracked_frame(scene):
    """record_history keeps each generation's global best and E; the records
    follow them: best E never rises within a frame, lies at or below the
    generation's smallest E, and ends at the swarm's global best."""
    trk = _tracker(scene, record_history=True)
    obs = _obs(scene)
    start = torch.from_numpy(scene.poses[-1]).cuda()
    buf = io.StringIO()
    log = RL.RunLog(buf)
    for f in range(2):
        trk.run_frame(obs, f, start if f == 0 else None)
        torch.cuda.synchronize()
        log.frame_from(trk, f, scene.gt)
    recs = [json.loads(ln) for ln in buf.getvalue().splitlines()]
    assert len(recs) == 2 * trk.gens
    for f in range(2):
        fr = [r for r in recs if r["frame"] == f]
        best = [r["best_E"] for r in fr]
        assert [r["gen"] for r in fr] == list(range(1, trk.gens + 1))
        assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))
        assert all(r["best_E"] <= r["min_E"] <= r["mean_E"] for r in fr)
    assert recs[-1]["best_E"] == float(trk.swarm.gbest_E.cpu()[0])
    assert hs.hs_get_device_status(clear=True) == 0


@pytest.mark.parametrize("kind", ["graph", "hybrid"])
def test_resume_from_checkpoint_is_bit_identical(scene, kind, tmp_path):
    """Frames 0-3 in one tracker against frames 0-1, a checkpoint, and frames
    2-3 in a fresh tracker restored from it: the same state bit for bit."""
    obs = _obs(scene)
    start = torch.from_numpy(scene.poses[-1]).cuda()
    make = (lambda: _tracker(scene)) if kind == "graph" else (
        lambda: T.HybridTracker(scene.model_g, hs.camera(*[float(v) for v in scene.cam]), P=32, gens=3, seed=5,
                                k=4, steps=2))

    def run(trk, frames):
        for f in frames:
            trk.run_frame(obs, f, start if f == 0 else None)
        torch.cuda.synchronize()

    ref = make()
    run(ref, range(4))
    a = make()
    run(a, range(2))
    path = tmp_path / "ck.pt"
    RL.save_checkpoint(a, path, next_frame=2)
    del a
    b = make()
    nxt = RL.load_checkpoint(b, path)
    assert nxt == 2
    run(b, range(nxt, 4))
    for x, y in zip(ref._state(), b._state()):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    assert hs.hs_get_device_status(clear=True) == 0


def test_batch_tracker_resume(tmp_path):
    """The same for a batch of uneven swarms (BatchTracker)."""
    scenes = [C.make_scene(64, 48, 16, 921, noisy=True), C.make_scene(80, 60, 24, 922, noisy=True, f32=False)]
    dev = torch.device("cuda")
    obs = [hs.Obs.from_numpy(sc.Od, sc.S, dev) for sc in scenes]
    cams = [hs.camera(*[float(v) for v in sc.cam]) for sc in scenes]
    b = hs.Batch(scenes[0].model_g, obs, cams, [sc.poses.shape[0] for sc in scenes], [0x5EED0200, 0x5EED0201])
    starts = torch.from_numpy(np.stack([sc.gt for sc in scenes]).astype(np.float32)).cuda()

    def run(trk, frames):
        for f in frames:
            trk.run_frame(f, starts if f == 0 else None)
        torch.cuda.synchronize()

    ref = T.BatchTracker(scenes[0].model_g, b, gens=4)
    run(ref, range(3))
    a = T.BatchTracker(scenes[0].model_g, b, gens=4)
    run(a, range(1))
    RL.save_checkpoint(a, tmp_path / "b.pt", next_frame=1)
    c = T.BatchTracker(scenes[0].model_g, b, gens=4)
    run(c, range(RL.load_checkpoint(c, tmp_path / "b.pt"), 3))
    for x, y in zip(ref._state(), c._state()):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    assert hs.hs_get_device_status(clear=True) == 0
