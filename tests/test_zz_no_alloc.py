"""The allocation-free scoring entry point (render_score_batch_noalloc).

Callers that cannot allocate device memory (a plugin whose host owns every
allocation, a real-time loop that must not allocate) score through this entry
point, whose scratch is a fixed array inside the library.  It must give the
same E as render_score_batch with a caller workspace, on two calls in a row
(the second call finds the array as the first left it).  This file is collected
last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from tests import gpu_common as C

pytestmark = pytest.mark.gpu


def _prepared(sc):
    dev = torch.device("cuda")
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    hs.hs_obs_prepare(obs)
    cam = hs.camera(*[float(v) for v in sc.cam])
    P = sc.poses.shape[0]
    prims = torch.zeros(P, sc.model_g.n_prims, 16, device=dev)
    kc = torch.zeros(P, device=dev)
    hs.pose_fk(sc.model_g, torch.from_numpy(sc.poses).to(dev), cam, prims, kc)
    return obs, cam, prims, kc


@pytest.mark.parametrize("W,H,P,seed,kw", [
    (320, 240, 64, 2005070682, dict(noisy=True, f32=False)),
    (80, 60, 24, 7, dict(zoom=3.0, noisy=True, f32=False)),
])
def test_noalloc_matches_workspace_entry_point(W, H, P, seed, kw):
    B.build()
    sc = C.make_scene(W, H, P, seed, **kw)
    obs, cam, prims, kc = _prepared(sc)
    dev = prims.device
    E_ref = torch.zeros(P, device=dev)
    hs.render_score_batch(sc.model_g, obs, cam, prims, kc, hs.score_params(), hs.new_workspace(P, dev), E_ref)
    for _ in range(2):  # the second call sees the array as the first one left it
        E = torch.full((P,), float("nan"), device=dev)
        parts = torch.zeros(P, 4, dtype=torch.int32, device=dev)
        hs.render_score_batch_noalloc(sc.model_g, obs, cam, prims, kc, hs.score_params(), E, parts)
        torch.cuda.synchronize()
        e, r = E.cpu().numpy(), E_ref.cpu().numpy()
        assert np.all(np.abs(e - r) <= C.E_REL_TOL * np.abs(r) + C.E_ABS_TOL)
        assert np.all(parts.cpu().numpy()[:, 3] > 0)


def test_noalloc_rejects_p_over_the_limit():
    B.build()
    sc = C.make_scene(64, 48, 2, 3)
    obs, cam, prims, kc = _prepared(sc)
    P_max = hs.NOALLOC_SCRATCH_BYTES // 32
    big_kc = torch.zeros(P_max + 1, device=prims.device)
    with pytest.raises(hs.HandscoreError) as e:
        hs.render_score_batch_noalloc(sc.model_g, obs, cam, prims, big_kc, hs.score_params(),
                                      torch.zeros(P_max + 1, device=prims.device))
    assert e.value.status == hs.HS_ERR_SIZE
