"""The allocation-free scoring entry point (render_score_batch_noalloc).

Callers that cannot allocate device memory (a plugin whose host owns every
allocation, a real-time loop that must not allocate after start-up) score
through this entry point, whose scratch is a fixed array inside the library.
It runs the same kernel as render_score_batch with a caller workspace, and its
sums are order-independent integers, so E and the per-particle sums must equal
that entry point's bit for bit, on two calls in a row (the second call finds
the array as the first left it).  This file is collected last so that a
failure here does not hide the other tests.
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
    prm = hs.score_params()
    E_ref = torch.zeros(P, device=dev)
    parts_ref = torch.zeros(P, 4, dtype=torch.int32, device=dev)
    hs.render_score_batch(sc.model_g, obs, cam, prims, kc, prm, hs.new_workspace(P, dev), E_ref, parts_ref)
    torch.cuda.synchronize()
    e_ref, p_ref = E_ref.cpu().numpy(), parts_ref.cpu().numpy()
    # the workspace path itself is within the oracle's tolerance elsewhere; here
    # a sanity bound keeps a broken reference from passing vacuously
    assert np.all(np.isfinite(e_ref)) and np.all(p_ref[:, 3] > 0)
    for _ in range(2):  # the second call sees the array as the first one left it
        E = torch.full((P,), float("nan"), device=dev)
        parts = torch.full((P, 4), -1, dtype=torch.int32, device=dev)
        hs.render_score_batch_noalloc(sc.model_g, obs, cam, prims, kc, prm, E, parts)
        torch.cuda.synchronize()
        assert np.array_equal(E.cpu().numpy().view(np.uint32), e_ref.view(np.uint32))
        assert np.array_equal(parts.cpu().numpy(), p_ref)


def test_noalloc_rejects_p_over_the_limit():
    B.build()
    sc = C.make_scene(64, 48, 2, 3)
    obs, cam, prims, kc = _prepared(sc)
    # the largest P whose workspace fits the array, from the library's own size rule
    P_max = 1
    while hs.workspace_size(P_max + 1) <= hs.NOALLOC_SCRATCH_BYTES:
        P_max += 1
    assert hs.workspace_size(P_max) <= hs.NOALLOC_SCRATCH_BYTES < hs.workspace_size(P_max + 1)
    big_kc = torch.zeros(P_max + 1, device=prims.device)
    with pytest.raises(hs.HandscoreError) as e:
        hs.render_score_batch_noalloc(sc.model_g, obs, cam, prims, big_kc, hs.score_params(),
                                      torch.zeros(P_max + 1, device=prims.device))
    assert e.value.status == hs.HS_ERR_SIZE
