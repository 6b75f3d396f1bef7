"""GPU: the render kernels' bounded observation wait, tested without a fault.

A word of the caller's workspace (zero in every real call) makes the first
observation load of one particle's first warp expect 64 bytes more than its
TMA copies deliver, so that warp's wait runs out after its wall-clock limit.
The kernel must then flag HS_DEV_TMA_TIMEOUT, leave no copy in flight, leave
every other particle's E untouched (bit for bit), clear the workspace as
usual, and the next call must equal a clean call bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

TX_TEST_WORD = 7  # 32-bit word of a particle's 32-byte workspace slot that holds the test's extra bytes


@pytest.mark.parametrize("variant", [hs.RENDER_UNITS, hs.RENDER_TILES_32x32, hs.RENDER_STRIPS_8x32])
def test_observation_wait_time_limit_is_reported(variant):
    B.build()
    sc = C.make_scene(80, 60, 6, 7, zoom=3.0, noisy=True, f32=False)
    dev = torch.device("cuda")
    P = sc.poses.shape[0]
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    hs.hs_obs_prepare(obs)
    cam = hs.camera(*[float(v) for v in sc.cam])
    prims = torch.zeros(P, sc.model_g.n_prims, 16, device=dev)
    kc = torch.zeros(P, device=dev)
    hs.pose_fk(sc.model_g, torch.from_numpy(sc.poses).to(dev), cam, prims, kc)
    prm = hs.score_params(variant=variant)
    ws = hs.new_workspace(P, dev)

    def score():
        E = torch.full((P,), float("nan"), device=dev)
        parts = torch.zeros(P, 4, dtype=torch.int32, device=dev)
        hs.render_score_batch(sc.model_g, obs, cam, prims, kc, prm, ws, E, parts)
        torch.cuda.synchronize()
        return E.cpu().numpy(), parts.cpu().numpy()

    hs.hs_get_device_status(clear=True)
    E_ref, parts_ref = score()
    assert hs.hs_get_device_status(clear=True) == 0
    victim = 2
    ws.view(torch.int32)[8 * victim + TX_TEST_WORD] = 64
    E_bad, parts_bad = score()
    st = hs.hs_get_device_status(clear=True)
    assert st & hs.HS_DEV_TMA_TIMEOUT
    others = np.arange(P) != victim
    assert np.array_equal(E_bad[others].view(np.uint32), E_ref[others].view(np.uint32))
    assert np.array_equal(parts_bad[others], parts_ref[others])
    assert np.isfinite(E_bad[victim])  # the victim is scored from the units it finished
    assert int(ws.count_nonzero()) == 0  # the last contributor cleared every slot
    E_again, parts_again = score()
    assert hs.hs_get_device_status(clear=True) == 0
    assert np.array_equal(E_again.view(np.uint32), E_ref.view(np.uint32))
    assert np.array_equal(parts_again, parts_ref)
