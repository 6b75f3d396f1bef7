"""GPU: batches of independent swarms (uneven ROI sizes, particle counts and
depth types) in one launch per kernel.  Every swarm of a batch must reproduce,
bit for bit, the single-swarm entry points on the same inputs (the batch only
changes which CTA does what; sums are integer fixed point and the random
numbers are keyed by each particle's index within its swarm), and the
single-swarm results are checked against the FP64 oracle on the same scenes."""
import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import build as B
from paper_2005_07068_b300 import handscore as hs
from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import tracker as T
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

# (W, H, P, seed, kw): ROIs from 48x48 to 256x256 with ragged tails, P from 1
# to 256, float32 and uint16 depth, noise on some
SWARMS = [
    (48, 48, 32, 501, dict()),
    (67, 53, 17, 502, dict(noisy=True, f32=False)),
    (128, 96, 64, 503, dict(noisy=True)),
    (31, 200, 1, 504, dict(zoom=2.0)),
    (200, 150, 128, 505, dict(noisy=True, f32=False, spread=2.0)),
    (256, 256, 256, 506, dict(f32=False, noisy=True)),
]
ORACLE_MAX_PIXELS_X_P = 200 * 150 * 128  # scenes the FP64 oracle scores in seconds


@pytest.fixture(scope="module", autouse=True)
def _setup():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hs.hs_get_device_status(clear=True)


@pytest.fixture(scope="module")
def scenes():
    return [C.make_scene(W, H, P, seed, **kw) for W, H, P, seed, kw in SWARMS]


def _batch(scenes, seeds=None):
    dev = torch.device("cuda")
    obs = [hs.Obs.from_numpy(sc.Od, sc.S, dev) for sc in scenes]
    cams = [hs.camera(*[float(v) for v in sc.cam]) for sc in scenes]
    P = [sc.poses.shape[0] for sc in scenes]
    seeds = seeds or [1000 + s for s in range(len(scenes))]
    return obs, cams, hs.Batch(scenes[0].model_g, obs, cams, P, seeds)


def test_batch_fk_and_score_equal_single_swarms(scenes):
    obs, cams, b = _batch(scenes)
    m = scenes[0].model_g
    poses = torch.from_numpy(np.concatenate([sc.poses for sc in scenes])).cuda()
    prims = torch.zeros(b.P_total, m.n_prims, 16, device="cuda")
    kc = torch.zeros(b.P_total, device="cuda")
    hs.hs_obs_prepare_multi(b)
    hs.pose_fk_multi(m, b, poses, prims, kc)
    ws = hs.new_workspace(b.P_total)
    E = torch.zeros(b.P_total, device="cuda")
    parts = torch.zeros(b.P_total, 4, dtype=torch.int32, device="cuda")
    hs.render_score_multi(m, b, prims, kc, hs.score_params(), ws, E, parts)
    # twice in a row: the workspace is left zeroed for the next launch
    E2 = torch.zeros_like(E)
    hs.render_score_multi(m, b, prims, kc, hs.score_params(), ws, E2)
    torch.cuda.synchronize()
    assert torch.equal(E, E2)
    assert hs.hs_get_device_status(clear=True) == 0
    stats_multi = [o.stats.cpu().numpy().copy() for o in obs]
    for s, sc in enumerate(scenes):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        gr = C.run_gpu(sc, debug=True)  # single-swarm entry points (re-prepares its own observation)
        assert np.array_equal(prims[lo:hi].cpu().numpy(), gr.prims), s
        assert np.array_equal(kc[lo:hi].cpu().numpy(), gr.kc), s
        assert np.array_equal(E[lo:hi].cpu().numpy(), gr.E), s
        pa = parts[lo:hi].cpu().numpy()
        assert np.array_equal(pa[:, 1:].view(np.uint32), gr.parts[:, 1:].astype(np.uint32)), s
        assert np.array_equal(pa[:, 0].view(np.float32), gr.parts[:, 0].astype(np.float32)), s
        # per-swarm observation totals
        valid = (sc.S != 0) & (sc.Od.astype(np.float64) > 0)
        assert stats_multi[s].tolist() == [int(valid.sum()), int((sc.S != 0).sum())], s
        # and the single-swarm result against the FP64 oracle
        if sc.W * sc.H * sc.poses.shape[0] <= ORACLE_MAX_PIXELS_X_P:
            C.check_parity(sc, gr, C.run_oracle(sc))


def _track_single(sc, seed, frames, gens, start):
    dev = torch.device("cuda")
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    cam = hs.camera(*[float(v) for v in sc.cam])
    P = sc.poses.shape[0]
    tr = T.Tracker(sc.model_g, cam, P=P, gens=gens, seed=seed)
    out = []
    for f in range(frames):
        tr.run_frame(obs, f, torch.from_numpy(start).cuda() if f == 0 else None, graph=False)
        torch.cuda.synchronize()
        out.append((tr.swarm.x.cpu().numpy().copy(), tr.swarm.gbest.cpu().numpy().copy(),
                    float(tr.swarm.gbest_E.cpu()[0]), tr.prims.cpu().numpy().copy()))
    return out


@pytest.mark.parametrize("graph,variant", [(False, hs.HS_KC_ABDUCTION), (True, hs.HS_KC_ABDUCTION),
                                           (False, hs.HS_KC_ABD_PEN)])
def test_batch_tracking_equals_single_swarm_trackers(scenes, graph, variant):
    """Two frames x 7 generations (mutation at 3 and 6) of every sequence at once
    == each sequence tracked alone, bit for bit; also with the interpenetration
    term in kc (the batched step then copies the collision data once per CTA and
    serves several particles from it)."""
    for sc in scenes:
        sc.model_g.set_kc(variant, 0.05 if variant != hs.HS_KC_ABDUCTION else 0.0)
    try:
        _batch_tracking_equals_single(scenes, graph)
    finally:
        for sc in scenes:
            sc.model_g.set_kc(hs.HS_KC_ABDUCTION, 0.0)


def _batch_tracking_equals_single(scenes, graph):
    frames, gens = 2, 7
    seeds = [0x5EED0000 + 17 * s for s in range(len(scenes))]
    obs, cams, b = _batch(scenes, seeds)
    m = scenes[0].model_g
    starts = np.stack([sc.poses[-1] for sc in scenes]).astype(np.float32)
    bt = T.BatchTracker(m, b, gens=gens)
    res = []
    for f in range(frames):
        bt.run_frame(f, torch.from_numpy(starts).cuda() if f == 0 else None, graph=graph)
        torch.cuda.synchronize()
        res.append((bt.swarm.x.cpu().numpy().copy(), bt.swarm.gbest.cpu().numpy().copy(),
                    bt.swarm.gbest_E.cpu().numpy().copy(), bt.prims.cpu().numpy().copy()))
    assert hs.hs_get_device_status(clear=True) == 0
    for s, sc in enumerate(scenes):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        single = _track_single(sc, seeds[s], frames, gens, starts[s])
        for f in range(frames):
            x, gb, gE, pr = single[f]
            assert np.array_equal(res[f][0][lo:hi], x), (s, f)
            assert np.array_equal(res[f][1][s], gb), (s, f)
            assert res[f][2][s] == np.float32(gE), (s, f)
            assert np.array_equal(res[f][3][lo:hi], pr), (s, f)
        # the search makes progress on every sequence
        assert res[-1][2][s] <= res[0][2][s]


def test_packed_observations_one_copy(scenes):
    """PackedObs: all sequences' frames in one buffer, uploaded in one copy, give
    the same scores as separately allocated observations."""
    sizes = [(sc.W, sc.H) for sc in scenes if sc.Od.dtype == np.uint16]
    sub = [sc for sc in scenes if sc.Od.dtype == np.uint16]
    po = T.PackedObs(sizes, depth_f32=False)
    for s, sc in enumerate(sub):
        po.write_host(s, sc.Od, sc.S)
    po.upload()
    cams = [hs.camera(*[float(v) for v in sc.cam]) for sc in sub]
    m = sub[0].model_g
    b1 = hs.Batch(m, po.obs, cams, [sc.poses.shape[0] for sc in sub], [7] * len(sub))
    _, _, b2 = _batch(sub)
    poses = torch.from_numpy(np.concatenate([sc.poses for sc in sub])).cuda()
    out = []
    for b in (b1, b2):
        prims = torch.zeros(b.P_total, m.n_prims, 16, device="cuda")
        kc = torch.zeros(b.P_total, device="cuda")
        E = torch.zeros(b.P_total, device="cuda")
        hs.hs_obs_prepare_multi(b)
        hs.pose_fk_multi(m, b, poses, prims, kc)
        hs.render_score_multi(m, b, prims, kc, hs.score_params(), hs.new_workspace(b.P_total), E)
        out.append(E.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_batch_of_many_small_swarms():
    """A batch larger than one wave (P_total = 2400 over 40 swarms of 60):
    sampled swarms against the single-swarm path."""
    sc = C.make_scene(96, 72, 60, 511, noisy=True, f32=False)
    S = 40
    rng = np.random.default_rng(5)
    poses = [np.clip(sc.poses + rng.normal(0, 0.02, sc.poses.shape), *(a.astype(np.float32) for a in
                     I.search_limits())).astype(np.float32) for _ in range(S)]
    obs, cams, b = _batch([sc] * S)
    m = sc.model_g
    tp = torch.from_numpy(np.concatenate(poses)).cuda()
    prims = torch.zeros(b.P_total, m.n_prims, 16, device="cuda")
    kc = torch.zeros(b.P_total, device="cuda")
    E = torch.zeros(b.P_total, device="cuda")
    hs.hs_obs_prepare_multi(b)
    hs.pose_fk_multi(m, b, tp, prims, kc)
    hs.render_score_multi(m, b, prims, kc, hs.score_params(), hs.new_workspace(b.P_total), E)
    torch.cuda.synchronize()
    for s in (0, 17, 39):
        gr = C.run_gpu(sc, debug=False, poses=poses[s])
        assert np.array_equal(E[60 * s:60 * (s + 1)].cpu().numpy(), gr.E), s


def test_autotune_picks_a_valid_shape_and_keeps_results(scenes):
    """The autotuner times real candidates, returns one of them, and the choice
    does not change E (single swarm and batch)."""
    sc = scenes[2]
    gr = C.run_gpu(sc, debug=False)
    dev = torch.device("cuda")
    obs = hs.Obs.from_numpy(sc.Od, sc.S, dev)
    hs.hs_obs_prepare(obs)
    cam = hs.camera(*[float(v) for v in sc.cam])
    P = sc.poses.shape[0]
    prims = torch.from_numpy(gr.prims).to(dev)
    kc = torch.from_numpy(gr.kc).to(dev)
    E = torch.zeros(P, device=dev)
    prm, table = hs.render_score_batch_autotune(sc.model_g, obs, cam, prims, kc, hs.score_params(),
                                                hs.new_workspace(P), E, reps=2)
    assert prm.variant in range(1, len(hs.RENDER_VARIANTS)) and prm.ctas_per_particle in hs.TUNE_CTAS
    assert len(table) >= 5 and all(t > 0 for t in table.values())
    assert min(table.values()) == table[f"{hs.render_variant(prm, P)}/k{prm.ctas_per_particle}"]
    assert np.float32(prm.d_M) == 40.0
    E2 = torch.zeros(P, device=dev)
    hs.render_score_batch(sc.model_g, obs, cam, prims, kc, prm, hs.new_workspace(P), E2)
    torch.cuda.synchronize()
    assert np.all(np.abs(E2.cpu().numpy() - gr.E) <= 1e-6 * np.abs(gr.E) + 1e-5)
    # the batch tracker's tuning leaves its state untouched
    obs_l, cams, b = _batch(scenes)
    bt = T.BatchTracker(sc.model_g, b, gens=3)
    before = [t.clone() for t in bt._state()]
    starts = torch.from_numpy(np.stack([s.poses[0] for s in scenes])).cuda()
    table = bt.autotune(starts, reps=1)
    assert bt.score.variant in range(1, len(hs.RENDER_VARIANTS)) and len(table) >= 5
    assert all(torch.equal(a, c) for a, c in zip(before, bt._state()))


@pytest.mark.parametrize("variant", [hs.RENDER_PERSISTENT_8x16, hs.RENDER_PERSISTENT_8x32])
def test_persistent_render_equals_grid_kernels(scenes, variant):
    """The persistent launch (resident CTAs taking particles from a counter)
    gives the grid kernels' E and sums bit for bit: on the uneven batch, on
    2400 particles (several per CTA), twice in a row (its counters return to
    zero), and on a single swarm."""
    obs, cams, b = _batch(scenes)
    m = scenes[0].model_g
    poses = torch.from_numpy(np.concatenate([sc.poses for sc in scenes])).cuda()
    prims = torch.zeros(b.P_total, m.n_prims, 16, device="cuda")
    kc = torch.zeros(b.P_total, device="cuda")
    hs.hs_obs_prepare_multi(b)
    hs.pose_fk_multi(m, b, poses, prims, kc)

    def score(v, bb, pr, k):
        E = torch.zeros(bb.P_total, device="cuda")
        parts = torch.zeros(bb.P_total, 4, dtype=torch.int32, device="cuda")
        ws = hs.new_workspace(bb.P_total)
        hs.render_score_multi(m, bb, pr, k, hs.score_params(variant=v), ws, E, parts)
        hs.render_score_multi(m, bb, pr, k, hs.score_params(variant=v), ws, E, parts)
        torch.cuda.synchronize()
        assert int(ws.count_nonzero()) == 0
        return E.cpu().numpy(), parts.cpu().numpy()

    ref = score(hs.RENDER_STRIPS_8x16, b, prims, kc)
    got = score(variant, b, prims, kc)
    assert np.array_equal(got[0].view(np.uint32), ref[0].view(np.uint32)) and np.array_equal(got[1], ref[1])
    # many particles: the CTAs take several each
    sc = C.make_scene(96, 72, 60, 511, noisy=True, f32=False)
    _, _, b2 = _batch([sc] * 40)
    tp = torch.from_numpy(np.concatenate([sc.poses] * 40)).cuda()
    pr2 = torch.zeros(b2.P_total, m.n_prims, 16, device="cuda")
    kc2 = torch.zeros(b2.P_total, device="cuda")
    hs.hs_obs_prepare_multi(b2)
    hs.pose_fk_multi(m, b2, tp, pr2, kc2)
    ref = score(hs.RENDER_UNITS, b2, pr2, kc2)
    got = score(variant, b2, pr2, kc2)
    assert np.array_equal(got[0].view(np.uint32), ref[0].view(np.uint32)) and np.array_equal(got[1], ref[1])
    # a single swarm
    gr = C.run_gpu(scenes[2], debug=True, variant=variant)
    gu = C.run_gpu(scenes[2], debug=True, variant=hs.RENDER_UNITS)
    assert np.array_equal(gr.E.view(np.uint32), gu.E.view(np.uint32)) and np.array_equal(gr.mask, gu.mask)
    assert hs.hs_get_device_status(clear=True) == 0


def _run_batch_frame(m, b, starts, gens, e_stop, seeds_key=0):
    """One frame of every swarm through the batch calls, step by step; the
    global best E of every swarm after each generation."""
    sw = hs.batch_swarm(b, torch.device("cuda"))
    x_buf = (sw.x, torch.zeros_like(sw.x))
    prims = torch.zeros(b.P_total, m.n_prims, 16, device="cuda")
    kc = torch.zeros(b.P_total, device="cuda")
    ws = hs.new_workspace(b.P_total)
    scale = np.full(26, np.radians(10.0), np.float32)
    scale[:3] = 10.0
    pso = hs.pso_params(e_stop=e_stop)
    hs.hs_obs_prepare_multi(b)
    cur, nxt = x_buf
    sw.x = cur
    hs.pso_init_multi(m, b, sw, torch.from_numpy(starts).cuda(), scale, 0)
    hs.pose_fk_multi(m, b, cur, prims, kc)
    traj = []
    for g in range(1, gens + 1):
        hs.render_score_multi(m, b, prims, kc, hs.score_params(), ws, sw.E)
        sw.x = cur
        hs.pso_step_fk_multi(m, b, sw, nxt, pso, 0, g, prims, kc)
        cur, nxt = nxt, cur
        torch.cuda.synchronize()
        traj.append((sw.gbest_E.cpu().numpy().copy(), sw.gbest.cpu().numpy().copy(), cur.cpu().numpy().copy(),
                     sw.E.cpu().numpy().copy()))
    return traj


def test_device_stop_flags(scenes):
    """Section III.B's stopping rule on the device (e_stop): a swarm whose best
    E falls below e_stop after generation g keeps generation g's bests, stays
    where it was, and is neither scored nor moved again in the frame, while
    the other swarms go on exactly as without the rule; the next frame's init
    starts every swarm again."""
    sub = scenes[:4]
    obs, cams, b = _batch(sub)
    m = sub[0].model_g
    starts = np.stack([sc.poses[-1] for sc in sub]).astype(np.float32)
    gens = 7
    free = _run_batch_frame(m, b, starts, gens, 0.0)
    gE = np.stack([t[0] for t in free])  # [gens, S]
    # a threshold that swarm 0 crosses at generation 3 at the latest
    e_stop = float(np.nextafter(np.float32(gE[2, 0]), np.float32(np.inf)))
    stop_gen = [next((g + 1 for g in range(gens) if gE[g, s] < e_stop), None) for s in range(len(sub))]
    assert stop_gen[0] is not None and stop_gen[0] <= 3
    got = _run_batch_frame(m, b, starts, gens, e_stop)
    last = got[-1]
    for s in range(len(sub)):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        g = stop_gen[s]
        if g is None:  # never stopped: exactly the run without the rule
            assert last[0][s] == free[-1][0][s] and np.array_equal(last[1][s], free[-1][1][s]), s
            assert np.array_equal(last[2][lo:hi], free[-1][2][lo:hi]), s
        else:
            # generation g's bests, and the positions scored at generation g
            assert last[0][s] == gE[g - 1, s] and np.array_equal(last[1][s], free[g - 1][1][s]), s
            scored = free[g - 2][2][lo:hi] if g >= 2 else None
            if scored is not None:
                assert np.array_equal(last[2][lo:hi], scored), s
            assert np.array_equal(last[3][lo:hi], free[g - 1][3][lo:hi]), s  # E not scored again
    # the next frame's init starts every swarm again: with the rule off it
    # equals the free run
    again = _run_batch_frame(m, b, starts, gens, 0.0)
    assert np.array_equal(again[-1][0], free[-1][0]) and np.array_equal(again[-1][2], free[-1][2])
