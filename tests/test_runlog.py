"""Run records (JSON lines) and tracker checkpoints, on the host."""
import io
import json

import numpy as np
import pytest
import torch

from paper_2005_07068_b300 import runlog as RL
from paper_2005_07068_b300 import sweep as SW


def test_generation_records():
    rng = np.random.default_rng(5)
    G, P = 6, 9
    E = rng.uniform(1.0, 30.0, (G, P))
    best = np.minimum.accumulate(E.min(axis=1))
    gbest = rng.normal(0.0, 0.3, (G, 26))
    gt = rng.normal(0.0, 0.3, 26)
    buf = io.StringIO()
    log = RL.RunLog(buf)
    log.generations(4, gbest, best, E, gt, setting="plain 64x6")
    log.run(evals_per_s=1.5e6, roofline_frac=0.02)
    lines = [json.loads(ln) for ln in buf.getvalue().splitlines()]
    assert len(lines) == G + 1
    for g, rec in enumerate(lines[:G]):
        assert rec["type"] == "generation" and rec["frame"] == 4 and rec["gen"] == g + 1
        assert rec["best_E"] == best[g] and rec["min_E"] == E[g].min()
        assert rec["mean_E"] == pytest.approx(E[g].mean(), rel=1e-15)
        assert rec["best_error_deg"] == pytest.approx(float(SW.mean_joint_error_deg(gbest[g], gt)), rel=1e-15)
        assert rec["setting"] == "plain 64x6"
        assert rec["best_E"] <= rec["min_E"] <= rec["mean_E"]
    assert lines[-1] == {"type": "run", "evals_per_s": 1.5e6, "roofline_frac": 0.02}
    with pytest.raises(ValueError):
        log.generations(0, gbest[:3], best, E)


def test_generation_records_without_ground_truth(tmp_path):
    path = str(tmp_path / "run.jsonl")
    with RL.RunLog(path) as log:
        log.generations(0, np.zeros((2, 26)), np.array([3.0, 2.0]), np.array([[3.0, 4.0], [2.0, 5.0]]))
    with RL.RunLog(path) as log:  # appends
        log.run(frames=1)
    lines = [json.loads(ln) for ln in open(path)]
    assert [r["type"] for r in lines] == ["generation", "generation", "run"]
    assert "best_error_deg" not in lines[0] and lines[1]["mean_E"] == 3.5


class _Swarm:
    def __init__(self, x):
        self.x = x


class FakeTracker:
    """The attributes the checkpoint functions use, on the host."""

    def __init__(self, P=5, gens=3, seed=7):
        g = torch.Generator().manual_seed(P * 100 + gens)
        self.gens, self.seed = gens, seed
        self.x_buf = (torch.rand(P, 26, generator=g), torch.rand(P, 26, generator=g))
        self.v = torch.rand(P, 26, generator=g)
        self.E = torch.rand(P, generator=g)
        self.prims = torch.rand(P, 4, 16, generator=g)
        self.swarm = _Swarm(self.x_buf[1])

    def _state(self):
        return [*self.x_buf, self.v, self.E, self.prims]


def test_checkpoint_round_trip(tmp_path):
    a = FakeTracker()
    path = tmp_path / "ck.pt"
    RL.save_checkpoint(a, path, next_frame=12)
    b = FakeTracker(gens=3)
    for t in b._state():
        t.zero_()
    b.swarm.x = b.x_buf[0]
    assert RL.load_checkpoint(b, path) == 12
    assert all(torch.equal(x, y) for x, y in zip(a._state(), b._state()))
    assert b.swarm.x is b.x_buf[1]  # the current position buffer too


def test_checkpoint_rejects_other_settings(tmp_path):
    path = tmp_path / "ck.pt"
    RL.save_checkpoint(FakeTracker(), path, next_frame=1)
    for other in (FakeTracker(gens=4), FakeTracker(seed=8), FakeTracker(P=6)):
        with pytest.raises(ValueError):
            RL.load_checkpoint(other, path)
    ck = torch.load(path, weights_only=True)
    ck["version"] = 99
    torch.save(ck, path)
    with pytest.raises(ValueError):
        RL.load_checkpoint(FakeTracker(), path)
