"""The full-frame sweep's accuracy bookkeeping on CPU: the joint-angle error
matches the oracle's definition, and the summary / selection follow from the
per-frame results."""
import numpy as np

import oracle
from paper_2005_07068_b300 import inputs as I
from paper_2005_07068_b300 import sweep as SW


def test_mean_joint_error_matches_oracle():
    rng = np.random.default_rng(3)
    lo, hi = I.search_limits()
    a = I.sample_poses(rng, 20, lo, hi)
    b = I.sample_poses(rng, 20, lo, hi)
    ours = SW.mean_joint_error_deg(a, b)
    for k in range(20):
        assert abs(ours[k] - oracle.mean_joint_error_deg(a[k], b[k])) < 1e-9
    # translation does not count; one angle off by 23 degrees is 1 degree on average
    c = a[0].copy()
    c[:3] += 50.0
    assert SW.mean_joint_error_deg(c, a[0]) == 0.0
    c[10] += np.radians(23.0)
    assert abs(SW.mean_joint_error_deg(c, a[0]) - 1.0) < 1e-12


def test_summary_and_fastest_setting():
    rs = [SW.FrameResult(f, 10.0 + f, e, 1.0) for f, e in enumerate([1.0, 4.0, 6.0, 3.0])]
    s = SW.summarize(rs)
    assert s["within_fraction"] == 0.75
    assert s["final_error_deg_mean"] == 3.5 and s["frame_ms_mean"] == 11.5
    fast_bad = dict(within_fraction=0.5, frame_ms_mean=1.0)
    slow_ok = dict(within_fraction=0.95, frame_ms_mean=9.0)
    mid_ok = dict(within_fraction=0.9, frame_ms_mean=4.0)
    assert SW.fastest_within([fast_bad, slow_ok, mid_ok]) is mid_ok
    assert SW.fastest_within([fast_bad]) is None
