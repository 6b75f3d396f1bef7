"""Pins of the oracle's swarm (Section III.B, Eq. 6-7, mutation).

A hand-computed single step with injected r1, r2; clamping; monotone personal
and global bests; the strict-improvement and lowest-index rules; mutation of
exactly the worst half on the 20 finger dims; the tracking initialisation;
and convergence on a convex bowl (a sign error in Eq. 6 diverges).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_07068_b300 import inputs as I

LO, HI = I.search_limits()
W = oracle.pso_w()


def test_single_step_hand_computed():
    x = np.full(26, 0.1)
    v = np.full(26, 0.02)
    p = np.full(26, 0.3)
    g = np.full(26, 0.5)
    r1 = np.full(26, 0.5)
    r2 = np.full(26, 0.25)
    lo, hi = np.full(26, -10.0), np.full(26, 10.0)
    xo, vo = oracle.pso_update(x, v, p, g, r1, r2, lo, hi, c1=2.8, c2=1.3)
    # v' = w (0.02 + 2.8*0.5*0.2 + 1.3*0.25*0.4) = w * 0.43 ; x' = 0.1 + v'
    assert np.allclose(vo, 0.43 * 0.7298437881, atol=1e-10)
    assert np.allclose(xo, 0.1 + 0.43 * 0.7298437881, atol=1e-10)
    # clamped position, velocity kept
    xo2, vo2 = oracle.pso_update(x, v, p, g, r1, r2, lo, np.full(26, 0.2))
    assert np.all(xo2 == 0.2) and np.allclose(vo2, vo)


def _swarm(P=16, seed=5):
    pose = I.ground_truth_pose(seed)
    return oracle.pso_init(P, pose, I.perturbation_scale(), LO, HI, 77, 3)


def test_init():
    pose = I.ground_truth_pose(5)
    sw = _swarm()
    assert np.array_equal(sw.x[0], np.clip(pose, LO, HI))
    assert np.all(sw.x >= LO) and np.all(sw.x <= HI)
    assert np.all(np.abs(sw.x - pose) <= I.perturbation_scale() + 1e-12)
    assert np.all(sw.v == 0) and np.array_equal(sw.pbest, sw.x)
    assert np.all(np.isinf(sw.pbest_E)) and math.isinf(sw.gbest_E)
    assert len({tuple(r) for r in sw.x}) == len(sw.x)  # distinct particles
    sw2 = _swarm()
    assert np.array_equal(sw.x, sw2.x)  # counter-based: reproducible
    sw3 = oracle.pso_init(16, pose, I.perturbation_scale(), LO, HI, 78, 3)
    assert not np.array_equal(sw.x, sw3.x)


def test_personal_and_global_best_rules():
    sw = _swarm(8)
    E = np.array([5.0, 3.0, 3.0, 9.0, 7.0, 4.0, 8.0, 6.0])
    s1 = oracle.pso_step(sw, E, LO, HI, 77, 3, 1, mutate_every=0)
    assert np.array_equal(s1.pbest_E, E)
    assert np.array_equal(s1.pbest, sw.x)
    assert s1.gbest_E == 3.0 and np.array_equal(s1.gbest, sw.x[1])  # lowest index wins the tie
    E2 = np.array([5.0, 2.0, 3.5, 9.0, 1.0, 4.0, np.nan, 6.0])  # equal E does not replace (strict <)
    s2 = oracle.pso_step(s1, E2, LO, HI, 77, 3, 2, mutate_every=0)
    assert np.array_equal(s2.pbest[0], s1.pbest[0])            # 5.0 == 5.0: kept
    assert np.array_equal(s2.pbest[1], s1.x[1])                # improved
    assert np.array_equal(s2.pbest[2], s1.pbest[2])            # worse: kept
    assert s2.pbest_E[6] == 8.0                                # NaN never improves
    assert s2.gbest_E == 1.0 and np.array_equal(s2.gbest, s1.x[4])


def test_bests_monotone_and_clamped():
    sw = _swarm(12)
    rng = np.random.default_rng(0)
    prev = np.inf
    prev_pb = sw.pbest_E.copy()
    for g in range(1, 10):
        E = rng.uniform(0, 50, 12)
        sw = oracle.pso_step(sw, E, LO, HI, 77, 3, g)
        assert sw.gbest_E <= prev and np.all(sw.pbest_E <= prev_pb)
        assert sw.gbest_E == sw.pbest_E.min()
        prev, prev_pb = sw.gbest_E, sw.pbest_E.copy()
        assert np.all(sw.x >= LO) and np.all(sw.x <= HI)
        c = np.clip(sw.x, LO, HI)
        assert np.array_equal(c, sw.x)  # clamping idempotent


@pytest.mark.parametrize("P", [8, 9, 16])
def test_mutation_worst_half(P):
    sw = _swarm(P)
    rng = np.random.default_rng(P)
    E = rng.permutation(P).astype(float)
    E[1] = E[2]  # a tie: the larger index is the worse
    plain = oracle.pso_step(sw, E, LO, HI, 77, 3, 3, mutate_every=0)
    mut = oracle.pso_step(sw, E, LO, HI, 77, 3, 3, mutate_every=3)
    order = sorted(range(P), key=lambda i: (E[i], i))
    worst = set(order[P - P // 2:])
    for i in range(P):
        if i in worst:
            assert np.array_equal(mut.x[i, :6], plain.x[i, :6])
            assert not np.array_equal(mut.x[i, 6:], plain.x[i, 6:])
            assert np.all(mut.v[i, 6:] == 0) and np.array_equal(mut.v[i, :6], plain.v[i, :6])
            assert np.all(mut.x[i, 6:] >= LO[6:]) and np.all(mut.x[i, 6:] < HI[6:])
        else:
            assert np.array_equal(mut.x[i], plain.x[i]) and np.array_equal(mut.v[i], plain.v[i])
    assert np.array_equal(mut.pbest, plain.pbest)  # personal bests kept
    # not a mutation generation: identical
    m2 = oracle.pso_step(sw, E, LO, HI, 77, 3, 4, mutate_every=3)
    p2 = oracle.pso_step(sw, E, LO, HI, 77, 3, 4, mutate_every=0)
    assert np.array_equal(m2.x, p2.x)


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_swarm_converges_on_convex_bowl(seed):
    """With Eq. 6-7 as printed, a 64-particle swarm spread over the box
    contracts onto the minimum of |x - x*|^2 (a flipped sign in Eq. 6 or a
    missing constriction drives it to the walls instead)."""
    target = np.clip(I.ground_truth_pose(seed), LO, HI)
    scale = HI - LO
    sw = oracle.pso_init(64, (LO + HI) / 2, scale / 2, LO, HI, 9, 0)

    def f(x):
        return (((x - target) / scale) ** 2).sum(axis=1)

    first = None
    for g in range(1, 151):
        sw = oracle.pso_step(sw, f(sw.x), LO, HI, 9, 0, g, mutate_every=0)
        if first is None:
            first = sw.gbest_E
    assert sw.gbest_E < 0.01 * first
    assert np.abs((sw.gbest - target) / scale).max() < 0.15
