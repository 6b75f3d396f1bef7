"""Pins of the oracle's constants and random numbers against printed values.

Tables 1-2 (Section II.A), the constants of Section III.A/III.B, the published
value of the constriction factor and the Philox4x32-10 known-answer vectors.
"""
import math

import numpy as np

import oracle
from paper_2005_07068_b300 import inputs as I
from tests.conftest import golden_path


def _read(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_joint_limits_match_tables_1_2():
    lo, hi = I.paper_joint_limits()
    for row in _read("paper_tables_1_2.txt"):
        if row[0] == "table1":
            f = I.FINGERS.index(row[1])
            for j, cell in enumerate(row[2:]):
                a, b = (float(x) for x in cell.split(":"))
                k = 6 + 4 * f + j
                assert math.isclose(lo[k], math.radians(a), abs_tol=1e-15)
                assert math.isclose(hi[k], math.radians(b), abs_tol=1e-15)
        else:
            k = ["x_c", "y_c", "z_c", "theta_x", "theta_y", "theta_z"].index(row[1])
            a, b = (float(x) for x in row[2].split(":"))
            scale = 1000.0 if k < 3 else math.pi / 180.0
            assert math.isclose(lo[k], a * scale, rel_tol=1e-15, abs_tol=1e-12)
            assert math.isclose(hi[k], b * scale, rel_tol=1e-15, abs_tol=1e-12)


def test_search_limits_inside_tables():
    lo, hi = I.paper_joint_limits()
    slo, shi = I.search_limits()
    assert np.all(slo >= lo) and np.all(shi <= hi) and np.all(slo < shi)
    # finger dims are exactly Table 1
    assert np.array_equal(slo[6:], lo[6:]) and np.array_equal(shi[6:], hi[6:])


def test_cost_and_pso_constants():
    c = {r[0]: float(r[1]) for r in _read("constants.txt")}
    dm, dM, lam, lamk = oracle.DEFAULT_PARAMS
    assert dm == c["d_m_cm"] * 10 and dM == c["d_M_cm"] * 10
    assert lam == c["lambda"] and lamk == c["lambda_k"]
    assert oracle.PSO_C1 == c["c1"] and oracle.PSO_C2 == c["c2"]


def test_constriction_factor_published_value():
    c = {r[0]: float(r[1]) for r in _read("constants.txt")}
    assert abs(oracle.pso_w(2.8, 1.3) - c["w_psi_4_1"]) < 1e-10
    # the factor depends on psi only
    assert abs(oracle.pso_w(2.05, 2.05) - c["w_psi_4_1"]) < 1e-10


def test_philox_known_answers():
    for row in _read("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(v[:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_mapping_exact():
    assert oracle.uniform(0) == 0.0
    assert oracle.uniform(255) == 0.0
    assert oracle.uniform(256) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # representable in float32 as well
    for u in (0x12345678, 0xDEADBEEF, 0x80000000):
        x = oracle.uniform(u)
        assert float(np.float32(x)) == x
