"""Pins of the hypothesis grids that feed both the oracle and the CUDA path (Section IV-B.2a, IV-B.3).

The longitudinal rule of Section IV-B.2a samples the minimum, zero and the maximum of the acceleration
range and spreads the remaining samples evenly over the negative part; the values below are written out by
hand as fractions, not recomputed from the rule.
"""
import math

import numpy as np

from paper_2005_06773_gb300 import scenarios as S

F32 = np.float32


def test_paper_rule_four_samples_on_minus6_plus2():
    np.testing.assert_array_equal(S.accel_grid_paper(4, -6.0, 2.0), np.array([-6.0, -3.0, 0.0, 2.0], F32))


def test_paper_rule_three_samples_is_min_zero_max():
    np.testing.assert_array_equal(S.accel_grid_paper(3, -8.0, 3.0), np.array([-8.0, 0.0, 3.0], F32))


def test_paper_rule_21_samples_on_minus8_plus3():
    want = [-8.0, -144 / 19, -136 / 19, -128 / 19, -120 / 19, -112 / 19, -104 / 19, -96 / 19, -88 / 19, -80 / 19,
            -72 / 19, -64 / 19, -56 / 19, -48 / 19, -40 / 19, -32 / 19, -24 / 19, -16 / 19, -8 / 19, 0.0, 3.0]
    got = S.accel_grid_paper(21, -8.0, 3.0)
    assert got.dtype == F32 and got.size == 21
    np.testing.assert_array_equal(got, np.array(want, F32))


def test_tiny_crossing_grids():
    sc = S.tiny_crossing(1)
    for o in sc.objects:
        np.testing.assert_array_equal(o.grid_a, np.array([-6.0, -3.0, 0.0, 2.0], F32))
        np.testing.assert_array_equal(o.grid_b, np.array([-0.1, -1 / 30, 1 / 30, 0.1], F32))
        assert o.n_hyp == 16


def test_intersection11_grids_and_counts():
    sc = S.intersection11(2)
    cars = [o for o in sc.objects if o.kind == S.VEHICLE]
    peds = [o for o in sc.objects if o.kind == S.PEDESTRIAN]
    assert len(cars) == 7 and len(peds) == 4
    for o in cars:
        np.testing.assert_array_equal(o.grid_a, S.accel_grid_paper(21, -8.0, 3.0))
        np.testing.assert_array_equal(o.grid_b, np.array([-0.3 + 0.03 * q for q in range(21)], F32))
        assert (o.length, o.width) == (F32(4.5), F32(1.8)) and o.n_hyp == 441
    for o in peds:
        np.testing.assert_array_equal(o.grid_a, np.array([0.3 * q for q in range(11)], F32))
        np.testing.assert_array_equal(o.grid_b, np.array([math.radians(-60 + 12 * q) for q in range(11)], F32))
        assert o.radius == F32(0.4) and o.n_hyp == 121
    assert sc.n_steps == 30 and sc.n_traj_pairs() == 5_666_055 and sc.n_tests() == 169_981_650
