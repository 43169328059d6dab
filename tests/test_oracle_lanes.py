"""Pins of the oracle's street-data step (Section IV-A) and path sampling (Section IV-B.2b; readings R-v,
R-w): divider fits recover known parabolas and agree with a least-squares library fit through three
points; straight parallel lanes give the samples at 1/4, 1/2, 3/4 of the own lane and 1/3, 2/3 of each
neighbour in closed form; a curved lane's section direction follows its centre line; missing neighbours
drop their samples; the EGO gets every combination in a fixed order."""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300.scenarios import SplitMix64


def parabola(a, b, c, xs):
    return [[x, a * x * x + b * x + c] for x in xs]


def test_divider_fit_recovers_parabolas_and_matches_polyfit(orc):
    rng = SplitMix64(41)
    for _ in range(500):
        a, b, c = rng.uniform(-0.01, 0.01), rng.uniform(-0.2, 0.2), rng.uniform(-8, 8)
        xs = sorted(rng.uniform(-5, 80) for _ in range(3))
        if min(np.diff(xs)) < 0.5:
            continue
        cf = orc.divider_fit(parabola(a, b, c, xs))
        np.testing.assert_allclose(cf, [a, b, c], rtol=1e-8, atol=1e-10)
        pts = np.array([[x, rng.uniform(-5, 5)] for x in xs])
        np.testing.assert_allclose(orc.divider_fit(pts), np.polyfit(pts[:, 0], pts[:, 1], 2), rtol=1e-7, atol=1e-9)


def test_divider_fit_rejects_repeated_abscissae(orc):
    assert orc.divider_fit([[1.0, 0.0], [1.0, 1.0], [5.0, 2.0]]) is None


STRAIGHT = [parabola(0, 0, y, [0.0, 30.0, 60.0]) for y in (-5.25, -1.75, 1.75, 5.25)]


def test_straight_lanes_closed_form(orc):
    x0, y0, psi0, v0 = 10.0, -3.0, 0.3, 12.0
    p = orc.lane_paths(STRAIGHT, x0, y0, psi0, v0)
    lat = [-5.25 + 3.5 / 3, -5.25 + 7.0 / 3, -0.875, 0.0, 0.875, 1.75 + 3.5 / 3, 1.75 + 7.0 / 3]
    assert p.shape == (7, 3, 3)
    c, s = math.cos(psi0), math.sin(psi0)
    for q, off in enumerate(lat):
        for k, t in enumerate((1.0, 1.5, 2.0)):
            bx = v0 * t
            np.testing.assert_allclose(p[q, k], [x0 + c * bx - s * off, y0 + s * bx + c * off, psi0], atol=1e-12)


def test_curved_lane_direction_follows_the_centre_line(orc):
    dividers = [parabola(0.004, 0.01, -1.75, [0.0, 20.0, 40.0]), parabola(0.004, 0.01, 1.75, [0.0, 20.0, 40.0])]
    p = orc.lane_paths(dividers, 0.0, 0.0, 0.0, 15.0)
    assert p.shape == (3, 3, 3)                        # no neighbours: the own lane's three samples only
    for k, t in enumerate((1.0, 1.5, 2.0)):
        x = 15.0 * t
        slope = 2 * 0.004 * x + 0.01                   # d/dx of the centre line
        assert abs(p[1, k, 2] - math.atan(slope)) < 1e-12
        assert abs(p[1, k, 1] - (0.004 * x * x + 0.01 * x)) < 1e-12
        assert p[0, k, 1] < p[1, k, 1] < p[2, k, 1]    # right to left


def test_missing_neighbour_and_ego_combinations(orc):
    p = orc.lane_paths(STRAIGHT[:3], 0.0, 0.0, 0.0, 10.0)      # own lane and its right neighbour
    assert p.shape == (5, 3, 3)
    e = orc.lane_paths(STRAIGHT, 0.0, 0.0, 0.0, 10.0, ego=True)
    assert e.shape == (343, 3, 3)
    co = orc.lane_paths(STRAIGHT, 0.0, 0.0, 0.0, 10.0)
    for i0 in range(7):
        for i1 in range(7):
            for i2 in range(7):
                q = (i0 * 7 + i1) * 7 + i2
                np.testing.assert_array_equal(e[q, 0], co[i0, 0])
                np.testing.assert_array_equal(e[q, 1], co[i1, 1])
                np.testing.assert_array_equal(e[q, 2], co[i2, 2])


def test_vehicle_outside_every_lane(orc):
    assert orc.lane_paths([parabola(0, 0, y, [0.0, 30.0, 60.0]) for y in (1.0, 4.5)], 0, 0, 0, 10.0) is None
