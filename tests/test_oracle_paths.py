"""Pins of the oracle's path hypotheses (Section IV-B.2b, Eq. controller; readings R-s, R-t, R-u): a vehicle
on its path never steers and matches the pinned constant-steering integration; mirror images and rigid
motions of the whole set-up transform the trajectory alike (which fixes the signs of the distance and yaw
errors); the steering limits hold at every sub-step; a lane change converges; the sections switch at
1.0 s and 1.5 s."""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S

TAU, K = float(np.float32(0.1)), 5
TAU_I = TAU / K


def straight(y=0.0, psi=0.0, x=0.0):
    return [[x, y, psi]] * 3


def test_on_path_vehicle_never_steers_and_matches_constant_steering(orc):
    for v0, acc in ((15.0, 0.0), (10.0, -3.0), (8.0, 2.0), (1.5, 0.5)):
        r = orc.path_steering(-20.0, 3.0, 0.0, v0, acc, straight(3.0), n_steps=30, tau=TAU, substeps=K)
        assert np.all(r["delta"] == 0.0)
        car = S.Obj(S.VEHICLE, 4.5, 1.8, 0.0, -20.0, 3.0, 0.0, v0, np.array([acc]), np.array([0.0]),
                    S.DEFAULT_VEH_PARAMS)
        ref = orc.generate(S.Scenario([car], tau=TAU, n_steps=30, substeps=K))
        np.testing.assert_array_equal(r["x"], ref["x"][0])
        np.testing.assert_array_equal(r["y"], ref["y"][0])


@pytest.mark.parametrize("v0,acc,y0,psi0", [(15.0, 0.0, -1.75, 0.0), (12.0, -4.0, 1.0, 0.05), (20.0, 2.0, 0.6, -0.1)])
def test_mirror_symmetry(orc, v0, acc, y0, psi0):
    path = [[0.0, 0.5, 0.02], [10.0, -1.0, -0.03], [25.0, 2.0, 0.0]]
    mirror = [[x, -y, -p] for x, y, p in path]
    a = orc.path_steering(-10.0, y0, psi0, v0, acc, path, n_steps=40, tau=TAU, substeps=K)
    b = orc.path_steering(-10.0, -y0, -psi0, v0, acc, mirror, n_steps=40, tau=TAU, substeps=K)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-9)
    np.testing.assert_allclose(a["y"], -b["y"], atol=1e-9)
    np.testing.assert_allclose(a["psi"], -b["psi"], atol=1e-12)
    np.testing.assert_allclose(a["delta"], -b["delta"], atol=1e-12)


def test_rigid_motion_invariance(orc):
    path = [[0.0, 1.75, 0.0], [12.0, 1.75, 0.0], [20.0, 5.25, 0.1]]
    base = orc.path_steering(-15.0, -1.0, 0.1, 14.0, -1.0, path, n_steps=40, tau=TAU, substeps=K)
    for th, tx, ty in ((math.pi / 2, 30.0, -40.0), (2.5, -7.0, 3.0), (-1.2, 100.0, 50.0)):
        c, s = math.cos(th), math.sin(th)
        rot = lambda x, y: (tx + c * x - s * y, ty + s * x + c * y)
        moved = [[*rot(x, y), p + th] for x, y, p in path]
        x0, y0 = rot(-15.0, -1.0)
        r = orc.path_steering(x0, y0, 0.1 + th, 14.0, -1.0, moved, n_steps=40, tau=TAU, substeps=K)
        bx, by = rot(base["x"], base["y"])
        np.testing.assert_allclose(r["x"], bx, atol=1e-8)
        np.testing.assert_allclose(r["y"], by, atol=1e-8)
        np.testing.assert_allclose(np.unwrap(r["psi"]) - th, np.unwrap(base["psi"]), atol=1e-9)
        np.testing.assert_allclose(r["delta"], base["delta"], atol=1e-10)


def test_steering_limits_at_every_substep(orc):
    for path, y0, psi0 in ((straight(), -3.5, 0.0), (straight(), 6.0, 0.8), ([[0, 0, 0], [0, 10, 1.5], [0, -10, -1.5]], 0.0, 0.0)):
        r = orc.path_steering(-10.0, y0, psi0, 12.0, 0.0, path, n_steps=40, tau=TAU, substeps=K)
        d = np.concatenate([[0.0], r["delta"]])
        assert np.all(np.abs(d) <= 0.5 + 1e-15)
        assert np.all(np.abs(np.diff(d)) <= 0.5 * TAU_I * (1 + 1e-12))
        assert np.max(np.abs(np.diff(d))) > 0.9 * 0.5 * TAU_I     # large errors do hit the rate limit


@pytest.mark.parametrize("v0", [10.0, 15.0, 25.0])
def test_lane_change_converges(orc, v0):
    """Starting one lane (3.5 m) or half a lane beside a straight path, the lateral error shrinks without
    changing sign (a little ringing after a full lane change at speed) and the heading settles back toward
    the path direction."""
    for y0 in (-3.5, -1.75, 1.75):
        r = orc.path_steering(-30.0, y0, 0.0, v0, 0.0, straight(), n_steps=50, tau=TAU, substeps=K)
        e = np.abs(r["y"])
        assert np.all(np.sign(r["y"]) == np.sign(y0))
        assert e[-1] < 0.35 * abs(y0)
        assert np.all(np.diff(e[:8]) <= 1e-9)                   # closing in during the first 0.8 s
        assert np.all(e[10:] <= e[10] + 1e-9)                   # and never wider again after 1 s
        assert abs(r["psi"][-1]) < 0.25 * np.max(np.abs(r["psi"]))
        first = r["delta"][:K]
        assert np.all(np.sign(first[first != 0]) == np.sign(-y0))  # steers toward the path at once


def test_sections_switch_at_one_and_one_and_a_half_seconds(orc):
    """Sections on y = 0, then y = 3.5 from 1.0 s: the command changes sign of its target exactly there."""
    path = [[0.0, 0.0, 0.0], [0.0, 3.5, 0.0], [0.0, 3.5, 0.0]]
    r = orc.path_steering(-30.0, 0.0, 0.0, 15.0, 0.0, path, n_steps=40, tau=TAU, substeps=K)
    n1 = next(n for n in range(200) if n * TAU_I >= 1.0)
    assert np.all(r["delta"][:n1] == 0.0)                      # on the first section: no steering
    assert r["delta"][n1] > 0.0                                # the second section lies to the left
    assert r["y"][-1] > 1.5
    path2 = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, -3.5, 0.0]]
    r2 = orc.path_steering(-30.0, 0.0, 0.0, 15.0, 0.0, path2, n_steps=40, tau=TAU, substeps=K)
    n2 = next(n for n in range(200) if n * TAU_I >= 1.5)
    assert np.all(r2["delta"][:n2] == 0.0) and r2["delta"][n2] < 0.0


def test_scenario_paths_feed_generation(orc):
    """Through the scenario path: a two-path car gives, per acceleration, exactly the single-hypothesis
    integrations of its paths."""
    paths = np.array([straight(0.0), straight(3.5)], np.float32)
    car = S.Obj(S.VEHICLE, 4.5, 1.8, 0.0, -20.0, 0.0, 0.0, 12.0, np.array([0.0, -2.0]), np.zeros(2),
                S.DEFAULT_VEH_PARAMS, paths=paths)
    ref = orc.generate(S.Scenario([car], tau=TAU, n_steps=30, substeps=K))
    for ia, acc in enumerate((0.0, -2.0)):
        for ib in range(2):
            r = orc.path_steering(-20.0, 0.0, 0.0, 12.0, acc, paths[ib].astype(float),
                                  params=np.asarray(S.DEFAULT_VEH_PARAMS, np.float32).astype(float),
                                  n_steps=30, tau=TAU, substeps=K)
            np.testing.assert_array_equal(ref["x"][2 * ia + ib], r["x"])
            np.testing.assert_array_equal(ref["y"][2 * ia + ib], r["y"])


# Eq. (controller) by hand, in degrees: g = |(-0.018 v + 1.5) d|, delta = (g + 0.5) d + (-g + 9.5)(3.8197 e).
# (v m/s, d_path m, e_psi rad, delta deg); each gain changes at least one of these values.
CONTROLLER_CASES = [
    (10.0, 1.0, 0.0, 1.82),            # g = 1.32
    (10.0, -1.0, 0.0, -1.82),          # the magnitude in g, the sign from d
    (100.0, 1.0, 0.0, 0.8),            # -0.018 v + 1.5 < 0: g = |-0.3| = 0.3
    (5.0, 0.0, -0.1, -3.628715),       # g = 0: 9.5 x 3.8197 x (-0.1)
    (20.0, -0.5, 0.05, 1.17049605),    # g = 0.57: -0.535 + 8.93 x 0.190985
    (30.0, 2.0, 0.02, 5.41906652),     # g = 1.92: 4.84 + 7.58 x 0.076394
]


@pytest.mark.parametrize("v,d,e,want_deg", CONTROLLER_CASES)
def test_controller_gains_by_hand(orc, v, d, e, want_deg):
    """The first sub-step's steering angle is the controller's command itself: the vehicle starts at the
    origin heading along x with beta = 0, so its centre of gravity predicted 0.5 s ahead is (0.5 v, 0);
    section 0 passes through (0.5 v, d / cos e) with direction e, so the line lies d to the left of that
    point (d_path = d) and the yaw error is e.  With tau_i = 10 s the rate limit (0.5 rad/s x tau_i) is out of
    reach and every command here stays below the 0.5 rad angle limit."""
    path = [[0.5 * v, d / math.cos(e), e]] * 3
    r = orc.path_steering(0.0, 0.0, 0.0, v, 0.0, path, n_steps=1, tau=10.0, substeps=1)
    assert r["delta"][0] == pytest.approx(math.radians(want_deg), rel=1e-12, abs=1e-15)
