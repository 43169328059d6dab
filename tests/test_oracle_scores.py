"""Pins of the oracle's trajectory scores (Eq. normTraj with the factors of reading R-x; the paper fixes
neither): the reference hypothesis (keeping speed and lane) scores highest, scores fall with the deviation
in acceleration, steering, path offset or heading, mirror-image hypotheses score alike, a path into the
counter-traffic lane scores half its mirror, a lane change inside a path costs its complexity factor, and
a hand-computed case; the normalised probabilities of an object sum to one."""
import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S


def car(ga, gb, paths=None):
    return S.Obj(S.VEHICLE, 4.5, 1.8, 0.0, 0.0, 0.0, 0.0, 12.0, np.asarray(ga, np.float32), np.asarray(gb, np.float32),
                 S.DEFAULT_VEH_PARAMS, paths=paths)


def test_constant_steering_scores(orc):
    ga = [-6.0, -3.0, 0.0, 2.0]
    gb = [-0.1, -0.05, 0.0, 0.05, 0.1]
    sc = S.Scenario([car(ga, gb), car([0.0], [0.0])])
    w = orc.scores(sc)[0].reshape(len(ga), len(gb))
    assert w.max() == w[2, 2] == 1.0                         # no acceleration, no steering
    assert np.all(np.diff(w[2, 2:]) < 0) and np.all(np.diff(w[:3, 2]) > 0)   # falls off with |delta|, |vdot|
    np.testing.assert_allclose(w[:, 0], w[:, 4], rtol=0, atol=1e-15)      # mirror steering angles alike
    np.testing.assert_allclose(w[:, 1], w[:, 3], rtol=0, atol=1e-15)
    g32 = lambda v: float(np.float32(v))
    n_acc, d_str = 1 / (1 + 3.0 / 2), 1 / (1 + g32(0.05) / 0.05)
    assert abs(w[1, 3] - 0.5 * (n_acc + d_str)) < 1e-12   # vdot = -3, delta = 0.05: (0.4 + 0.5) / 2


def test_path_scores(orc):
    def straight(off):
        return [[10.0 * (k + 1), off, 0.0] for k in range(3)]
    paths = np.array([straight(0.0), straight(-0.875), straight(0.875), straight(-3.5), straight(3.5),
                      [[10.0, 0.0, 0.0], [20.0, 3.5, 0.0], [30.0, 3.5, 0.0]],      # a lane change to the left
                      [[10.0, 0.0, 0.0], [20.0, -3.5, 0.0], [30.0, -3.5, 0.0]]],   # and to the right
                     np.float32)
    sc = S.Scenario([car([0.0, -4.0], np.zeros(len(paths)), paths=paths), car([0.0], [0.0])])
    w = orc.scores(sc)[0].reshape(2, len(paths))
    assert w[0].argmax() == 0 and w[0, 0] == 1.0              # cruising on the lane centre
    assert abs(w[0, 1] - w[0, 2]) < 1e-12                     # within the own lane: mirror offsets alike
    assert abs(w[0, 4] - w[0, 3] / 2) < 1e-12                 # the counter-traffic lane: half its mirror
    d_str = 1 / (1 + 3.5 / 1.75)
    assert abs(w[0, 3] - 0.5 * (1 + d_str)) < 1e-12
    assert abs(w[0, 6] - w[0, 3] / 2) < 1e-12                 # a lane change doubles c_com (1 + 3.5 / 3.5)
    assert np.all(w[1] < w[0])                                # braking scores lower on every path


def test_pedestrian_scores(orc):
    ped = S.Obj(S.PEDESTRIAN, 0, 0, 0.4, 0, 0, 0, 1.5, np.array([0.0, 1.5, 3.0], np.float32),
                np.array([-0.5, 0.0, 0.5], np.float32))
    sc = S.Scenario([car([0.0], [0.0]), ped])
    w = orc.scores(sc)[1].reshape(3, 3)
    assert w.max() == w[1, 1] == 1.0                          # current speed, straight on
    assert abs(w[0, 1] - w[2, 1]) < 1e-12 and abs(w[1, 0] - w[1, 2]) < 1e-12


def test_scores_normalise_to_probabilities(orc):
    sc = S.intersection11(3, n_steps=10, n_acc=5, n_str=5, n_ped_v=3, n_ped_h=3)
    p = orc.normalise(sc, orc.scores(sc))
    off = orc.traj_offsets(sc)
    for q in range(len(sc.objects)):
        assert abs(p[off[q]:off[q + 1]].sum() - 1.0) < 1e-12
