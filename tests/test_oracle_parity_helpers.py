"""The table comparison used by the parity tests and the benchmark (oracle/parity.py), checked on the CPU
against the oracle's own tables: identical tables agree, a planted non-borderline change is an error, a
change at a step whose margin is within 1 mm is excused, and the band count equals a brute-force count
over every pose pair."""
import numpy as np

from oracle import parity
from paper_2005_06773_gb300 import scenarios as S


def _scene():
    return S.intersection11(5, n_steps=12, n_acc=4, n_str=3, n_ped_v=3, n_ped_h=3)


def test_identical_tables_agree(orc):
    sc = _scene()
    poses = orc.generate(sc)
    tab, poff, pairs = orc.table(sc, poses)
    r = parity.table_agreement(sc, tab, tab.copy(), poses, pairs, poff)
    assert r == {"n_disagree": 0, "n_excused": 0, "n_bad": 0, "bad": []}


def _two_discs(gap_b):
    """Two discs (r = 0.4 m, one hypothesis each) with hand-placed poses: disc A rests at the origin, disc
    B's centre is 0.8 m + gap_b[k] away at step k, so the oracle's margin at step k is gap_b[k]."""
    ped = lambda x: S.Obj(S.PEDESTRIAN, 0, 0, 0.4, x, 0.0, 0.0, 0.0, np.array([0.0], np.float32),
                          np.array([0.0], np.float32))
    sc = S.Scenario([ped(0.0), ped(5.0)], tau=0.1, n_steps=len(gap_b), substeps=5)
    N = len(gap_b)
    x = np.concatenate([np.zeros(N), 0.8 + np.asarray(gap_b, np.float64)])
    poses = {"x": x, "y": np.zeros(2 * N), "c": np.ones(2 * N), "s": np.zeros(2 * N)}
    return sc, poses


def test_planted_errors_and_borderline_excuses(orc):
    sc, poses = _two_discs([1.2, 0.0005, -0.3])
    tab, poff, pairs = orc.table(sc, poses)
    np.testing.assert_allclose(orc.margins(sc, poses, [0], [0], [1], [1])[0], [1.2, 0.0005, -0.3], atol=1e-7)  # r rounded to FP32
    assert tab.tolist() == [2]
    agree = lambda g: parity.table_agreement(sc, np.array([g], np.int16), tab, poses, pairs, poff)
    assert agree(2)["n_disagree"] == 0
    assert agree(1)["n_excused"] == 1        # a hit where the oracle sees a 0.5 mm gap: borderline
    assert agree(0)["n_bad"] == 1            # a hit across a 1.2 m gap
    assert agree(-1)["n_bad"] == 1           # the 0.3 m overlap at step 2 missed
    sc2, poses2 = _two_discs([1.2, -0.0005, -0.3])
    tab2, _, _ = orc.table(sc2, poses2)
    assert tab2.tolist() == [1]
    r = parity.table_agreement(sc2, np.array([2], np.int16), tab2, poses2, pairs, poff)
    assert r["n_excused"] == 1 and r["n_bad"] == 0   # a 0.5 mm overlap missed: borderline
    r = parity.table_agreement(sc2, np.array([-1], np.int16), tab2, poses2, pairs, poff)
    assert r["n_bad"] == 1


def test_band_count_equals_brute_force(orc):
    sc = _scene()
    poses = orc.generate(sc)
    off = orc.traj_offsets(sc)
    pairs = orc.pair_list(sc)
    for tol in (1e-3, 0.05, 0.3):
        want = 0
        for a, b in pairs:
            i, j = np.meshgrid(np.arange(off[a], off[a + 1]), np.arange(off[b], off[b + 1]), indexing="ij")
            m = orc.margins(sc, poses, np.full(i.size, a), i.ravel(), np.full(j.size, b), j.ravel())
            want += int((np.abs(m) < tol).sum())
        assert parity.band_count(sc, poses, tol=tol, rows=7) == want
    assert parity.band_count(sc, poses, tol=0.3) > 0
