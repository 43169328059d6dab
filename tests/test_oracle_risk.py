"""Pins of the oracle's risk assessment (Section IV-D): brute force over joint CO trajectory assignments,
the telescoping identity of the chronological scaling (Eq. p21), probability bounds and exact rational
values for uniform weights."""
import itertools

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S


def tiny_structure(hs, n_steps=6, ego=0, pair_mode=S.ALL_PAIRS):
    objs = []
    for h in hs:
        objs.append(S.Obj(S.VEHICLE, 4.5, 1.8, 0.0, 0, 0, 0, 10, np.zeros(h), np.zeros(1), S.DEFAULT_VEH_PARAMS))
    return S.Scenario(objs, n_steps=n_steps, ego=ego, pair_mode=pair_mode)


def random_table(orc, sc, seed, p_hit=0.35):
    rng = S.SplitMix64(seed)
    poff = orc.pair_offsets(sc)
    tab = np.full(int(poff[-1]), -1, np.int16)
    for i in range(tab.size):
        if rng.uniform() < p_hit:
            tab[i] = rng.randint(0, sc.n_steps - 1)
    return tab


def ego_rows(orc, sc, tab):
    """T(e, i, b, j) for every CO b as dict b -> [h_e, h_b] array, read from either pair orientation."""
    off = orc.traj_offsets(sc)
    h = np.diff(off)
    poff = orc.pair_offsets(sc)
    rows = {}
    for q, (a, b) in enumerate(orc.pair_list(sc)):
        blk = tab[poff[q]:poff[q + 1]].reshape(h[a], h[b])
        if a == sc.ego:
            rows[b] = blk
        elif b == sc.ego:
            rows[a] = blk.T
    return rows


@pytest.mark.parametrize("ego", [0, 1, 2])
def test_independent_risk_equals_brute_force(orc, ego):
    """Enumerate every joint assignment of the COs' trajectories (independent, with their probabilities):
    P(EGO trajectory i collides with someone) = 1 - prod_b (1 - P_b(i)).  The oracle's per-object
    independence measure must equal it exactly (up to rounding)."""
    sc = tiny_structure([5, 4, 3], ego=ego)
    tab = random_table(orc, sc, 41 + ego)
    w = S.random_weights(sc, 42)
    r = orc.risk(sc, tab, weights=w)
    prob = r["prob"]
    off = orc.traj_offsets(sc)
    rows = ego_rows(orc, sc, tab)
    cos = sorted(rows)
    pb = {b: prob[off[b]:off[b + 1]] for b in cos}
    for i in range(int(off[ego + 1] - off[ego])):
        total = 0.0
        for js in itertools.product(*[range(len(pb[b])) for b in cos]):
            pr = np.prod([pb[b][j] for b, j in zip(cos, js)])
            if any(rows[b][i, j] >= 0 for b, j in zip(cos, js)):
                total += pr
        assert abs(r["indep"][i] - total) < 1e-14


def test_chronological_scaling_telescopes_and_is_bounded(orc):
    """Eq. p21: scaling each later combination by the survivor product of the earlier ones sums to
    1 - prod(1 - p) over the EGO trajectory's colliding entries, whatever the order; and
    0 <= cond <= indep <= naive (Weierstrass product inequality, union bound)."""
    sc = tiny_structure([6, 5, 4, 3], n_steps=5)
    tab = random_table(orc, sc, 43, p_hit=0.5)
    r = orc.risk(sc, tab, weights=S.random_weights(sc, 44))
    prob = r["prob"]
    off = orc.traj_offsets(sc)
    rows = ego_rows(orc, sc, tab)
    for i in range(6):
        ps = [prob[off[b] + j] for b in rows for j in range(rows[b].shape[1]) if rows[b][i, j] >= 0]
        assert abs(r["cond"][i] - (1.0 - np.prod([1 - p for p in ps]))) < 1e-14
        assert abs(r["naive"][i] - sum(ps)) < 1e-14
        assert r["hits"][i] == len(ps)
        assert -1e-15 <= r["cond"][i] <= r["indep"][i] + 1e-15 <= r["naive"][i] + 2e-15


def test_single_collision_per_trajectory_makes_all_measures_equal(orc):
    sc = tiny_structure([4, 4, 4], n_steps=4)
    poff = orc.pair_offsets(sc)
    tab = np.full(int(poff[-1]), -1, np.int16)
    # EGO trajectory i collides only with CO 1 trajectory i at step i
    for i in range(4):
        tab[poff[0] + i * 4 + i] = i
    r = orc.risk(sc, tab)
    np.testing.assert_allclose(r["cond"], r["naive"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["indep"], r["naive"], rtol=0, atol=1e-15)


def test_uniform_weights_give_rational_crash_probability(orc):
    """Eq. totalCrashProb with uniform probabilities: p_cra = sum_b C_eb / (h_e h_b)."""
    sc = tiny_structure([7, 3, 5, 2], n_steps=8)
    tab = random_table(orc, sc, 45)
    r = orc.risk(sc, tab)
    h = np.diff(orc.traj_offsets(sc))
    rows = ego_rows(orc, sc, tab)
    expect = sum((rows[b] >= 0).sum() / (h[0] * h[b]) for b in rows)
    assert abs(r["p_cra"] - expect) < 1e-15
    for q, (a, b) in enumerate(orc.pair_list(sc)):
        assert r["count"][q] == (tab[orc.pair_offsets(sc)[q]:orc.pair_offsets(sc)[q + 1]] >= 0).sum()
        assert abs(r["P"][q] - r["count"][q] / (h[a] * h[b])) < 1e-15


def test_histograms_sum_to_totals(orc):
    sc = tiny_structure([5, 6, 4], n_steps=7)
    tab = random_table(orc, sc, 46)
    r = orc.risk(sc, tab, weights=S.random_weights(sc, 47))
    np.testing.assert_array_equal(r["count_k"].sum(1), r["count"])
    np.testing.assert_allclose(r["H"].sum(1), r["P"], atol=1e-15)
    assert abs(r["attr_obj"].sum() - r["p_cra_cond"]) < 1e-15
    assert abs(r["attr_step"].sum() - r["p_cra_cond"]) < 1e-15
    assert r["attr_obj"][sc.ego] == 0.0


def test_paper_conditional_example(orc):
    """Eq. p21 worked by hand: along one EGO trajectory, combination A (p = 0.5) at step 1, B (p = 0.4) at
    step 2 and C (p = 0.2) at step 3 contribute P(A) = 0.5, P(B and not A) ~ 0.5 * 0.4 = 0.2 and
    P(C and not B and not A) ~ 0.5 * 0.6 * 0.2 = 0.06.  The objects are numbered against time order
    (A is CO 3, C is CO 1) so that only a chronological ordering gives these shares."""
    sc = tiny_structure([1, 5, 5, 2], n_steps=5)
    # CO 3: trajectory 0 with weight 1 (p = 0.5) collides at step 1
    # CO 2: trajectory 0 with weight 2 (p = 0.4) at step 2; CO 1: trajectory 0 (p = 0.2) at step 3
    w = [np.ones(1), np.array([1.0, 1.0, 1.0, 1.0, 1.0]), np.array([2.0, 0.75, 0.75, 0.75, 0.75]),
         np.array([1.0, 1.0])]
    poff = orc.pair_offsets(sc)
    tab = np.full(int(poff[-1]), -1, np.int16)
    tab[poff[2] + 0] = 1
    tab[poff[1] + 0] = 2
    tab[poff[0] + 0] = 3
    r = orc.risk(sc, tab, weights=w)
    np.testing.assert_allclose(r["attr_step"], [0, 0.5, 0.2, 0.06, 0], atol=1e-15)
    np.testing.assert_allclose(r["attr_obj"], [0, 0.06, 0.2, 0.5], atol=1e-15)
    assert abs(r["p_cra_cond"] - 0.76) < 1e-15
    assert abs(r["p_cra"] - 1.1) < 1e-15


def test_escape_routes(orc):
    """Collision-free EGO trajectories, most probable first, ties by index (Section VI-A)."""
    sc = tiny_structure([8, 3, 3], n_steps=4)
    poff = orc.pair_offsets(sc)
    tab = np.full(int(poff[-1]), -1, np.int16)
    for i in (1, 4, 6):
        tab[poff[0] + i * 3 + 2] = 0
    w = [np.array([1, 5, 2, 2, 9, 3, 1, 4.0]), np.ones(3), np.ones(3)]
    r = orc.risk(sc, tab, weights=w)
    assert list(r["escape"]) == [7, 5, 2, 3, 0]
    assert list(r["hits"]) == [0, 1, 0, 0, 1, 0, 1, 0]


def test_weights_rejected_when_invalid(orc):
    sc = tiny_structure([3, 2])
    with pytest.raises(ValueError):
        orc.normalise(sc, [np.array([1.0, -1.0, 1.0]), np.ones(2)])
    with pytest.raises(ValueError):
        orc.normalise(sc, [np.zeros(3), np.ones(2)])


def test_end_to_end_on_tiny_crossing(orc):
    """The whole method on the tiny crossing: fast hypotheses collide late, escape routes exist."""
    sc = S.tiny_crossing(1)
    out = orc.run(sc)
    tab = out["table"]
    assert 0 < (tab >= 0).sum() < tab.size
    assert tab[tab >= 0].min() >= 10
    r = out["risk"]
    assert 0 < r["p_cra_cond"] <= r["p_cra"] < 1
    assert len(r["escape"]) > 0
