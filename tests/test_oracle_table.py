"""Pins of the oracle's first-collision tables (Section IV-C) against analytic collision times, the paper's
printed counts and tunnelling speeds, and structural invariants."""
import math
import os

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
f32 = lambda v: float(np.float32(v))


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            name, val, tol = line.split()
            out[name] = (float(val), float(tol))
    return out


def car(x0, y0, psi0, v0, acc=0.0, steer=0.0, L=4.5, W=1.8):
    return S.Obj(S.VEHICLE, L, W, 0.0, x0, y0, psi0, v0, np.array([acc]), np.array([steer]), S.DEFAULT_VEH_PARAMS)


def first_step(orc, objs, n, tau=0.1, k=5):
    sc = S.Scenario(objs, tau=tau, n_steps=n, substeps=k)
    p = orc.generate(sc)
    tab, _, _ = orc.table(sc, p, pairs=[(0, 1)])
    return int(tab[0]), sc, p


def times(tau, n):
    return (np.arange(n) + 1) * f32(tau)


def analytic_first(cond, t, tol=1e-9):
    """First sample time at which cond(t) holds; None if some sample sits within tol of a boundary."""
    for k, tk in enumerate(t):
        val = cond(tk)
        if abs(val) < tol:
            return None
        if val <= 0:
            return k
    return -1


def test_crossing_constant_speed(orc):
    """90 degree crossing of two 4.5 x 1.8 cars from 30 m: both box footprints are axis-aligned, so they
    overlap iff |x_A| <= 2.25 + 0.9 and |y_B| <= 0.9 + 2.25."""
    rng = S.SplitMix64(21)
    n, checked = 40, 0
    for _ in range(60):
        va, vb = f32(rng.uniform(6, 16)), f32(rng.uniform(6, 16))
        T, _, _ = first_step(orc, [car(-30, 0, 0, va), car(0, -30, math.pi / 2, vb)], n)
        cond = lambda t: max(abs(-30 + va * t) - 3.15, abs(-30 + vb * t) - 3.15)
        expect = analytic_first(cond, times(0.1, n))
        if expect is None:
            continue
        checked += 1
        assert T == expect, (va, vb, T, expect)
    assert checked > 50


def test_crossing_constant_acceleration(orc):
    rng = S.SplitMix64(22)
    n = 40
    for _ in range(40):
        va, vb = f32(rng.uniform(8, 15)), f32(rng.uniform(8, 15))
        aa, ab = f32(rng.uniform(-3, 2)), f32(rng.uniform(-3, 2))
        T, _, _ = first_step(orc, [car(-30, 0, 0, va, aa), car(0, -30, math.pi / 2, vb, ab)], n)

        def pos(v, a, t):
            if a < 0 and t > v / -a:
                return v * v / (2 * -a)
            return v * t + a * t * t / 2

        cond = lambda t: max(abs(-30 + pos(va, aa, t)) - 3.15, abs(-30 + pos(vb, ab, t)) - 3.15)
        expect = analytic_first(cond, times(0.1, n))
        if expect is not None:
            assert T == expect, (va, vb, aa, ab, T, expect)


@pytest.mark.parametrize("e", [0.0, 0.9, 1.79, 1.81, 2.5])
def test_head_on(orc, e):
    """Head-on from 60 m apart with lateral offset e: collide iff |e| <= 1.8, first when the gap closes to 4.5 m,
    t* = (60 - 4.5) / (v_A + v_B)."""
    va, vb = f32(11.0), f32(13.0)
    e32 = f32(e)
    T, _, _ = first_step(orc, [car(-30, e32, 0, va), car(30, 0, math.pi, vb)], 40)
    if abs(e32) > 1.8:
        assert T == -1
    else:
        t_star = (60 - 4.5) / (va + vb)
        assert T == int(math.ceil(t_star / f32(0.1) - 1e-9)) - 1


@pytest.mark.parametrize("xp", [0.0, 1.5, -2.0, 2.4, 2.6, 2.7, -3.0])
def test_pedestrian_crossing_in_front_of_parked_car(orc, xp):
    """A pedestrian (r = 0.4) walks north at u across a parked 4.5 x 1.8 car.  Along the side: contact when the
    centre is 0.9 + 0.4 from the axis; past the corner: contact with the corner's 0.4 m circle; beyond
    2.25 + 0.4 never."""
    u = f32(1.7)
    xp = f32(xp)
    p = S.Obj(S.PEDESTRIAN, 0, 0, 0.4, xp, -10.0, math.pi / 2, 0.0, np.array([u]), np.array([0.0]))
    T, _, _ = first_step(orc, [car(0, 0, 0, 0.0), p], 80)
    ax = abs(xp)
    if ax <= 2.25:
        y_contact = -(0.9 + 0.4)
    elif ax < 2.65:
        y_contact = -0.9 - math.sqrt(0.16 - (ax - 2.25) ** 2)
    else:
        assert T == -1
        return
    t_star = (y_contact + 10.0) / u
    assert T == int(math.ceil(t_star / f32(0.1) - 1e-9)) - 1


def _tunnel(orc, v, crosswise, phases=40):
    """Share of start phases in which a car driving at v through a parked car is never seen overlapping."""
    L, W = golden()["car_length"][0], golden()["car_width"][0]
    tau = golden()["tau"][0]
    missed = 0
    for q in range(phases):
        x0 = -40.0 - v * tau * q / phases
        objs = [car(x0, 0.0, 0.0, v, L=L, W=W), car(0.0, 0.0, math.pi / 2 if crosswise else 0.0, 0.0, L=L, W=W)]
        T, _, _ = first_step(orc, objs, 40, tau=tau, k=1)
        missed += T == -1
    return missed


def test_tunnelling_speeds_match_paper(orc):
    """Section IV-C.2: the smallest car (3.13 x 1.46 m) at 20 ms can be stepped over above ~229 m/s (T-bone)
    and ~313 m/s (longitudinal).  Below the bound every phase is detected; above it some are missed."""
    g = golden()
    L, W, tau = g["car_length"][0], g["car_width"][0], g["tau"][0]
    v_tbone, v_long = (L + W) / tau, 2 * L / tau
    assert abs(v_tbone - g["tunnel_tbone"][0]) <= g["tunnel_tbone"][1]
    assert abs(v_long - g["tunnel_long"][0]) <= g["tunnel_long"][1]
    assert _tunnel(orc, 0.98 * v_tbone, True) == 0
    assert _tunnel(orc, 1.05 * v_tbone, True) > 0
    assert _tunnel(orc, 0.98 * v_long, False) == 0
    assert _tunnel(orc, 1.05 * v_long, False) > 0


def small_scene(seed=31, n=20):
    return S.intersection11(seed, n_steps=n, n_acc=4, n_str=5, n_ped_v=3, n_ped_h=4)


def test_table_symmetry_and_range(orc):
    sc = small_scene()
    p = orc.generate(sc)
    pairs = orc.pair_list(sc)
    assert all(a != b for a, b in pairs)
    tab, poff, _ = orc.table(sc, p, pairs)
    rev = [(b, a) for a, b in pairs]
    tab_r, poff_r, _ = orc.table(sc, p, rev)
    h = np.diff(orc.traj_offsets(sc))
    assert tab.min() >= -1 and tab.max() < sc.n_steps
    for q, (a, b) in enumerate(pairs):
        t1 = tab[poff[q]:poff[q + 1]].reshape(h[a], h[b])
        t2 = tab_r[poff_r[q]:poff_r[q + 1]].reshape(h[b], h[a])
        assert np.array_equal(t1, t2.T)
    assert (tab >= 0).sum() > 0


def test_table_is_first_overlapping_step(orc):
    sc = small_scene(32)
    p = orc.generate(sc)
    tab, poff, pairs = orc.table(sc, p)
    off = orc.traj_offsets(sc)
    h = np.diff(off)
    rng = S.SplitMix64(33)
    oa, ta, ob, tb, expect = [], [], [], [], []
    for _ in range(400):
        q = rng.randint(0, len(pairs) - 1)
        a, b = pairs[q]
        i, j = rng.randint(0, h[a] - 1), rng.randint(0, h[b] - 1)
        oa.append(a); ob.append(b); ta.append(off[a] + i); tb.append(off[b] + j)
        expect.append(tab[poff[q] + i * h[b] + j])
    m = orc.margins(sc, p, oa, ta, ob, tb)
    for row, e in zip(m, expect):
        hits = np.nonzero(row <= 0)[0]
        assert (hits[0] if hits.size else -1) == e


def test_longer_horizon_keeps_earlier_steps(orc):
    s20, s30 = small_scene(34, 20), small_scene(34, 30)
    t20, _, _ = orc.table(s20, orc.generate(s20))
    t30, _, _ = orc.table(s30, orc.generate(s30))
    hit = t20 >= 0
    assert np.array_equal(t30[hit], t20[hit])
    assert np.all((t30[~hit] == -1) | (t30[~hit] >= 20))


def test_inflating_shapes_never_delays_collisions(orc):
    sc = small_scene(35)
    p = orc.generate(sc)
    t0, _, _ = orc.table(sc, p)
    for o in sc.objects:
        o.length += 0.3; o.width += 0.2; o.radius += 0.1
    t1, _, _ = orc.table(sc, p)
    hit = t0 >= 0
    assert np.all(t1[hit] >= 0) and np.all(t1[hit] <= t0[hit])
    assert (t1 >= 0).sum() > (t0 >= 0).sum()


def test_rigid_motion_of_scene_keeps_table(orc):
    sc = small_scene(36)
    p = orc.generate(sc)
    t0, poff, pairs = orc.table(sc, p)
    th, tx, ty = 0.9, 120.0, -40.0
    for o in sc.objects:
        x, y = o.x0, o.y0
        o.x0 = f32(tx + math.cos(th) * x - math.sin(th) * y)
        o.y0 = f32(ty + math.sin(th) * x + math.cos(th) * y)
        o.psi0 = f32(o.psi0 + th)
    p2 = orc.generate(sc)
    t1, _, _ = orc.table(sc, p2)
    diff = np.nonzero(t0 != t1)[0]
    # inputs were re-rounded to FP32, so only borderline pairs may move
    assert diff.size <= 1e-3 * t0.size
    off = orc.traj_offsets(sc)
    h = np.diff(off)
    for idx in diff[:50]:
        q = int(np.searchsorted(poff, idx, side="right") - 1)
        a, b = pairs[q]
        i, j = divmod(int(idx - poff[q]), int(h[b]))
        k = min(x for x in (t0[idx], t1[idx]) if x >= 0)
        m = orc.margins(sc, p, [a], [off[a] + i], [b], [off[b] + j])[0]
        assert abs(m[k]) < 1e-4


def test_paper_counts(orc):
    """Trajectory, combination and pose-combination counts of the paper's S1/S2 shape (golden values)."""
    g = golden()
    for n_co, prof, key in ((10, 6, "s2_6"), (3, 6, "s1_6"), (3, 5, "s1_5"), (10, 5, "s2_5")):
        sc = S.paper_s1s2(n_co, prof)
        h = np.diff(orc.traj_offsets(sc))
        pairs = orc.pair_list(sc)
        assert len(pairs) == n_co and all(a == 0 for a, _ in pairs)
        combos = sum(int(h[a]) * int(h[b]) for a, b in pairs)
        poses = combos * sc.n_steps
        val, tol = g[key]
        assert abs(poses - val) <= tol, (key, poses)
        if key == "s2_6":
            assert int(h.sum()) == g["r_tra"][0]
            assert int(h[0]) == g["h_ego"][0] and int(h[1]) == g["h_co"][0]
            assert combos == g["r_col"][0]
            assert 2 * poses == g["overlap_calls"][0]
            assert abs(int(h[0]) * int(h[1]) * sc.n_steps - g["pose_per_co"][0]) <= g["pose_per_co"][1]
            assert sc.n_steps * f32(sc.tau) == pytest.approx(2.0, rel=1e-6)


def test_workload_counts():
    sc = S.intersection11(2)
    assert sc.n_traj_pairs() == 5_666_055 and sc.n_tests() == 169_981_650
    big = S.stress32(4)
    assert big.n_traj_pairs() == 496 * 2048 * 2048 and big.n_tests() == 104_018_739_200
