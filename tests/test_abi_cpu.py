"""The C-ABI library builds, loads and exports every entry point declared in include/mhc.h; host-side
layout and validation behave as documented.  No GPU is touched."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2005_06773_gb300 import build as B
from paper_2005_06773_gb300 import scenarios as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mhc.h")


@pytest.fixture(scope="module")
def mhc():
    B.build()
    from paper_2005_06773_gb300 import mhc as m
    return m


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mhc_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(mhc):
    names = declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(B.LIB)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(mhc):
    assert mhc.lib.mhc_status_string(-1) == b"MHC_E_INVALID"
    assert mhc.lib.mhc_status_string(0) == b"MHC_OK"
    assert b"sm_103a" in mhc.lib.mhc_version()


def test_layout_counts(mhc):
    lay = mhc.layout(S.intersection11(2))
    assert lay["n_traj"] == 3571 and lay["n_pairs"] == 55 and lay["n_entries"] == 5_666_055 and lay["h_ego"] == 441
    big = mhc.layout(S.stress32(4))
    assert big["n_entries"] == 496 * 2048 * 2048
    s2 = S.paper_s1s2(10, 6)
    lay = mhc.layout(s2)
    assert lay["n_entries"] == 864_360 and lay["n_traj"] == 2478 and lay["n_pairs"] == 10


def test_pair_table_matches_oracle(mhc, orc):
    for sc in (S.intersection11(2), S.paper_s1s2(3, 5), S.stress32(4)):
        pa, pb, poff = mhc.pair_table(sc)
        assert list(zip(pa.tolist(), pb.tolist())) == orc.pair_list(sc)
        assert np.array_equal(poff, orc.pair_offsets(sc))
    sc = S.intersection11(3)
    sc.pair_mode, sc.ego = S.EGO_ONLY, 4
    pa, pb, _ = mhc.pair_table(sc)
    assert set(pa.tolist()) == {4} and 4 not in pb.tolist() and len(pb) == 10


def _bad(mutate):
    sc = S.tiny_crossing(1)
    mutate(sc)
    return sc


BAD = {
    "zero_steps": lambda s: setattr(s, "n_steps", 0),
    "too_many_steps": lambda s: setattr(s, "n_steps", 40000),
    "zero_tau": lambda s: setattr(s, "tau", 0.0),
    "nan_tau": lambda s: setattr(s, "tau", float("nan")),
    "zero_substeps": lambda s: setattr(s, "substeps", 0),
    "bad_pair_mode": lambda s: setattr(s, "pair_mode", 5),
    "bad_model": lambda s: setattr(s, "model", 3),
    "ego_out_of_range": lambda s: setattr(s, "ego", 2),
    "bad_kind": lambda s: setattr(s.objects[0], "kind", 7),
    "empty_grid": lambda s: setattr(s.objects[0], "grid_a", np.zeros(0, np.float32)),
    "nan_grid": lambda s: s.objects[1].grid_b.__setitem__(0, np.nan),
    "zero_length": lambda s: setattr(s.objects[0], "length", 0.0),
    "negative_speed": lambda s: setattr(s.objects[0], "v0", -1.0),
    "negative_param": lambda s: setattr(s.objects[0], "params", -S.DEFAULT_VEH_PARAMS),
    "inf_position": lambda s: setattr(s.objects[1], "x0", float("inf")),
}


@pytest.mark.parametrize("case", list(BAD))
def test_invalid_scenarios_rejected(mhc, case):
    sc = _bad(BAD[case])
    with pytest.raises(mhc.MhcError) as e:
        mhc.layout(sc)
    assert e.value.code == -1


def test_invalid_pedestrian_and_pairing(mhc):
    ped = S.Obj(S.PEDESTRIAN, 0, 0, 0.4, 0, 0, 0, 0, np.array([-1.0]), np.array([0.0]))
    car = S.tiny_crossing(1).objects[0]
    with pytest.raises(mhc.MhcError):
        mhc.layout(S.Scenario([car, ped]))
    ped0 = S.Obj(S.PEDESTRIAN, 0, 0, 0.0, 0, 0, 0, 0, np.array([1.0]), np.array([0.0]))
    with pytest.raises(mhc.MhcError):
        mhc.layout(S.Scenario([car, ped0]))
    with pytest.raises(mhc.MhcError):
        mhc.layout(S.Scenario([car], pair_mode=S.EGO_ONLY))
    # a single object with all pairs is valid: no pairs, an empty table
    lay = mhc.layout(S.Scenario([car]))
    assert lay["n_pairs"] == 0 and lay["n_entries"] == 0


def _with_outline(outline, obj=0):
    sc = S.tiny_crossing(1)
    sc.objects[obj].outline = np.asarray(outline, np.float32).reshape(-1, 2)
    return sc


def _regular(n, r=1.0, turns=1):
    return [[r * math.cos(2 * math.pi * turns * q / n), r * math.sin(2 * math.pi * turns * q / n)] for q in range(n)]


BAD_OUTLINES = {
    "two_vertices": [[1, 0], [-1, 0]],
    "seventeen_vertices": _regular(17),
    "dart": [[2, 0], [-1, 1], [0, 0], [-1, -1]],                 # reflex vertex at the origin
    "pentagram": _regular(5, turns=2),                           # every turn the same way, but twice round
    "repeated_vertex": [[1, 1], [-1, 1], [-1, 1], [-1, -1], [1, -1]],
    "collinear_vertex": [[1, 1], [0, 1], [-1, 1], [-1, -1], [1, -1]],
    "no_area": [[1, 0], [0, 0], [-1, 0]],
    "nan_vertex": [[1, 1], [-1, 1], [float("nan"), -1], [1, -1]],
}


@pytest.mark.parametrize("case", list(BAD_OUTLINES))
def test_invalid_outlines_rejected(mhc, case):
    with pytest.raises(mhc.MhcError) as e:
        mhc.layout(_with_outline(BAD_OUTLINES[case]))
    assert e.value.code == -1


def test_outlines_accepted_in_either_orientation(mhc):
    plain = mhc.layout(S.tiny_crossing(1))
    ccw = S.chamfered_outline(4.5, 1.8, 0.3)
    for outline in (ccw, ccw[::-1], _regular(16, 2.0), _regular(3, 2.0)):
        lay = mhc.layout(_with_outline(outline))
        sizes = [k for k in plain if k not in ("scratch", "run_bytes")]
        assert {k: lay[k] for k in sizes} == {k: plain[k] for k in sizes}   # no output array changes size
        assert lay["scratch"] > plain["scratch"]                             # the vertices travel with the descriptors
    ped = S.Obj(S.PEDESTRIAN, 0, 0, 0.4, 0, 0, 0, 0, np.array([1.0]), np.array([0.0]),
                outline=np.array([[1, 0], [0, 1], [-1, 0]], np.float32))
    with pytest.raises(mhc.MhcError):
        mhc.layout(S.Scenario([S.tiny_crossing(1).objects[0], ped]))


def test_invalid_paths_rejected(mhc):
    sc = S.with_lane_paths(S.tiny_crossing(1))
    sc.objects[0].paths[2, 1, 0] = np.nan
    with pytest.raises(mhc.MhcError):
        mhc.layout(sc)
    car = S.tiny_crossing(1).objects[0]
    ped = S.Obj(S.PEDESTRIAN, 0, 0, 0.4, 0, 0, 0, 0, np.array([1.0]), np.zeros(2),
                paths=np.zeros((2, 3, 3), np.float32))
    with pytest.raises(mhc.MhcError):
        mhc.layout(S.Scenario([car, ped]))
    bad = S.with_lane_paths(S.tiny_crossing(1))
    bad.objects[1].paths = bad.objects[1].paths[:3]                 # fewer paths than n_b
    with pytest.raises(ValueError):
        mhc.layout(bad)
    assert mhc.layout(S.with_lane_paths(S.tiny_crossing(1)))["n_traj"] == 2 * 4 * 7


def _random_lanes(rng, n_div):
    """n_div dividers, right to left, 3.5 m apart with a common curvature, around the vehicle's lane."""
    a, b = rng.uniform(-0.004, 0.004), rng.uniform(-0.05, 0.05)
    own = rng.randint(0, n_div - 2)                        # the vehicle sits between dividers own and own + 1
    base = -rng.uniform(0.3, 3.2) - 3.5 * own
    xs = [rng.uniform(-2, 2), rng.uniform(15, 25), rng.uniform(40, 60)]
    return np.array([[[x, a * x * x + b * x + base + 3.5 * j] for x in xs] for j in range(n_div)], np.float32)


def test_lane_paths_match_the_oracle(mhc, orc):
    """Street data processing runs on the host inside the library (FP64, FP32 output): the same paths as
    the oracle's FP64 restatement on the same FP32 inputs, for 2 to 4 dividers, COs and the EGO."""
    from paper_2005_06773_gb300.scenarios import SplitMix64
    rng = SplitMix64(77)
    for trial in range(60):
        n_div = 2 + trial % 3
        div = _random_lanes(rng, n_div)
        x0, y0, psi0, v0 = (float(np.float32(v)) for v in (rng.uniform(-50, 50), rng.uniform(-50, 50),
                                                           rng.uniform(-3, 3), rng.uniform(0, 30)))
        for ego in (False, True):
            got = mhc.lane_paths(div, x0, y0, psi0, v0, ego=ego)
            ref = orc.lane_paths(div.astype(np.float64), x0, y0, psi0, v0, ego=ego)
            assert got.shape == ref.shape
            np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)


def test_lane_paths_errors(mhc):
    flat = np.array([[[0, y], [30, y], [60, y]] for y in (-1.75, 1.75)], np.float32)
    assert mhc.lane_paths(flat, 0, 0, 0, 10).shape == (3, 3, 3)
    assert mhc.lane_paths(flat, 0, 0, 0, 10, ego=True).shape == (27, 3, 3)
    for bad in (flat[:1], flat + np.array([0, 5], np.float32), np.concatenate([flat] * 3)):
        with pytest.raises(mhc.MhcError):
            mhc.lane_paths(bad, 0, 0, 0, 10)
    rep = flat.copy()
    rep[0, 1, 0] = rep[0, 0, 0]                             # repeated abscissa
    with pytest.raises(mhc.MhcError):
        mhc.lane_paths(rep, 0, 0, 0, 10)
    with pytest.raises(mhc.MhcError):
        mhc.lane_paths(flat, 0, 0, 0, -1.0)


def test_misaligned_arena_rejected_before_any_device_call(mhc):
    """A caller's arena must be 256-byte aligned (it holds float4 bounds and the descriptor copy's 16-byte
    words); a misaligned one is an MHC_E_INVALID, decided before the library touches a device."""
    h = ctypes.c_void_p()
    assert mhc.lib.mhc_create(ctypes.byref(h), 0, ctypes.c_void_p(0x10000010), 1 << 20) == -1   # MHC_E_INVALID
    assert b"256-byte aligned" in mhc.lib.mhc_last_error()
    assert not h.value


def test_misaligned_device_arrays_rejected_before_any_device_call(mhc):
    """Caller device arrays at less than their elements' alignment are an MHC_E_INVALID, decided on the
    host before any launch (the addresses below are never dereferenced)."""
    cs = mhc.as_c(S.tiny_crossing())
    fake_ctx = ctypes.c_void_p(0x1000)        # not dereferenced: the argument checks come first
    good = [0x20000000 + 0x100000 * q for q in range(4)]

    def poses(addrs):
        return mhc.MhcPoses(*addrs)

    p_bad = poses([good[0], good[1] + 2, good[2], good[3]])
    assert mhc.lib.mhc_generate_trajectories(fake_ctx, cs.ref, ctypes.byref(p_bad), None) == -1
    assert b"4-byte aligned" in mhc.lib.mhc_last_error()
    p_ok = poses(good)
    assert mhc.lib.mhc_detect_collisions(fake_ctx, cs.ref, ctypes.byref(p_ok), ctypes.c_void_p(0x30000001), None) == -1
    assert b"2-byte aligned" in mhc.lib.mhc_last_error()
    assert mhc.lib.mhc_detect_collisions_static(cs.ref, ctypes.byref(p_bad), ctypes.c_void_p(0x30000000), None) == -1
    assert b"4-byte aligned" in mhc.lib.mhc_last_error()
    risk = mhc.MhcRisk()
    risk.P = 0x40000004
    assert mhc.lib.mhc_assess_risk(fake_ctx, cs.ref, ctypes.c_void_p(0x30000000), None, ctypes.byref(risk), None) == -1
    assert b"element size" in mhc.lib.mhc_last_error()
