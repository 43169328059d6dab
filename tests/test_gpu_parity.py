"""GPU parity: every kernel of the hot path, called through the C ABI, against the FP64 oracle on the
same seeded inputs (element by element), plus full-size checks of the 11-object intersection and a
sampled check of the 32-vehicle stress scenario."""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S
from parity_util import POSE_TOL, check_risk, check_table, corner_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mhc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06773_gb300 import mhc as m
    return m


@pytest.fixture(scope="module")
def ctx(mhc):
    c = mhc.Context(0, 1 << 30)
    yield c
    c.close()


def _ragged():
    """Hypothesis counts that straddle tile edges (1, 33, 65, 127) and all four shape combinations."""
    objs = [
        S.Obj(S.VEHICLE, 4.5, 1.8, 0, -20.0, -1.75, 0.0, 11.0, S.accel_grid_paper(5, -8, 3), S.linspace(-0.3, 0.3, 13),
              S.DEFAULT_VEH_PARAMS),                                           # 65
        S.Obj(S.PEDESTRIAN, 0, 0, 0.4, 6.0, -6.0, math.pi / 2, 0.0, S.linspace(0, 3, 3), S.linspace(-1, 1, 11)),  # 33
        S.Obj(S.VEHICLE, 3.13, 1.46, 0, 1.75, -25.0, math.pi / 2, 9.0, np.array([0.0]), np.array([0.0]),
              S.DEFAULT_VEH_PARAMS),                                           # 1
        S.Obj(S.VEHICLE, 5.0, 2.0, 0, 25.0, 1.75, math.pi, 12.0, S.accel_grid_paper(127, -8, 3), np.array([0.02]),
              S.DEFAULT_VEH_PARAMS),                                           # 127
        S.Obj(S.PEDESTRIAN, 0, 0, 0.5, -6.0, 6.0, -math.pi / 2, 0.0, S.linspace(0.5, 2.5, 4), S.linspace(-0.5, 0.5, 8)),  # 32
    ]
    return S.Scenario(objs, tau=0.1, n_steps=37, substeps=5, ego=3, name="ragged")


def _ped_accel():
    sc = S.intersection11(9, n_steps=25, n_acc=6, n_str=6, n_ped_v=5, n_ped_h=7)
    for o in sc.objects:
        if o.kind == S.PEDESTRIAN:
            o.flags = S.PED_ACCEL_GRID
            o.v0 = float(np.float32(1.2))
            o.v_max = float(np.float32(2.7))
            o.grid_a = S.linspace(-12, 12, 5)
    sc.name = "ped_accel"
    return sc


# convex outlines (body frame, metres): a pointed nose, a hexagon, an ellipse as a 16-gon, a triangle and a
# body whose pose point sits at its rear end
OUTLINES = [
    [[2.25, 0.0], [1.5, 0.9], [-2.25, 0.9], [-2.25, -0.9], [1.5, -0.9]],
    [[2.25, 0.0], [1.2, 0.9], [-1.2, 0.9], [-2.25, 0.0], [-1.2, -0.9], [1.2, -0.9]],
    [[2.25 * math.cos(2 * math.pi * q / 16), 0.9 * math.sin(2 * math.pi * q / 16)] for q in range(16)],
    [[2.5, 0.0], [-2.0, 1.0], [-2.0, -1.0]],
    [[3.6, -0.9], [3.6, 0.9], [-0.9, 0.9], [-0.9, -0.9]],
]


def _outline_shapes():
    """Vehicles drawn with the assorted outlines above, one in six left a rectangle; pedestrians as discs:
    every pairing of rectangle, outline and disc."""
    sc = S.intersection11(14, n_steps=30, n_acc=5, n_str=7, n_ped_v=3, n_ped_h=5)
    k = 0
    for o in sc.objects:
        if o.kind == S.VEHICLE:
            if k % 6 < 5:
                o.outline = np.asarray(OUTLINES[k % 6], np.float32)
            k += 1
    sc.name = "outline_shapes"
    return sc


def _scenes():
    out = {
        "outline_shapes": _outline_shapes(),
        "outline_ragged": S.with_outlines(_ragged(), cut=0.4),
        "outline_half": S.with_outlines(S.intersection11(5, n_steps=40, n_acc=9, n_str=7, n_ped_v=5, n_ped_h=9),
                                        cut=0.35, every=2),
        "lane_paths": S.with_lane_paths(S.intersection11(17, n_steps=30, n_acc=5, n_str=7, n_ped_v=3, n_ped_h=3)),
        "lane_paths_long": S.with_lane_paths(S.intersection11(18, n_steps=60, n_acc=4, n_str=3, n_ped_v=2, n_ped_h=3),
                                             every=2),
        "outline_paper_peds": S.paper_pedestrians(
            S.with_outlines(S.intersection11(16, n_steps=50, n_acc=7, n_str=7), cut=0.3), n_acc=9, n_head=12),
        "tiny": S.tiny_crossing(1),
        "tiny_near": S.tiny_crossing(1, 15.0),
        "mixed_small": S.intersection11(5, n_steps=40, n_acc=9, n_str=7, n_ped_v=5, n_ped_h=9),
        "ragged": _ragged(),
        "ped_accel": _ped_accel(),
        "paper_s1": S.paper_s1s2(3, 6),
    }
    sc = S.intersection11(6, n_steps=70, n_acc=5, n_str=9, n_ped_v=4, n_ped_h=6)
    sc.pair_mode, sc.ego, sc.name = S.EGO_ONLY, 2, "ego_only_ego2_n70"
    out[sc.name] = sc
    sc = S.intersection11(7, n_steps=30, n_acc=6, n_str=8, n_ped_v=3, n_ped_h=3)
    sc.model, sc.name = S.MODEL_KIN, "kinematic"
    out[sc.name] = sc
    sc = S.intersection11(8, n_steps=1, n_acc=4, n_str=4, n_ped_v=3, n_ped_h=3)
    sc.name = "one_step"
    out[sc.name] = sc
    # long horizons: more than 160 steps (the fused per-CTA survival cells give way to global atomics) and
    # more than 1024 (so do the per-CTA step histograms); many 32-step activity words in every layout
    sc = S.intersection11(12, n_steps=1200, n_acc=3, n_str=3, n_ped_v=2, n_ped_h=3)
    sc.tau, sc.substeps, sc.name = S.F32(0.01), 1, "long_n1200"
    out[sc.name] = sc
    sc = S.intersection11(13, n_steps=300, n_acc=4, n_str=5, n_ped_v=3, n_ped_h=3)
    sc.pair_mode, sc.ego, sc.tau, sc.substeps, sc.name = S.EGO_ONLY, 1, S.F32(0.02), 2, "ego_only_n300"
    out[sc.name] = sc
    return out


_CACHE = {}
SCENE_NAMES = ["tiny", "tiny_near", "mixed_small", "ragged", "ped_accel", "paper_s1", "ego_only_ego2_n70",
               "kinematic", "one_step", "long_n1200", "ego_only_n300", "outline_shapes", "outline_ragged",
               "outline_half", "outline_paper_peds", "lane_paths", "lane_paths_long"]


def scene(name):
    if not _CACHE:
        _CACHE.update(_scenes())
    return _CACHE[name]


@pytest.mark.parametrize("name", SCENE_NAMES)
@pytest.mark.parametrize("layout", [0, 1])
def test_generation_matches_oracle(mhc, ctx, orc, name, layout):
    """Both generation layouts: a thread per hypothesis (sub-steps in order) and a warp per hypothesis
    (sub-steps in parallel: scans of the state maps and of the heading / position increments)."""
    sc = scene(name)
    ref = orc.generate(sc)
    ctx.set_option(mhc.MHC_OPT_GEN_SCAN, layout)
    try:
        p = mhc.generate(ctx, sc)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(mhc.MHC_OPT_GEN_SCAN, 2)
    g = {k: mhc.poses_by_trajectory(sc, p[k]).astype(np.float64) for k in ("x", "y", "c", "s")}
    err = corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"])
    assert err < POSE_TOL, err


def _oracle_poses_f32(orc, sc):
    """Oracle poses rounded to FP32 (the GPU's storage format), as FP64 arrays for the oracle."""
    ref = orc.generate(sc)
    return {k: ref[k].astype(np.float32).astype(np.float64) for k in ("x", "y", "c", "s")}


@pytest.mark.parametrize("name", SCENE_NAMES)
def test_collision_kernel_on_oracle_poses(mhc, ctx, orc, name):
    """The collision kernel alone: same FP32 poses on both sides; culled and unculled tables identical."""
    sc = scene(name)
    p32 = _oracle_poses_f32(orc, sc)
    dev = {k: mhc.poses_to_device(sc, p32[k]) for k in p32}
    tab_o, poff, pairs = orc.table(sc, p32)
    ctx.set_option(mhc.MHC_OPT_CULL, 1)
    t1 = mhc.detect(ctx, sc, dev).cpu().numpy()
    ctx.set_option(mhc.MHC_OPT_CULL, 0)
    t0 = mhc.detect(ctx, sc, dev).cpu().numpy()
    ctx.set_option(mhc.MHC_OPT_CULL, 1)
    assert np.array_equal(t0, t1)
    check_table(orc, sc, t1, tab_o, p32, pairs, poff)


@pytest.mark.parametrize("name", SCENE_NAMES)
def test_pipeline_matches_oracle(mhc, ctx, orc, name):
    """Generation + collision on the GPU against generation + table in the oracle."""
    sc = scene(name)
    ref = orc.generate(sc)
    tab_o, poff, pairs = orc.table(sc, ref)
    p = mhc.generate(ctx, sc)
    t = mhc.detect(ctx, sc, p).cpu().numpy()
    check_table(orc, sc, t, tab_o, ref, pairs, poff)


@pytest.mark.parametrize("name", SCENE_NAMES)
@pytest.mark.parametrize("weighted", [False, True])
def test_risk_kernels_on_oracle_table(mhc, ctx, orc, name, weighted):
    sc = scene(name)
    ref = orc.generate(sc)
    tab_o, poff, pairs = orc.table(sc, ref)
    w = S.random_weights(sc, 77) if weighted else None
    r_o = orc.risk(sc, tab_o, pairs, w)
    dev_tab = torch.from_numpy(tab_o).cuda()
    r_g = mhc.assess(ctx, sc, dev_tab, weights=w)
    torch.cuda.synchronize()
    check_risk(r_g, r_o, mhc.layout(sc)["h_ego"])


def test_run_equals_separate_calls(mhc, ctx, orc):
    sc = scene("mixed_small")
    w = S.random_weights(sc, 5)
    p = mhc.generate(ctx, sc)
    t = mhc.detect(ctx, sc, p)
    r1 = mhc.assess(ctx, sc, t, weights=w)
    torch.cuda.synchronize()
    r2 = mhc.run(ctx, sc, weights=w)
    for k in r1:
        a, b = r1[k].cpu().numpy(), r2[k].numpy()
        if a.dtype.kind == "f":   # FP64 sums built with atomics: order-dependent in the last bits
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-18, err_msg=k)
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)


@pytest.mark.parametrize("name", ["mixed_small", "ragged", "ego_only_ego2_n70", "paper_s1", "ped_accel",
                                  "outline_shapes"])
def test_fused_evaluate_equals_separate_calls(mhc, ctx, name):
    """mhc_evaluate accumulates the risk terms inside the collision kernel; the result must equal generate +
    detect + assess: tables and every fixed-point sum bit for bit, the FP64 scalar totals to 1e-12."""
    sc = scene(name)
    w = S.random_weights(sc, 11)
    p = mhc.generate(ctx, sc)
    t = mhc.detect(ctx, sc, p)
    r1 = mhc.assess(ctx, sc, t, weights=w)
    p2, t2, r2 = mhc.evaluate(ctx, sc, weights=w)
    torch.cuda.synchronize()
    for k in p:
        assert torch.equal(p[k], p2[k])
    assert torch.equal(t, t2)
    for k in r1:
        a, b = r1[k].cpu().numpy(), r2[k].cpu().numpy()
        if k == "scalars":
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-18)
        else:
            np.testing.assert_array_equal(a, b, err_msg=k)


@pytest.mark.parametrize("name", ["mixed_small", "ragged", "ego_only_ego2_n70", "paper_s1", "kinematic", "long_n1200",
                                  "ego_only_n300", "outline_shapes", "outline_ragged"])
def test_collision_variants_agree(mhc, ctx, name):
    """Every thread layout of the collision kernel (and culling on / off) gives the same table and, fused,
    the same risk outputs."""
    sc = scene(name)
    p = mhc.generate(ctx, sc)
    ref_t, ref_r = None, None
    try:
        for variant in (1, 2, 3, 4, 5, 6, 7, 8):
            for cull in (1, 0):
                ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, variant)
                ctx.set_option(mhc.MHC_OPT_CULL, cull)
                t = mhc.detect(ctx, sc, p).cpu().numpy()
                _, _, r = mhc.evaluate(ctx, sc, poses=p)
                r = {k: v.cpu().numpy() for k, v in r.items()}
                if ref_t is None:
                    ref_t, ref_r = t, r
                    continue
                assert np.array_equal(t, ref_t), (variant, cull)
                for k in r:
                    if k == "scalars":
                        np.testing.assert_allclose(r[k], ref_r[k], rtol=1e-12, atol=1e-18)
                    else:
                        np.testing.assert_array_equal(r[k], ref_r[k], err_msg=f"{k} variant {variant} cull {cull}")
    finally:
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, 0)
        ctx.set_option(mhc.MHC_OPT_CULL, 1)


def test_autotune_picks_a_layout_and_keeps_results(mhc):
    sc = scene("mixed_small")
    c = mhc.Context(0, 256 << 20)
    try:
        p = mhc.generate(c, sc)
        before = mhc.detect(c, sc, p).clone()
        v, cull = mhc.autotune(c, sc, p)
        assert v in (1, 2, 3, 4, 5, 6, 7, 8) and cull in (0, 1)
        after = mhc.detect(c, sc, p)
        torch.cuda.synchronize()
        assert torch.equal(before, after)
    finally:
        c.close()


@pytest.mark.parametrize("name", ["mixed_small", "paper_s1", "outline_shapes"])
def test_profiled_and_overlapped_launches_agree(mhc, ctx, name):
    """Without profiling, consecutive kernels are launched as programmatic dependents (each waits for its
    predecessor inside the kernel); with profiling, event records separate them.  Both orders must give
    the same poses, table and risk outputs (FP64 scalar totals to 1e-12), in every collision layout."""
    sc = scene(name)
    w = S.random_weights(sc, 17)
    try:
        for variant in (0, 4, 5, 6, 7, 8):
            ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, variant)
            ctx.profile(False)
            p1, t1, r1 = mhc.evaluate(ctx, sc, weights=w)
            ctx.profile(True)
            p2, t2, r2 = mhc.evaluate(ctx, sc, weights=w)
            ctx.profile(False)
            ctx.profile_read(reset=True)
            torch.cuda.synchronize()
            for k in p1:
                assert torch.equal(p1[k], p2[k]), (variant, k)
            assert torch.equal(t1, t2), variant
            for k in r1:
                a, b = r1[k].cpu().numpy(), r2[k].cpu().numpy()
                if k == "scalars":
                    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-18)
                else:
                    np.testing.assert_array_equal(a, b, err_msg=f"{k} variant {variant}")
    finally:
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, 0)
        ctx.profile(False)


def test_paths_from_lane_dividers(mhc, ctx, orc):
    """The street-data step feeding the controller: each car's paths from three curved lane dividers
    (mhc_lane_paths on the host, the EGO with every combination), then generation and the whole pipeline
    on the GPU against the oracle on the same paths."""
    import dataclasses
    base = S.intersection11(19, n_steps=30, n_acc=3, n_str=1, n_ped_v=3, n_ped_h=3)
    objs = []
    for q, o in enumerate(base.objects):
        if o.kind == S.VEHICLE:
            xs = np.array([0.0, 25.0, 50.0])
            curv = 0.002 * (1 if q % 2 else -1)
            div = np.array([[[x, curv * x * x + y] for x in xs] for y in (-5.25, -1.75, 1.75, 5.25)], np.float32)
            paths = mhc.lane_paths(div, o.x0, o.y0, o.psi0, o.v0, ego=(q == base.ego))
            o = dataclasses.replace(o, grid_b=np.zeros(len(paths), np.float32), paths=paths)
        objs.append(o)
    sc = dataclasses.replace(base, objects=objs, name="lane_dividers")
    assert sc.objects[base.ego].n_hyp == 3 * 343
    ref = orc.generate(sc)
    p = mhc.generate(ctx, sc)
    g = {k: mhc.poses_by_trajectory(sc, p[k]).astype(np.float64) for k in ("x", "y", "c", "s")}
    assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL
    tab_o, poff, pairs = orc.table(sc, ref)
    t = mhc.detect(ctx, sc, p).cpu().numpy()
    check_table(orc, sc, t, tab_o, ref, pairs, poff)


@pytest.mark.parametrize("name", ["mixed_small", "lane_paths", "ped_accel"])
def test_scored_probabilities_match_oracle(mhc, ctx, orc, name):
    """MHC_OPT_SCORE: with no caller weights the risk preparation scores every hypothesis by Eq. normTraj
    (constant steering, paths, pedestrian speed and acceleration grids); the risk outputs match the
    oracle's from its own scores, and caller weights still take precedence."""
    sc = scene(name)
    ref = orc.generate(sc)
    tab_o, poff, pairs = orc.table(sc, ref)
    dev_tab = torch.from_numpy(tab_o).cuda()
    try:
        ctx.set_option(mhc.MHC_OPT_SCORE, 1)
        r_g = mhc.assess(ctx, sc, dev_tab)
        w = S.random_weights(sc, 5)
        r_w = mhc.assess(ctx, sc, dev_tab, weights=w)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(mhc.MHC_OPT_SCORE, 0)
    check_risk(r_g, orc.risk(sc, tab_o, pairs, orc.scores(sc)), mhc.layout(sc)["h_ego"])
    check_risk(r_w, orc.risk(sc, tab_o, pairs, w), mhc.layout(sc)["h_ego"])


def test_deterministic_and_stream_independent(mhc, ctx):
    sc = scene("mixed_small")
    s2 = torch.cuda.Stream()
    p = mhc.generate(ctx, sc)
    t1 = mhc.detect(ctx, sc, p).clone()
    with torch.cuda.stream(s2):
        p2 = mhc.generate(ctx, sc, stream=s2)
        t2 = mhc.detect(ctx, sc, p2, stream=s2)
    s2.synchronize()
    torch.cuda.synchronize()
    for k in p:
        assert torch.equal(p[k], p2[k])
    assert torch.equal(t1, t2)


def test_full_intersection11(mhc, ctx, orc):
    """The 11-object intersection at full size (the benchmarked workload): the whole table and the risk
    measures against the oracle."""
    sc = S.intersection11(2)
    ref = orc.generate(sc)
    p = mhc.generate(ctx, sc)
    torch.cuda.synchronize()
    g = {k: mhc.poses_by_trajectory(sc, p[k]).astype(np.float64) for k in ("x", "y", "c", "s")}
    assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL
    tab_o, poff, pairs = orc.table(sc, ref)
    t = mhc.detect(ctx, sc, p)
    t_host = t.cpu().numpy()
    check_table(orc, sc, t_host, tab_o, ref, pairs, poff, n_tests=sc.n_tests())
    r_g = mhc.assess(ctx, sc, torch.from_numpy(tab_o).cuda())
    torch.cuda.synchronize()
    check_risk(r_g, orc.risk(sc, tab_o, pairs), mhc.layout(sc)["h_ego"])
    # and the GPU's own table through the GPU risk kernels equals the oracle risk when the tables agree
    if np.array_equal(t_host, tab_o):
        r_self = mhc.assess(ctx, sc, t)
        torch.cuda.synchronize()
        check_risk(r_self, orc.risk(sc, tab_o, pairs), mhc.layout(sc)["h_ego"])


def test_stress32_sampled(mhc, orc):
    """32 vehicles x 2048 hypotheses x 50 steps (1.04e11 pose tests, 4.2 GB table): sampled rows of every
    object pair against the oracle."""
    sc = S.stress32(4)
    lay = mhc.layout(sc)
    c = mhc.Context(0, 256 << 20)
    try:
        p = mhc.generate(c, sc)
        table = torch.empty(lay["n_entries"], dtype=torch.int16, device="cuda")
        mhc.detect(c, sc, p, table)
        torch.cuda.synchronize()
        ref = orc.generate(sc)
        g = {k: mhc.poses_by_trajectory(sc, p[k]).astype(np.float64) for k in ("x", "y", "c", "s")}
        assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL
        pairs = orc.pair_list(sc)
        poff = orc.pair_offsets(sc)
        off = orc.traj_offsets(sc)
        rng = S.SplitMix64(99)
        idx, oa, ta, ob, tb = [], [], [], [], []
        for q, (a, b) in enumerate(pairs):
            for _ in range(3):          # 3 sampled rows per object pair, every column
                i = rng.randint(0, 2047)
                cols = np.arange(2048)
                idx.append(poff[q] + i * 2048 + cols)
                oa.append(np.full(2048, a)); ob.append(np.full(2048, b))
                ta.append(np.full(2048, off[a] + i)); tb.append(off[b] + cols)
        idx = np.concatenate(idx)
        tg = table[torch.from_numpy(idx).cuda()].cpu().numpy()
        to = orc.first_steps(sc, ref, np.concatenate(oa), np.concatenate(ta), np.concatenate(ob), np.concatenate(tb))
        check_table(orc, sc, tg, to, ref, pairs, poff, idx=idx)
        assert (to >= 0).sum() > 0
        del table
    finally:
        c.close()
        torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", [4, 5, 6, 7, 8])
def test_counters_and_culling_work(mhc, ctx, variant):
    """Culling leaves fewer executed tests than nominal ones, and the narrow-phase tests by shape class add
    up to their total (rectangle-rectangle, rectangle-disc and disc-disc pairs all occur in the scene)."""
    sc = S.intersection11(2)
    p = mhc.generate(ctx, sc)
    ctx.counters(reset=True)
    try:
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, variant)
        mhc.detect(ctx, sc, p)
    finally:
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, 0)
    w = ctx.work(reset=True)
    nominal = sc.n_tests()
    assert 0 < w["narrow"] < w["executed"] < nominal
    assert w["rect_rect"] + w["rect_disc"] + w["disc_disc"] + w["outline_outline"] + w["outline_disc"] == w["narrow"]
    assert w["rect_rect"] > 0 and w["rect_disc"] > 0 and w["outline_outline"] == 0 and w["outline_disc"] == 0


def test_errors_leave_context_usable(mhc, ctx):
    sc = scene("tiny")
    bad = S.tiny_crossing(1)
    bad.n_steps = 0
    with pytest.raises(mhc.MhcError):
        mhc.generate(ctx, bad, poses=mhc.alloc_poses(sc))
    with pytest.raises(mhc.MhcError):
        mhc.assess(ctx, sc, torch.zeros(256, dtype=torch.int16, device="cuda"),
                   weights=[np.zeros(16), np.ones(16)])
    p = mhc.generate(ctx, sc)
    assert torch.isfinite(p["x"]).all()


def _risk_np(r):
    return {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)) for k, v in r.items()}


def _check_risk_against_tables(orc, sc, r_gpu, tab_gpu, tab_o, pairs, n_excused):
    """Risk outputs of the GPU's own table: equal to the oracle's risk from that table (integers exactly,
    probabilities to 1e-6), and within the excused pairs of the oracle's risk from its own table."""
    he = int(np.diff(orc.traj_offsets(sc))[sc.ego])
    check_risk({k: torch.as_tensor(v) for k, v in r_gpu.items()}, orc.risk(sc, tab_gpu, pairs), he)
    ref = orc.risk(sc, tab_o, pairs)
    assert int(np.abs(r_gpu["count"] - ref["count"]).sum()) <= n_excused
    if n_excused == 0:
        check_risk({k: torch.as_tensor(v) for k, v in r_gpu.items()}, ref, he)


def test_benchmarked_calls_full_size(mhc, orc):
    """The benchmark's own step at full size: mhc_evaluate (generation, fused collision + risk in the
    layout the autotuner picks, EGO walk) on device buffers, and mhc_run with host inputs and outputs, on
    the 11-object intersection (1.70e8 pose tests).  The whole table against the oracle's (borderline
    pairs excused and counted), every risk output against the oracle's; the number of pose tests inside
    the +-1 mm band is counted beside it."""
    from oracle import parity
    sc = S.intersection11(2)
    cs = mhc.as_c(sc)
    lay = mhc.layout(cs)
    ref = orc.generate(sc)
    tab_o, poff, pairs = orc.table(sc, ref)
    ctx = mhc.Context(0, 512 << 20)
    try:
        poses = mhc.alloc_poses(sc)
        table = torch.empty(lay["n_entries"], dtype=torch.int16, device="cuda")
        risk = mhc.alloc_risk(cs)
        mhc.generate(ctx, cs, poses)
        tuned = mhc.autotune(ctx, cs, poses, table)
        results = {}
        for variant in sorted({tuned[0], 6, 7, 8}):
            ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, variant)
            table.fill_(1234)
            mhc.evaluate(ctx, cs, poses, table, out=risk)
            torch.cuda.synchronize()
            results[variant] = (table.cpu().numpy(), _risk_np(risk))
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, 0)
        g = {k: mhc.poses_by_trajectory(sc, poses[k]).astype(np.float64) for k in ("x", "y", "c", "s")}
        assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL
        for variant, (t_host, r_host) in results.items():
            n_dis, n_exc = check_table(orc, sc, t_host, tab_o, ref, pairs, poff, n_tests=sc.n_tests())
            _check_risk_against_tables(orc, sc, r_host, t_host, tab_o, pairs, n_exc)
            print(f"variant {variant}: {n_dis} entries differ from the oracle, {n_exc} excused")
        # mhc_run: host scenario in, host risk out (its own context, as the end-to-end benchmark runs it)
        run_ctx = mhc.Context(0, max(lay["run_bytes"] + (64 << 20), 256 << 20))
        try:
            host = mhc.alloc_risk(cs, device="cpu", pin=True)
            mhc.run(run_ctx, cs, out=host)
            r_run = _risk_np(host)
        finally:
            run_ctx.close()
        t_tuned = results[tuned[0]][0]
        _check_risk_against_tables(orc, sc, r_run, t_tuned, tab_o, pairs,
                                   check_table(orc, sc, t_tuned, tab_o, ref, pairs, poff, n_tests=sc.n_tests())[1])
        for k in ("count", "count_k", "hits", "escape", "n_escape"):
            np.testing.assert_array_equal(r_run[k], results[tuned[0]][1][k], err_msg=k)
        band = parity.band_count(sc, ref)
        print(f"pose tests within +-1 mm of contact (oracle margins): {band} of {sc.n_tests()}")
        assert band < 1e-4 * sc.n_tests()
    finally:
        ctx.close()
