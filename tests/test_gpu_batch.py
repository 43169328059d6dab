"""GPU batches and plans: many uneven scenarios in one launch sequence (mhc_evaluate_batch) and as a
replayed CUDA graph (mhc_plan_*).  Per scenario the batch must give exactly what the scenario gives alone
(poses, tables and every integer / fixed-point output bit for bit, the FP64 scalar totals to 1e-12), and
that must match the oracle."""
import copy

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


def mixed_batch():
    """Uneven small scenarios: different horizons (1 to 100 steps), sub-steps, pairings, EGO positions, motion
    models and ragged hypothesis counts, so that every per-scenario base in the descriptors is exercised."""
    from test_gpu_parity import scene
    out = [S.tiny_crossing(1)]
    out += S.batch_scenarios(seed=31, count=5, n_lo=2, n_hi=6, h_lo=8, h_hi=80)
    out += [copy.deepcopy(scene(n)) for n in ("ragged", "one_step", "ego_only_ego2_n70", "kinematic", "paper_s1")]
    out += [S.tiny_crossing(2, start=15.0)]
    return out


def _weights(batch, seed):
    w = []
    for q, sc in enumerate(batch):
        w += S.random_weights(sc, seed + q)
    return w


def _compare_single(mhc, ctx, batch, poses, table, out, sls, weights=None, idx=None):
    """Each scenario alone through mhc_evaluate against its part of the batch outputs."""
    wo = 0
    for q, (sc, sl) in enumerate(zip(batch, sls)):
        n_obj = len(sc.objects)
        w = None if weights is None else weights[wo: wo + n_obj]
        wo += n_obj
        if idx is not None and q not in idx:
            continue
        p1, t1, r1 = mhc.evaluate(ctx, sc, weights=w)
        torch.cuda.synchronize()
        n_pose = p1["x"].numel()
        for k in p1:
            assert torch.equal(p1[k], poses[k][sl["pose0"]: sl["pose0"] + n_pose]), (q, k)
        assert torch.equal(t1, table[sl["entry0"]: sl["entry0"] + t1.numel()]), q
        view = mhc.scenario_view(out, sl)
        for k in r1:
            a, b = r1[k].cpu().numpy(), view[k].cpu().numpy()
            if k == "scalars":
                np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-18, err_msg=f"scenario {q}")
            else:
                np.testing.assert_array_equal(b, a, err_msg=f"{k} scenario {q}")


@pytest.mark.parametrize("weighted", [False, True])
def test_batch_equals_each_scenario_alone(mhc, ctx, weighted):
    batch = mixed_batch()
    w = _weights(batch, 40) if weighted else None
    info, sls = mhc.batch_slices(batch)
    assert info["n_scenarios"] == len(batch) and info["max_steps"] == 100
    poses, table, out = mhc.evaluate_batch(ctx, batch, weights=w)
    torch.cuda.synchronize()
    _compare_single(mhc, ctx, batch, poses, table, out, sls, weights=w)


def test_batch_matches_oracle(mhc, ctx, orc):
    """Every scenario of the batch against the oracle: poses, first-collision tables, and the risk measures
    the oracle computes from the GPU's table."""
    batch = mixed_batch()
    w = _weights(batch, 90)
    info, sls = mhc.batch_slices(batch)
    poses, table, out = mhc.evaluate_batch(ctx, batch, weights=w)
    torch.cuda.synchronize()
    wo = 0
    for q, (sc, sl) in enumerate(zip(batch, sls)):
        ws = w[wo: wo + len(sc.objects)]
        wo += len(sc.objects)
        ref = orc.generate(sc)
        n_pose = int(sum(o.n_hyp for o in sc.objects)) * sc.n_steps
        g = {k: mhc.poses_by_trajectory(sc, poses[k][sl["pose0"]: sl["pose0"] + n_pose]).astype(np.float64)
             for k in ("x", "y", "c", "s")}
        assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL, q
        tab_o, poff, pairs = orc.table(sc, ref)
        t_g = table[sl["entry0"]: sl["entry0"] + tab_o.size].cpu().numpy()
        check_table(orc, sc, t_g, tab_o, ref, pairs, poff)
        check_risk(mhc.scenario_view(out, sl), orc.risk(sc, t_g, pairs, ws), sl["h_ego"])


def test_batch_with_outlines(mhc, ctx, orc):
    """Scenarios with convex outlines batched with plain ones: the batch runs the outline kernels, and each
    scenario still gets exactly what it gets alone (the plain ones alone run the kernels without outline
    tests); the outline scenarios' tables match the oracle."""
    from test_gpu_parity import scene
    batch = [S.tiny_crossing(1), copy.deepcopy(scene("outline_shapes")), copy.deepcopy(scene("ragged")),
             copy.deepcopy(scene("outline_ragged"))]
    w = _weights(batch, 60)
    info, sls = mhc.batch_slices(batch)
    poses, table, out = mhc.evaluate_batch(ctx, batch, weights=w)
    torch.cuda.synchronize()
    _compare_single(mhc, ctx, batch, poses, table, out, sls, weights=w)
    for q in (1, 3):
        sc, sl = batch[q], sls[q]
        ref = orc.generate(sc)
        tab_o, poff, pairs = orc.table(sc, ref)
        t_g = table[sl["entry0"]: sl["entry0"] + tab_o.size].cpu().numpy()
        check_table(orc, sc, t_g, tab_o, ref, pairs, poff)


def test_batch_with_lane_paths(mhc, ctx, orc):
    """Path hypotheses (the controller in the generation loop) batched with constant-steering scenarios
    small enough for the warp-per-hypothesis layout: each scenario gets exactly what it gets alone, and
    the path scenario's poses match the oracle."""
    from test_gpu_parity import scene
    batch = [S.tiny_crossing(1), copy.deepcopy(scene("lane_paths")), copy.deepcopy(scene("ragged"))]
    w = _weights(batch, 70)
    info, sls = mhc.batch_slices(batch)
    poses, table, out = mhc.evaluate_batch(ctx, batch, weights=w)
    torch.cuda.synchronize()
    _compare_single(mhc, ctx, batch, poses, table, out, sls, weights=w)
    sc, sl = batch[1], sls[1]
    ref = orc.generate(sc)
    n_pose = int(sum(o.n_hyp for o in sc.objects)) * sc.n_steps
    g = {k: mhc.poses_by_trajectory(sc, poses[k][sl["pose0"]: sl["pose0"] + n_pose]).astype(np.float64)
         for k in ("x", "y", "c", "s")}
    assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL


def test_batch_pair_table_is_the_concatenation(mhc):
    batch = mixed_batch()
    pa, pb, poff = mhc.batch_pair_table(batch)
    info, sls = mhc.batch_slices(batch)
    for sc, sl in zip(batch, sls):
        a1, b1, o1 = mhc.pair_table(sc)
        p0, n = sl["pair0"], sl["n_pairs"]
        np.testing.assert_array_equal(pa[p0: p0 + n], a1 + sl["obj0"])
        np.testing.assert_array_equal(pb[p0: p0 + n], b1 + sl["obj0"])
        np.testing.assert_array_equal(poff[p0: p0 + n + 1], o1 + sl["entry0"])
    assert poff[-1] == info["n_entries"]


@pytest.mark.parametrize("graph", [True, False])
def test_plan_replays_and_updates(mhc, ctx, graph):
    """A plan (captured as a CUDA graph or not) gives the batch result on every launch, and after an update
    with new initial states the result of the updated scenarios."""
    batch = mixed_batch()
    plan = mhc.Plan(ctx, batch, graph=graph)
    try:
        pb, tb, ob = mhc.evaluate_batch(ctx, batch)
        for _ in range(3):
            poses, table, out = plan.launch()
        torch.cuda.synchronize()
        assert torch.equal(table, tb)
        for k in poses:
            assert torch.equal(poses[k], pb[k])
        for k in out:
            if k != "scalars":
                assert torch.equal(out[k], ob[k]), k
        np.testing.assert_allclose(out["scalars"].cpu().numpy(), ob["scalars"].cpu().numpy(), rtol=1e-12, atol=1e-18)
        moved = copy.deepcopy(batch)
        for sc in moved:
            for o in sc.objects:
                o.x0 += 0.75
                o.v0 = o.v0 * 1.05 + 0.1
        plan.update(moved)
        poses, table, out = plan.launch()
        pm, tm, om = mhc.evaluate_batch(ctx, moved)
        torch.cuda.synchronize()
        assert torch.equal(table, tm)
        assert not torch.equal(tm, tb)
        for k in out:
            if k != "scalars":
                assert torch.equal(out[k], om[k]), k
    finally:
        plan.close()


def test_plan_rejects_other_structure(mhc, ctx):
    batch = mixed_batch()
    plan = mhc.Plan(ctx, batch, graph=True)
    try:
        other = copy.deepcopy(batch)
        other[3].n_steps += 1
        with pytest.raises(mhc.MhcError):
            plan.update(other)
        with pytest.raises(mhc.MhcError):
            plan.update(batch[:-1])
        plan.launch()          # still usable
        torch.cuda.synchronize()
    finally:
        plan.close()


def test_batch_errors_name_the_scenario(mhc, ctx):
    batch = mixed_batch()
    bad = copy.deepcopy(batch)
    bad[4].n_steps = 0
    with pytest.raises(mhc.MhcError, match="scenario 4"):
        mhc.evaluate_batch(ctx, bad)
    with pytest.raises(ValueError):
        mhc.batch_layout([])
    cb = mhc.as_batch(batch)
    info = mhc.MhcBatchInfo()
    assert mhc.lib.mhc_batch_layout(cb.ref, 0, info, None) == -1          # MHC_E_INVALID
    assert mhc.lib.mhc_batch_layout(cb.ref, 65537, info, None) == -1
    poses, table, out = mhc.evaluate_batch(ctx, batch[:2])
    torch.cuda.synchronize()


def test_full_batch_256_graph(mhc, orc):
    """The 256-scenario uneven batch (2 to 24 objects, 64 to 1024 hypotheses, 20 to 50 steps; about 1.07e11
    pose tests, a 6.1 GB table) as a replayed graph: equal to the one-call batch; sampled scenarios equal to
    their single runs; sampled rows of sampled scenarios and the poses of sampled scenarios against the
    oracle."""
    batch = S.batch_scenarios(seed=3, count=256)
    info, sls = mhc.batch_slices(batch)
    c = mhc.Context(0, int(info["scratch"]) + (64 << 20))
    plan = None
    try:
        plan = mhc.Plan(c, batch, graph=True)
        plan.launch()
        plan.launch()
        torch.cuda.synchronize()
        pb, tb, ob = mhc.evaluate_batch(c, batch)
        torch.cuda.synchronize()
        assert torch.equal(plan.table, tb)
        for k in ob:
            if k != "scalars":
                assert torch.equal(plan.out[k], ob[k]), k
        del pb, tb, ob
        torch.cuda.empty_cache()
        rng = S.SplitMix64(123)
        picks = sorted({rng.randint(0, 255) for _ in range(6)} | {0, 255})
        _compare_single(mhc, c, batch, plan.poses, plan.table, plan.out, sls, idx=set(picks))
        for q in picks[:4]:
            sc, sl = batch[q], sls[q]
            ref = orc.generate(sc)
            n_pose = int(sum(o.n_hyp for o in sc.objects)) * sc.n_steps
            g = {k: mhc.poses_by_trajectory(sc, plan.poses[k][sl["pose0"]: sl["pose0"] + n_pose]).astype(np.float64)
                 for k in ("x", "y", "c", "s")}
            assert corner_error(sc, ref, g["x"], g["y"], g["c"], g["s"]) < POSE_TOL, q
            pairs = orc.pair_list(sc)
            poff = orc.pair_offsets(sc)
            off = orc.traj_offsets(sc)
            idx, oa, ta, ob_, tb_ = [], [], [], [], []
            for p, (a, b) in enumerate(pairs):
                ha, hb = int(off[a + 1] - off[a]), int(off[b + 1] - off[b])
                i = rng.randint(0, ha - 1)
                cols = np.arange(hb)
                idx.append(poff[p] + i * hb + cols)
                oa.append(np.full(hb, a)); ob_.append(np.full(hb, b))
                ta.append(np.full(hb, off[a] + i)); tb_.append(off[b] + cols)
            idx = np.concatenate(idx)
            tg = plan.table[torch.from_numpy(idx + sl["entry0"]).cuda()].cpu().numpy()
            to = orc.first_steps(sc, ref, np.concatenate(oa), np.concatenate(ta), np.concatenate(ob_),
                                 np.concatenate(tb_))
            check_table(orc, sc, tg, to, ref, pairs, poff, idx=idx)
    finally:
        if plan is not None:
            plan.close()
        c.close()
        torch.cuda.empty_cache()


@pytest.mark.parametrize("graph", [True, False])
def test_pipelined_plan_equals_serial_plan(mhc, ctx, graph):
    """A plan of 12 uneven scenarios asked to pipeline (four runs of scenarios on two streams) and the serial
    plan give, with caller weights, the same poses, table and risk outputs, before and after an update with
    new initial states (FP64 scalar totals to rounding)."""
    batch = mixed_batch()
    w = _weights(batch, 7)
    pipe = mhc.Plan(ctx, batch, weights=w, graph=graph, pipeline=True)
    ser = mhc.Plan(ctx, batch, weights=w, graph=graph)
    try:
        for rnd in range(2):
            if rnd == 1:
                moved = copy.deepcopy(batch)
                for sc in moved:
                    for o in sc.objects:
                        o.x0 -= 0.5
                        o.v0 = o.v0 * 0.97 + 0.2
                pipe.update(moved)
                ser.update(moved)
            p1, t1, o1 = pipe.launch()
            p2, t2, o2 = ser.launch()
            torch.cuda.synchronize()
            assert torch.equal(t1, t2)
            for k in p1:
                assert torch.equal(p1[k], p2[k]), k
            for k in o1:
                if k == "scalars":
                    np.testing.assert_allclose(o1[k].cpu().numpy(), o2[k].cpu().numpy(), rtol=1e-12, atol=1e-18)
                else:
                    assert torch.equal(o1[k], o2[k]), (rnd, k)
            assert int((t1 >= 0).sum()) > 0
    finally:
        pipe.close()
        ser.close()
