"""The allocation-free collision entry point (mhc_detect_collisions_static), called through the C ABI.

It exists for callers that may not allocate memory while they run (real-time or safety controllers with a
memory plan fixed at start-up, plugins whose host framework owns all device memory).  Its result must equal
the ordinary entry point's table exactly (first-collision steps are integers), on consecutive calls that
reuse its one static scratch array, including a call on a different scenario in between.  This file is
collected last so that a failure here does not stop the rest of the suite first."""
import ctypes

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mhc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06773_gb300 import mhc as m
    m.lib.mhc_detect_collisions_static.argtypes = [ctypes.POINTER(m.MhcScenario), ctypes.POINTER(m.MhcPoses),
                                                   ctypes.c_void_p, ctypes.c_void_p]
    m.lib.mhc_detect_collisions_static.restype = ctypes.c_int
    return m


def _static_detect(mhc, cs, poses, table):
    ps = mhc.MhcPoses(poses["x"].data_ptr(), poses["y"].data_ptr(), poses["c"].data_ptr(), poses["s"].data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    return mhc.lib.mhc_detect_collisions_static(cs.ref, ctypes.byref(ps), table.data_ptr(), stream)


def _scenes():
    """The benchmark scene, a smaller one, EGO-only pairing with the EGO in the middle and pedestrians
    only (disc-disc pairs only)."""
    import dataclasses
    big = S.intersection11(2)
    small = S.intersection11(5, n_steps=40, n_acc=9, n_str=7, n_ped_v=5, n_ped_h=9)
    ego_only = dataclasses.replace(S.intersection11(7, n_steps=35, n_acc=7, n_str=5, n_ped_v=4, n_ped_h=5),
                                   pair_mode=S.EGO_ONLY, ego=5)
    peds = dataclasses.replace(small, objects=[o for o in small.objects if o.kind == S.PEDESTRIAN], ego=0)
    return [big, small, ego_only, peds]


def test_static_entry_matches_ordinary_entry(mhc):
    """Consecutive calls share the one static array: each result must equal mhc_detect_collisions' table
    exactly, and once the first call has loaded the module, later calls allocate no device memory."""
    ctx = mhc.Context(0, 256 << 20)
    try:
        scenes = [mhc.as_c(sc) for sc in _scenes()]
        refs, outs = [], []
        for cs in scenes:
            p = mhc.generate(ctx, cs)
            ref = mhc.detect(ctx, cs, p).clone()
            refs.append((p, ref))
            outs.append(torch.full_like(ref, 1234))
        torch.cuda.synchronize()
        assert _static_detect(mhc, scenes[1], refs[1][0], outs[1]) == 0    # first call: loads the module
        torch.cuda.synchronize()
        order = [0, 0, 1, 2, 3, 0, 2]          # two calls in a row, the others, then back
        got = [torch.full_like(refs[q][1], 1234) for q in order]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for q, out in zip(order, got):
            rc = _static_detect(mhc, scenes[q], refs[q][0], out)
            assert rc == 0, mhc.lib.mhc_last_error().decode()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 >= free0, (free0, free1)   # nothing allocated by the calls themselves
        for q, out in zip(order, got):
            assert torch.equal(out, refs[q][1]), q
        for q in range(len(scenes) - 1):
            assert int((refs[q][1] >= 0).sum()) > 0
    finally:
        ctx.close()


def test_static_entry_single_object_has_no_pairs(mhc):
    sc = S.tiny_crossing(1)
    sc.objects = sc.objects[:1]
    cs = mhc.as_c(sc)
    poses = mhc.alloc_poses(sc)
    ctx = mhc.Context(0, 64 << 20)
    try:
        mhc.generate(ctx, cs, poses)
    finally:
        ctx.close()
    table = torch.full((4,), 1234, dtype=torch.int16, device="cuda")
    rc = _static_detect(mhc, cs, poses, table)
    torch.cuda.synchronize()
    assert rc == 0, mhc.lib.mhc_last_error().decode()
    assert torch.all(table == 1234)          # no pairs: no entry written


def test_static_entry_refuses_a_capturing_stream(mhc):
    """Its descriptors sit in a host array that later calls rewrite, so it refuses stream capture; the
    capture itself and later calls are unaffected."""
    cs = mhc.as_c(S.tiny_crossing(1, start=15.0))
    ctx = mhc.Context(0, 64 << 20)
    try:
        poses = mhc.generate(ctx, cs)
        ref = mhc.detect(ctx, cs, poses).clone()
    finally:
        ctx.close()
    out = torch.full_like(ref, 1234)
    x = torch.zeros(8, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        ps = mhc.MhcPoses(poses["x"].data_ptr(), poses["y"].data_ptr(), poses["c"].data_ptr(), poses["s"].data_ptr())
        rc = mhc.lib.mhc_detect_collisions_static(cs.ref, ctypes.byref(ps), out.data_ptr(), s.cuda_stream)
        x.add_(1.0)
    assert rc == -1
    assert b"capture" in mhc.lib.mhc_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(x == 1.0) and torch.all(out == 1234)
    assert _static_detect(mhc, cs, poses, out) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_static_entry_rejects_scenarios_beyond_its_scratch(mhc):
    sc = S.stress32(4, n_steps=300)         # 2048 tiles x 300 steps x 16 B of bounds > 8 MiB
    cs = mhc.as_c(sc)
    dummy = {k: torch.zeros(1, dtype=torch.float32, device="cuda") for k in "xycs"}
    table = torch.zeros(1, dtype=torch.int16, device="cuda")
    rc = _static_detect(mhc, cs, dummy, table)
    assert rc == -1
    assert b"static scratch" in mhc.lib.mhc_last_error()


def test_static_entry_rejects_outlines(mhc):
    sc = S.with_outlines(S.tiny_crossing(1), cut=0.3)
    cs = mhc.as_c(sc)
    dummy = {k: torch.zeros(1, dtype=torch.float32, device="cuda") for k in "xycs"}
    table = torch.zeros(1, dtype=torch.int16, device="cuda")
    rc = _static_detect(mhc, cs, dummy, table)
    assert rc == -1
    assert b"rectangles only" in mhc.lib.mhc_last_error()
