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


def test_static_entry_matches_ordinary_entry(mhc):
    ctx = mhc.Context(0, 256 << 20)
    try:
        big = mhc.as_c(S.intersection11(2))
        small = mhc.as_c(S.intersection11(5, n_steps=40, n_acc=9, n_str=7, n_ped_v=5, n_ped_h=9))
        refs = {}
        for cs in (big, small):
            p = mhc.generate(ctx, cs)
            refs[id(cs)] = (p, mhc.detect(ctx, cs, p).clone())
        torch.cuda.synchronize()
        for cs in (big, big, small, big):        # two calls in a row, then another scenario, then back
            p, ref = refs[id(cs)]
            out = torch.full_like(ref, 1234)
            rc = _static_detect(mhc, cs, p, out)
            torch.cuda.synchronize()
            assert rc == 0, mhc.lib.mhc_last_error().decode()
            assert torch.equal(out, ref)
            assert int((ref >= 0).sum()) > 0
    finally:
        ctx.close()


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
