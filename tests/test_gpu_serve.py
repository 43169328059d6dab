"""GPU serving loop (continuous batching): every result is the same alone and in the mix; requests arriving
while batches run are admitted as slots and pool memory free up; small requests are not held behind a large
one; admission and error paths."""
import time

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
    return m


def _mix():
    """Requests of different shapes: small intersections, the 11-object scene, tiny crossings, EGO-only."""
    out = []
    for q in range(12):
        out.append(S.intersection11(20 + q, n_steps=20 + q, n_acc=5 + q % 4, n_str=7, n_ped_v=4, n_ped_h=5))
    out += [S.intersection11(2), S.intersection11(3), S.tiny_crossing(1), S.tiny_crossing(2, start=15.0)]
    sc = S.intersection11(9, n_steps=40, n_acc=6, n_str=6, n_ped_v=3, n_ped_h=3)
    sc.pair_mode, sc.ego = S.EGO_ONLY, 1
    out.append(sc)
    out += S.batch_scenarios(seed=33, count=6, n_lo=2, n_hi=8, h_lo=16, h_hi=200)
    return out


def _same(a, b, what):
    for k in a:
        x, y = a[k].numpy(), b[k].numpy()
        if k == "scalars":
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-18, err_msg=what)
        else:
            np.testing.assert_array_equal(x, y, err_msg=f"{k} {what}")


def test_results_alone_and_in_the_mix(mhc):
    """Each served result equals the plain single-scenario run (mhc_run) of the same request, whatever batch
    it shared; its resident table equals mhc_detect_collisions alone."""
    ctx = mhc.Context(0, 512 << 20)
    srv = mhc.Server(ctx, 1 << 30, max_batch=8)
    try:
        mix = _mix()
        ws = [S.random_weights(sc, 100 + q) if q % 3 == 0 else None for q, sc in enumerate(mix)]
        tickets = []
        srv.pause(True)                       # the first eight queue up and share a batch
        for q, sc in enumerate(mix):          # the rest arrive while batches run
            tickets.append(srv.submit(sc, ws[q]))
            if q == 7:
                srv.pause(False)
            if q > 7 and q % 5 == 4:
                time.sleep(0.0005)
        outs = []
        for t, sc in zip(tickets, mix):
            o = mhc.alloc_risk(sc, device="cpu")
            assert srv.poll(t, o, timeout_us=30_000_000)
            outs.append(o)
        sizes = [srv.times(t)[1] for t in tickets]
        assert max(sizes) > 1                 # some requests shared a batch
        solo = mhc.Context(0, 512 << 20)
        for q, (t, sc) in enumerate(zip(tickets, mix)):
            ref = mhc.run(solo, sc, weights=ws[q])
            _same(outs[q], ref, f"request {q}")
            if q % 4 == 0:
                poses, table_addr, _ = srv.buffers(t)
                n = mhc.layout(sc)["n_entries"]
                served = mhc.device_view(table_addr, n, torch.int16).clone()
                p = mhc.generate(solo, sc)
                alone = mhc.detect(solo, sc, p)
                torch.cuda.synchronize()
                assert torch.equal(served, alone), q
        solo.close()
        for t in tickets:
            srv.release(t)
        deadline = time.time() + 5
        while srv.stats()["pool_free"] != (1 << 30) and time.time() < deadline:
            time.sleep(0.01)
        st = srv.stats()
        assert st["pool_free"] == 1 << 30 and st["completed"] == len(mix)
    finally:
        srv.stop()
        ctx.close()


def test_small_requests_not_held_behind_a_large_one(mhc):
    """A 32-vehicle request (1e11 tests, large lane) in flight; small requests submitted after it finish
    before it."""
    ctx = mhc.Context(0, 256 << 20)
    srv = mhc.Server(ctx, 12 << 30)
    try:
        big_sc = mhc.as_c(S.stress32(4))
        small_sc = [mhc.as_c(S.intersection11(40 + q)) for q in range(10)]
        warm = srv.submit(small_sc[0])                  # module load, pinned buffers
        assert srv.poll(warm, None, timeout_us=30_000_000)
        srv.release(warm)
        big = srv.submit(big_sc)
        time.sleep(0.001)
        small = [srv.submit(cs) for cs in small_sc]
        assert srv.poll(big, None, timeout_us=0) is False      # the large request is still in flight
        for t in small:
            assert srv.poll(t, None, timeout_us=30_000_000)
        assert srv.poll(big, None, timeout_us=60_000_000)
        t_big = srv.times(big)[0][2]
        assert all(srv.times(t)[0][2] < t_big for t in small)
        for t in small + [big]:
            srv.release(t)
    finally:
        srv.stop()
        ctx.close()


def test_pause_pending_release_and_busy(mhc):
    ctx = mhc.Context(0, 64 << 20)
    srv = mhc.Server(ctx, 256 << 20, max_queue=3)
    try:
        srv.pause(True)
        a = srv.submit(S.tiny_crossing(1))
        b = srv.submit(S.tiny_crossing(3))
        c = srv.submit(S.tiny_crossing(4))
        with pytest.raises(mhc.MhcError) as e:
            srv.submit(S.tiny_crossing(5))
        assert e.value.code == -5                       # MHC_E_BUSY: queue full
        assert srv.poll(a, None, timeout_us=2000) is False   # paused: still pending
        srv.release(b)                                  # withdrawn while queued
        with pytest.raises(mhc.MhcError) as e:
            srv.poll(b, None, timeout_us=0)
        assert e.value.code == -6                       # MHC_E_NOTFOUND
        srv.pause(False)
        assert srv.poll(a, None, timeout_us=10_000_000) and srv.poll(c, None, timeout_us=10_000_000)
        srv.release(a)
        srv.release(c)
        with pytest.raises(mhc.MhcError):
            srv.release(a)
    finally:
        srv.stop()
        ctx.close()


def test_admission_errors(mhc):
    ctx = mhc.Context(0, 64 << 20)
    srv = mhc.Server(ctx, 2 << 20)
    try:
        with pytest.raises(mhc.MhcError) as e:
            srv.submit(S.intersection11(2))             # needs ~20 MB: never fits a 2 MiB pool
        assert e.value.code == -2
        bad = S.tiny_crossing(1)
        bad.n_steps = 0
        with pytest.raises(mhc.MhcError) as e:
            srv.submit(bad)
        assert e.value.code == -1
        t = srv.submit(S.tiny_crossing(1))
        assert srv.poll(t, None, timeout_us=10_000_000)
        srv.release(t)
    finally:
        srv.stop()
        ctx.close()


def test_memory_bounded_admission(mhc):
    """A pool that holds about three 11-object requests: twenty of them complete as memory is released."""
    ctx = mhc.Context(0, 64 << 20)
    one = mhc.layout(S.intersection11(2))["run_bytes"]
    srv = mhc.Server(ctx, int(3.5 * one))
    try:
        tickets = [srv.submit(S.intersection11(60 + q)) for q in range(20)]
        done = 0
        for t in tickets:
            assert srv.poll(t, None, timeout_us=30_000_000)
            srv.release(t)
            done += 1
        assert done == 20
    finally:
        srv.stop()
        ctx.close()
