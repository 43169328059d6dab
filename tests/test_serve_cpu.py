"""Host logic of the serving loop that needs no GPU: the first-fit pool allocator that admits requests by
free device memory, and the serving calls' error paths without a serving loop."""
import ctypes

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S


@pytest.fixture(scope="module")
def mhc():
    from paper_2005_06773_gb300 import mhc as m
    return m


def test_pool_first_fit_and_merge(mhc):
    p = mhc.Pool(1 << 20)
    a = p.alloc(1000)            # rounded to 1024
    b = p.alloc(256)
    c = p.alloc(4096)
    assert (a, b, c) == (0, 1024, 1280)
    free, largest, n = p.info()
    assert free == (1 << 20) - 1024 - 256 - 4096 and n == 1
    p.free(b)                    # a hole of 256 before c
    assert p.alloc(200) == 1024  # first fit reuses it
    p.free(1024)
    p.free(a)                    # merges with the hole after it: [0, 1280)
    free, largest, n = p.info()
    assert n == 2
    assert p.alloc(1280) == 0
    p.free(0)
    p.free(c)                    # everything merges back into one block
    assert p.info() == (1 << 20, 1 << 20, 1)
    p.close()


def test_pool_errors(mhc):
    p = mhc.Pool(4096)
    with pytest.raises(mhc.MhcError) as e:
        p.alloc(8192)
    assert e.value.code == -2            # MHC_E_NOMEM
    with pytest.raises(mhc.MhcError) as e:
        p.free(256)
    assert e.value.code == -6            # MHC_E_NOTFOUND
    x = p.alloc(4096)
    with pytest.raises(mhc.MhcError):
        p.alloc(1)
    p.free(x)
    with pytest.raises(mhc.MhcError) as e:
        p.free(x)                        # double free
    assert e.value.code == -6
    with pytest.raises(mhc.MhcError):
        mhc.Pool(100)
    p.close()


def test_pool_random_sequence_against_a_model(mhc):
    """Random alloc / free sequence against a byte-map model: blocks never overlap, free bytes add up, and
    first fit returns the lowest offset that fits."""
    rng = S.SplitMix64(7)
    size = 1 << 16
    p = mhc.Pool(size)
    used = np.zeros(size // 256, bool)
    live = {}
    for _ in range(2000):
        if live and rng.uniform(0, 1) < 0.45:
            off = list(live)[rng.randint(0, len(live) - 1)]
            p.free(off)
            used[off // 256: off // 256 + live.pop(off)] = False
        else:
            units = rng.randint(1, 24)
            # the model's first fit
            want = None
            run = 0
            for q in range(used.size):
                run = run + 1 if not used[q] else 0
                if run == units:
                    want = (q - units + 1) * 256
                    break
            if want is None:
                with pytest.raises(mhc.MhcError):
                    p.alloc(units * 256)
                continue
            off = p.alloc(units * 256 - rng.randint(0, 255))
            assert off == want
            used[off // 256: off // 256 + units] = True
            live[off] = units
        free, largest, n = p.info()
        assert free == (~used).sum() * 256
    p.close()


def test_serving_calls_without_a_loop(mhc):
    t = ctypes.c_uint64()
    sc = mhc.as_c(S.tiny_crossing(1))
    assert mhc.lib.mhc_submit(None, sc.ref, None, ctypes.byref(t)) == -6
    assert mhc.lib.mhc_poll(None, 1, None, 0) == -6
    assert mhc.lib.mhc_release(None, 1) == -6
    assert mhc.lib.mhc_serve_stop(None) == -6
    assert mhc.lib.mhc_serve_pause(None, 1) == -6
