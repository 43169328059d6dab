"""Shared helpers of the GPU-versus-oracle parity tests.

Acceptance (the method's tolerances):
  * poses: every rectangle corner (disc centre) within 1e-4 m of the oracle's;
  * first-collision tables: equal, except hypothesis pairs whose disagreeing steps are all borderline,
    i.e. the oracle's exact signed margin there is below 1e-3 m in magnitude; such excused pairs must stay
    below 1e-5 of all pose-pair tests;
  * risk measures computed from the same table: integer outputs identical, probabilities within 1e-6
    relative (the stated tolerance).  On the GPU every per-collision term is formed in FP32 (relative
    rounding ~2e-7) and summed exactly in 64-bit fixed point.
"""
import numpy as np

from oracle import parity
from oracle.parity import BORDER_TOL  # noqa: F401  (1 mm: the borderline band)

POSE_TOL = 1e-4
EXCUSE_FRACTION = 1e-5
PROB_RTOL = 1e-6


def corner_error(sc, orc_poses, gx, gy, gc, gs):
    """Largest corner (or centre) distance between GPU and oracle poses, per object kind."""
    ox, oy, oc, os_ = (orc_poses[k] for k in ("x", "y", "c", "s"))
    off = np.concatenate([[0], np.cumsum([o.grid_a.size * o.grid_b.size for o in sc.objects])])
    worst = 0.0
    for q, o in enumerate(sc.objects):
        sl = slice(off[q], off[q + 1])
        dx, dy = gx[sl] - ox[sl], gy[sl] - oy[sl]
        if o.kind == 0:
            hl, hw = o.length / 2, o.width / 2
            for sl_, sw in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                ex = dx + sl_ * hl * (gc[sl] - oc[sl]) - sw * hw * (gs[sl] - os_[sl])
                ey = dy + sl_ * hl * (gs[sl] - os_[sl]) + sw * hw * (gc[sl] - oc[sl])
                worst = max(worst, float(np.hypot(ex, ey).max()))
        else:
            worst = max(worst, float(np.hypot(dx, dy).max()))
    return worst


def check_table(orc, sc, tab_gpu, tab_orc, poses_orc, pairs, poff, n_tests=None, idx=None):
    """Assert the GPU table matches the oracle's up to borderline steps.  `idx` optionally lists the table
    indices the two arrays hold (sampled comparison).  Returns (n_disagree, n_excused).

    The excuse bound is EXCUSE_FRACTION of the pose tests rounded up to a whole pair: a scene of fewer
    than 1e5 tests may still have one excused pair (a single borderline pose pair), larger scenes have
    fewer than 1e-5 of their tests plus one."""
    tab_gpu = np.asarray(tab_gpu)
    tab_orc = np.asarray(tab_orc)
    assert tab_gpu.shape == tab_orc.shape
    assert tab_gpu.min(initial=-1) >= -1 and tab_gpu.max(initial=-1) < sc.n_steps
    r = parity.table_agreement(sc, tab_gpu, tab_orc, poses_orc, pairs, poff, idx=idx)
    assert r["n_bad"] == 0, r["bad"]
    total = n_tests if n_tests is not None else tab_gpu.size * sc.n_steps
    assert r["n_excused"] < EXCUSE_FRACTION * total + 1, (r["n_excused"], total)
    return r["n_disagree"], r["n_excused"]


def check_risk(gpu, orc_r, he):
    """GPU risk outputs (torch tensors) against the oracle's from the same table."""
    g = {k: v.detach().cpu().numpy() for k, v in gpu.items()}
    np.testing.assert_array_equal(g["count"], orc_r["count"])
    np.testing.assert_array_equal(g["count_k"], orc_r["count_k"])
    np.testing.assert_array_equal(g["hits"], orc_r["hits"])
    n_esc = int(g["n_escape"][0])
    assert n_esc == len(orc_r["escape"])
    np.testing.assert_array_equal(g["escape"][:n_esc], orc_r["escape"])
    assert np.all(g["escape"][n_esc:] == -1)
    for k in ("P", "H", "naive", "cond", "indep", "attr_obj", "attr_step"):
        np.testing.assert_allclose(g[k], orc_r[k], rtol=PROB_RTOL, atol=1e-15, err_msg=k)
    np.testing.assert_allclose(g["scalars"][:3], orc_r["scalars"], rtol=PROB_RTOL, atol=1e-15)
