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

POSE_TOL = 1e-4
BORDER_TOL = 1e-3
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


def locate(idx, poff, pairs, h):
    """Table index -> (pair, i, j)."""
    q = int(np.searchsorted(poff, idx, side="right") - 1)
    a, b = pairs[q]
    i, j = divmod(int(idx - poff[q]), int(h[b]))
    return q, a, b, i, j


def check_table(orc, sc, tab_gpu, tab_orc, poses_orc, pairs, poff, n_tests=None, idx=None):
    """Assert the GPU table matches the oracle's up to borderline steps.  `idx` optionally lists the table
    indices the two arrays hold (sampled comparison).  Returns (n_disagree, n_excused, band_count)."""
    tab_gpu = np.asarray(tab_gpu)
    tab_orc = np.asarray(tab_orc)
    assert tab_gpu.shape == tab_orc.shape
    assert tab_gpu.min() >= -1 and tab_gpu.max() < sc.n_steps
    diff = np.nonzero(tab_gpu != tab_orc)[0]
    if diff.size == 0:
        return 0, 0
    off = orc.traj_offsets(sc)
    h = np.diff(off)
    oa, ta, ob, tb = [], [], [], []
    for d in diff:
        where = int(d if idx is None else idx[d])
        _, a, b, i, j = locate(where, poff, pairs, h)
        oa.append(a); ob.append(b); ta.append(off[a] + i); tb.append(off[b] + j)
    m = orc.margins(sc, poses_orc, oa, ta, ob, tb)
    N = sc.n_steps
    for r, d in enumerate(diff):
        kg, ko = int(tab_gpu[d]), int(tab_orc[d])
        kg_eff = kg if kg >= 0 else N
        # oracle overlaps the GPU missed (before the GPU's first hit) must be borderline
        missed = np.nonzero(m[r, :kg_eff] <= 0)[0]
        assert np.all(np.abs(m[r, missed]) < BORDER_TOL), (d, kg, ko, m[r, missed])
        if kg >= 0 and m[r, kg] > 0:   # GPU hit where the oracle sees a gap: must be borderline
            assert m[r, kg] < BORDER_TOL, (d, kg, ko, m[r, kg])
    total = n_tests if n_tests is not None else tab_gpu.size * N
    assert diff.size < EXCUSE_FRACTION * total + 1, (diff.size, total)
    return int(diff.size), int(diff.size)


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
