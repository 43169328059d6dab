"""Agreement of a first-collision table with the oracle's (test infrastructure, like the rest of oracle/).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this module.  It holds no step of
the method: it compares a table against the oracle's table and measures, with the oracle's exact signed
margins (reading R-h: distance when disjoint, minus the penetration depth when overlapping), which
disagreements are borderline.

Acceptance of a table (GPU against oracle): a trajectory pair whose first-collision steps differ is
*excused* when every step on which the two disagree is borderline, i.e. the oracle's margin there lies
within BORDER_TOL = 1 mm of zero: steps before the GPU's first hit where the oracle sees an overlap, and
the GPU's first-hit step where the oracle sees a gap.  Any other disagreement is an error.
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from . import oracle as O

BORDER_TOL = 1e-3


def _locate(idx, poff, pairs, h):
    q = int(np.searchsorted(poff, idx, side="right") - 1)
    a, b = pairs[q]
    i, j = divmod(int(idx - poff[q]), int(h[b]))
    return a, b, i, j


def table_agreement(sc, tab_gpu, tab_orc, poses, pairs, poff, idx=None) -> Dict[str, object]:
    """Compare two tables entry by entry.  `idx` optionally lists the table indices both arrays hold (a
    sampled comparison).  Returns n_disagree, n_excused (disagreements with only borderline steps),
    n_bad (the others) and bad (up to 10 examples: index, GPU step, oracle step, offending margin)."""
    tab_gpu = np.asarray(tab_gpu)
    tab_orc = np.asarray(tab_orc)
    if tab_gpu.shape != tab_orc.shape:
        raise ValueError("tables of different shapes")
    diff = np.nonzero(tab_gpu != tab_orc)[0]
    out = {"n_disagree": int(diff.size), "n_excused": 0, "n_bad": 0, "bad": []}
    if diff.size == 0:
        return out
    off = O.traj_offsets(sc)
    h = np.diff(off)
    oa, ta, ob, tb = [], [], [], []
    for d in diff:
        a, b, i, j = _locate(int(d if idx is None else idx[d]), poff, pairs, h)
        oa.append(a); ob.append(b); ta.append(off[a] + i); tb.append(off[b] + j)
    m = O.margins(sc, poses, oa, ta, ob, tb)
    N = int(sc.n_steps)
    for r, d in enumerate(diff):
        kg, ko = int(tab_gpu[d]), int(tab_orc[d])
        kg_eff = kg if 0 <= kg < N else N
        missed = np.nonzero(m[r, :kg_eff] <= 0)[0]          # oracle overlaps before the GPU's first hit
        worst = float(np.abs(m[r, missed]).max()) if missed.size else 0.0
        if 0 <= kg < N and m[r, kg] > 0:                    # a GPU hit where the oracle sees a gap
            worst = max(worst, float(m[r, kg]))
        if kg >= N or kg < -1:
            worst = float("inf")
        if worst < BORDER_TOL:
            out["n_excused"] += 1
        else:
            out["n_bad"] += 1
            if len(out["bad"]) < 10:
                out["bad"].append((int(d), kg, ko, worst))
    return out


def circumradius(o) -> float:
    """Radius about the pose point of the circle that holds the object's shape."""
    outline = getattr(o, "outline", None)
    if outline is not None:
        v = np.asarray(outline, np.float64).reshape(-1, 2)
        return float(np.sqrt((v * v).sum(axis=1)).max())
    if o.kind == 0:
        return float(np.hypot(0.5 * float(o.length), 0.5 * float(o.width)))
    return float(o.radius)


def band_count(sc, poses, pairs=None, tol: float = BORDER_TOL, rows: Optional[int] = None) -> int:
    """Number of pose tests whose oracle margin lies strictly within tol of zero, over every trajectory
    pair of the listed object pairs.  A margin within tol needs the two centres within the sum of the
    circumradii plus tol, so only those pose pairs are handed to the oracle's margin function."""
    off = O.traj_offsets(sc)
    N = int(sc.n_steps)
    pairs = O.pair_list(sc) if pairs is None else list(pairs)
    X = np.asarray(poses["x"], np.float64).reshape(-1, N)
    Y = np.asarray(poses["y"], np.float64).reshape(-1, N)
    total = 0
    for a, b in pairs:
        reach = circumradius(sc.objects[a]) + circumradius(sc.objects[b]) + tol
        xa, ya = X[off[a]:off[a + 1]], Y[off[a]:off[a + 1]]
        xb, yb = X[off[b]:off[b + 1]], Y[off[b]:off[b + 1]]
        step = rows or max(1, (1 << 22) // max(1, xb.shape[0] * N))
        ii, jj = [], []
        for i0 in range(0, xa.shape[0], step):
            dx = xa[i0:i0 + step, None, :] - xb[None, :, :]
            dy = ya[i0:i0 + step, None, :] - yb[None, :, :]
            near = ((dx * dx + dy * dy) <= reach * reach).any(axis=2)
            i, j = np.nonzero(near)
            ii.append(i + i0); jj.append(j)
        i = np.concatenate(ii); j = np.concatenate(jj)
        if i.size == 0:
            continue
        m = O.margins(sc, poses, np.full(i.size, a), off[a] + i, np.full(j.size, b), off[b] + j)
        total += int((np.abs(m) < tol).sum())
    return total
