"""Python access to the FP64 CPU oracle (``mhc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg are the only users.  Nothing here imports the CUDA library or its Python binding; scenarios are read
by attribute (objects, tau, n_steps, substeps, model, pair_mode, ego), so any object with that shape works.

Each function names the part of the paper (arXiv 2005.06773) it restates; the C file carries the
formulas and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmhc_oracle.so")
_lock = threading.Lock()
_lib = None

# The oracle's own default one-track parameters (m, I_z, l_f, l_r, c_af, c_ar), used when an object
# carries none.  The paper does not print them (Section IV-B.1); these are the project's reading.
_DEFAULT_PARAMS = (1500.0, 2500.0, 1.2, 1.5, 80000.0, 80000.0)

D = np.float64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)
_sp = ctypes.POINTER(ctypes.c_int16)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, no architecture flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-D_DEFAULT_SOURCE", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_margin.restype = ctypes.c_double
            _lib.orc_margin.argtypes = [ctypes.c_int] + [ctypes.c_double] * 7 + [ctypes.c_int] + [ctypes.c_double] * 7
            _lib.orc_margin_shapes.restype = ctypes.c_double
            _lib.orc_overlap_pip.restype = ctypes.c_int
            _lib.orc_overlap_pip.argtypes = [ctypes.c_double] * 12
    return _lib


def _p(a: np.ndarray, ptr):
    return a.ctypes.data_as(ptr)


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.int32)


def _i64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.int64)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=D)


def traj_offsets(sc) -> np.ndarray:
    """Global trajectory index of hypothesis 0 of each object (prefix sum of h_a, Eq. threads:traj)."""
    h = [int(o.grid_a.size) * int(o.grid_b.size) for o in sc.objects]
    return _i64(np.concatenate([[0], np.cumsum(h)]))


def pair_list(sc) -> List[Tuple[int, int]]:
    """Object pairs tested for collisions: every pair a < b, or EGO against every CO (Section IV-C.1)."""
    n = len(sc.objects)
    if int(sc.pair_mode) == 1:
        return [(int(sc.ego), b) for b in range(n) if b != int(sc.ego)]
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def pair_offsets(sc, pairs=None) -> np.ndarray:
    pairs = pair_list(sc) if pairs is None else pairs
    h = np.diff(traj_offsets(sc))
    sizes = [int(h[a]) * int(h[b]) for a, b in pairs]
    return _i64(np.concatenate([[0], np.cumsum(sizes)]))


def _objects(sc):
    objs = sc.objects
    kind = _i32([o.kind for o in objs])
    f = lambda name: _f64([getattr(o, name) for o in objs])
    n_a = _i32([o.grid_a.size for o in objs])
    n_b = _i32([o.grid_b.size for o in objs])
    grids = _f64(np.concatenate([np.concatenate([np.asarray(o.grid_a, D), np.asarray(o.grid_b, D)]) for o in objs]))
    grid_off = _i64(np.concatenate([[0], np.cumsum(n_a.astype(np.int64) + n_b)])[:-1])
    params = _f64(np.concatenate([np.asarray(o.params if o.params is not None else _DEFAULT_PARAMS, D)
                                  for o in objs]))
    flags = _i32([getattr(o, "flags", 0) for o in objs])
    return dict(kind=kind, length=f("length"), width=f("width"), radius=f("radius"), x0=f("x0"), y0=f("y0"),
                psi0=f("psi0"), v0=f("v0"), v_max=f("v_max"), n_a=n_a, n_b=n_b, grids=grids,
                grid_off=grid_off, params=params, flags=flags)


def generate(sc) -> Dict[str, np.ndarray]:
    """Every hypothesis of every object integrated in FP64 (Section IV-B, Eqs. onetrack, EulerVelocity,
    pedestrianmotion).  Returns x, y, psi, c = cos(psi), s = sin(psi) as [n_traj_total, N] arrays and the
    trajectory offsets."""
    L = lib()
    ob = _objects(sc)
    off = traj_offsets(sc)
    T, N = int(off[-1]), int(sc.n_steps)
    x = np.zeros((T, N), D); y = np.zeros((T, N), D); psi = np.zeros((T, N), D)
    keep = _set_paths(sc)  # noqa: F841 (alive during the call)
    L.orc_generate(ctypes.c_int(len(sc.objects)), _p(ob["kind"], _ip), _p(ob["x0"], _dp), _p(ob["y0"], _dp),
                   _p(ob["psi0"], _dp), _p(ob["v0"], _dp), _p(ob["n_a"], _ip), _p(ob["n_b"], _ip),
                   _p(ob["grid_off"], _lp), _p(ob["grids"], _dp), _p(ob["params"], _dp), _p(ob["v_max"], _dp),
                   _p(ob["flags"], _ip), ctypes.c_double(sc.tau), ctypes.c_int(N), ctypes.c_int(int(sc.substeps)),
                   ctypes.c_int(int(sc.model)), _p(x, _dp), _p(y, _dp), _p(psi, _dp))
    return dict(x=x, y=y, psi=psi, c=np.cos(psi), s=np.sin(psi), traj_off=off)


def _set_paths(sc):
    """Registers the vehicles' paths (reading R-s: [n_b, 3 sections, (x, y, psi)]) with the C oracle for the
    next call (none: cleared).  Returns the arrays, which must stay alive during that call."""
    L = lib()
    has = [getattr(o, "paths", None) is not None for o in sc.objects]
    if not any(has):
        L.orc_set_paths(ctypes.c_int(0), None, None)
        return None
    off, data, at = [], [], 0
    for o, h in zip(sc.objects, has):
        if h:
            pa = np.asarray(o.paths, D).reshape(-1, 9)
            off.append(at)
            data.append(pa.reshape(-1))
            at += pa.shape[0]
        else:
            off.append(-1)
    off = _i64(off)
    data = _f64(np.concatenate(data))
    L.orc_set_paths(ctypes.c_int(len(sc.objects)), _p(off, _lp), _p(data, _dp))
    return off, data


def path_steering(x0, y0, psi0, v0, vdot, path, params=None, model=0, tau=0.1, n_steps=20, substeps=5):
    """One path hypothesis (readings R-s .. R-u): poses [N] x, y, psi and the steering angle of every
    sub-step [N K]."""
    L = lib()
    pa = _f64(np.asarray(path, D).reshape(-1))
    pr = _f64(params if params is not None else _DEFAULT_PARAMS)
    N, K = int(n_steps), int(substeps)
    x = np.zeros(N, D); y = np.zeros(N, D); psi = np.zeros(N, D); dl = np.zeros(N * K, D)
    L.orc_path_steering(ctypes.c_double(x0), ctypes.c_double(y0), ctypes.c_double(psi0), ctypes.c_double(v0),
                        ctypes.c_double(vdot), _p(pa, _dp), _p(pr, _dp), ctypes.c_int(model), ctypes.c_double(tau),
                        ctypes.c_int(N), ctypes.c_int(K), _p(x, _dp), _p(y, _dp), _p(psi, _dp), _p(dl, _dp))
    return dict(x=x, y=y, psi=psi, delta=dl)


def divider_fit(points):
    """y = a x^2 + b x + c through three (x, y) points (Section IV-A, Gauss-Jordan); None if undetermined."""
    pts = _f64(np.asarray(points, D).reshape(-1))
    cf = np.zeros(3, D)
    rc = lib().orc_divider_fit(_p(pts, _dp), _p(cf, _dp))
    return None if rc else cf


def lane_paths(dividers, x0, y0, psi0, v0, ego=False):
    """Paths of one vehicle from its lane dividers (readings R-v, R-w): dividers [n_div, 3, 2] in the
    vehicle frame, right to left.  Returns [n_paths, 3, 3] (x, y, psi) in the scenario frame, or None."""
    dv = _f64(np.asarray(dividers, D).reshape(-1))
    out = np.zeros((343, 3, 3), D)
    n = lib().orc_lane_paths(_p(dv, _dp), ctypes.c_int(len(dv) // 6), ctypes.c_double(x0), ctypes.c_double(y0),
                             ctypes.c_double(psi0), ctypes.c_double(v0), ctypes.c_int(int(ego)), _p(out, _dp))
    return None if n < 0 else out[:n].copy()


def _set_polygons(sc):
    """Registers the objects' convex outlines with the C oracle for the next call (none: cleared).
    Returns the arrays, which must stay alive during that call."""
    L = lib()
    nv = _i32([0 if getattr(o, "outline", None) is None else len(o.outline) for o in sc.objects])
    if not nv.any():
        L.orc_set_polygons(ctypes.c_int(0), None, None, None)
        return None
    off = _i64(np.concatenate([[0], np.cumsum(nv.astype(np.int64))])[:-1])
    verts = _f64(np.concatenate([np.asarray(o.outline, D).reshape(-1) for o in sc.objects
                                 if getattr(o, "outline", None) is not None]))
    L.orc_set_polygons(ctypes.c_int(len(sc.objects)), _p(nv, _ip), _p(off, _lp), _p(verts, _dp))
    return nv, off, verts


def table(sc, poses: Dict[str, np.ndarray], pairs=None) -> Tuple[np.ndarray, np.ndarray, list]:
    """First-collision step of every trajectory combination of every listed object pair (Section IV-C);
    -1 where the closed shapes never overlap within the horizon.  Returns (table, pair_off, pairs)."""
    L = lib()
    ob = _objects(sc)
    off = traj_offsets(sc)
    pairs = pair_list(sc) if pairs is None else list(pairs)
    poff = pair_offsets(sc, pairs)
    out = np.empty(int(poff[-1]), np.int16)
    pa = _i32([p[0] for p in pairs]); pb = _i32([p[1] for p in pairs])
    px, py, pc, ps = (_f64(poses[k]) for k in ("x", "y", "c", "s"))
    keep = _set_polygons(sc)  # noqa: F841 (alive during the call)
    L.orc_table(ctypes.c_int(len(sc.objects)), _p(ob["kind"], _ip), _p(ob["length"], _dp), _p(ob["width"], _dp),
                _p(ob["radius"], _dp), _p(off, _lp), ctypes.c_int(int(sc.n_steps)),
                _p(px, _dp), _p(py, _dp), _p(pc, _dp), _p(ps, _dp), ctypes.c_int(len(pairs)),
                _p(pa, _ip), _p(pb, _ip), _p(poff, _lp), _p(out, _sp))
    return out, poff, pairs


def margins(sc, poses, oa, ta, ob_, tb) -> np.ndarray:
    """Signed separation margin (m) at every step for the listed trajectory pairs: [n_q, N].
    oa/ob are object indices, ta/tb global trajectory indices."""
    L = lib()
    ob = _objects(sc)
    oa, ob_ = _i32(oa), _i32(ob_)
    ta, tb = _i64(ta), _i64(tb)
    N = int(sc.n_steps)
    out = np.empty((oa.size, N), D)
    px, py, pc, ps = (_f64(poses[k]) for k in ("x", "y", "c", "s"))
    keep = _set_polygons(sc)  # noqa: F841 (alive during the call)
    L.orc_margins(_p(ob["kind"], _ip), _p(ob["length"], _dp), _p(ob["width"], _dp), _p(ob["radius"], _dp),
                  ctypes.c_int(N), _p(px, _dp), _p(py, _dp), _p(pc, _dp), _p(ps, _dp),
                  ctypes.c_long(oa.size), _p(oa, _ip), _p(ta, _lp), _p(ob_, _ip), _p(tb, _lp), _p(out, _dp))
    return out


def first_steps(sc, poses, oa, ta, ob_, tb) -> np.ndarray:
    """First-collision step (or -1) of the listed trajectory pairs, same definition as table()."""
    L = lib()
    ob = _objects(sc)
    oa, ob_ = _i32(oa), _i32(ob_)
    ta, tb = _i64(ta), _i64(tb)
    out = np.empty(oa.size, np.int16)
    px, py, pc, ps = (_f64(poses[k]) for k in ("x", "y", "c", "s"))
    keep = _set_polygons(sc)  # noqa: F841 (alive during the call)
    L.orc_first(_p(ob["kind"], _ip), _p(ob["length"], _dp), _p(ob["width"], _dp), _p(ob["radius"], _dp),
                ctypes.c_int(int(sc.n_steps)), _p(px, _dp), _p(py, _dp), _p(pc, _dp), _p(ps, _dp),
                ctypes.c_long(oa.size), _p(oa, _ip), _p(ta, _lp), _p(ob_, _ip), _p(tb, _lp), _p(out, _sp))
    return out


def margin(kind_a, len_a, wid_a, rad_a, xa, ya, psi_a, kind_b, len_b, wid_b, rad_b, xb, yb, psi_b) -> float:
    """Signed margin of two shapes (rectangle: kind 0, disc: kind 1) given centre and heading."""
    return lib().orc_margin(kind_a, len_a, wid_a, rad_a, xa, ya, np.cos(psi_a), np.sin(psi_a),
                            kind_b, len_b, wid_b, rad_b, xb, yb, np.cos(psi_b), np.sin(psi_b))


def margin_shapes(a: dict, b: dict):
    """Signed margin and closed overlap flag of two shapes given directly as dicts with kind (0 rectangle,
    1 disc, 2 convex polygon), length, width, radius, outline ([n, 2] body frame), x, y, psi."""
    L = lib()
    args, keep = [], []
    for d in (a, b):
        v = _f64(np.asarray(d.get("outline", np.zeros((0, 2))), D).reshape(-1))
        keep.append(v)
        args += [ctypes.c_int(int(d["kind"])), ctypes.c_double(d.get("length", 0.0)), ctypes.c_double(d.get("width", 0.0)),
                 ctypes.c_double(d.get("radius", 0.0)), ctypes.c_int(v.size // 2), _p(v, _dp),
                 ctypes.c_double(d["x"]), ctypes.c_double(d["y"]), ctypes.c_double(np.cos(d["psi"])),
                 ctypes.c_double(np.sin(d["psi"]))]
    flag = ctypes.c_int(0)
    m = L.orc_margin_shapes(*args, ctypes.byref(flag))
    return float(m), bool(flag.value)


def overlap_pip(len_a, wid_a, xa, ya, psi_a, len_b, wid_b, xb, yb, psi_b) -> bool:
    """The paper's vertex-in-polygon test, both directions (Section IV-C.1)."""
    return bool(lib().orc_overlap_pip(len_a, wid_a, xa, ya, np.cos(psi_a), np.sin(psi_a),
                                      len_b, wid_b, xb, yb, np.cos(psi_b), np.sin(psi_b)))


def scores(sc) -> List[np.ndarray]:
    """Eq. (normTraj) scores n_h of every hypothesis (reading R-x), one array per object."""
    L = lib()
    ob = _objects(sc)
    off = traj_offsets(sc)
    out = np.zeros(int(off[-1]), D)
    keep = _set_paths(sc)  # noqa: F841 (alive during the call)
    L.orc_scores(ctypes.c_int(len(sc.objects)), _p(ob["kind"], _ip), _p(ob["x0"], _dp), _p(ob["y0"], _dp),
                 _p(ob["psi0"], _dp), _p(ob["v0"], _dp), _p(ob["n_a"], _ip), _p(ob["n_b"], _ip),
                 _p(ob["grid_off"], _lp), _p(ob["grids"], _dp), _p(ob["flags"], _ip), _p(out, _dp))
    return [out[off[q]:off[q + 1]].copy() for q in range(len(sc.objects))]


def normalise(sc, weights: Optional[Sequence[np.ndarray]] = None) -> np.ndarray:
    """Per-object L1 normalisation of trajectory weights into occurrence probabilities (Section IV-D.1).
    None means uniform weights."""
    off = traj_offsets(sc)
    if weights is None:
        w = np.ones(int(off[-1]), D)
    else:
        w = _f64(np.concatenate([np.asarray(x, D) for x in weights]))
    prob = np.empty_like(w)
    rc = lib().orc_normalise(ctypes.c_int(len(sc.objects)), _p(off, _lp), _p(w, _dp), _p(prob, _dp))
    if rc != 0:
        raise ValueError("trajectory weights must be non-negative with a positive sum per object")
    return prob


def risk(sc, tab: np.ndarray, pairs=None, weights=None) -> Dict[str, np.ndarray]:
    """Risk measures of Section IV-D from a first-collision table (see orc_risk in the C file)."""
    L = lib()
    off = traj_offsets(sc)
    pairs = pair_list(sc) if pairs is None else list(pairs)
    poff = pair_offsets(sc, pairs)
    prob = normalise(sc, weights)
    n_obj, N, e = len(sc.objects), int(sc.n_steps), int(sc.ego)
    he = int(off[e + 1] - off[e])
    npairs = len(pairs)
    pa = _i32([p[0] for p in pairs]); pb = _i32([p[1] for p in pairs])
    tab = np.ascontiguousarray(tab, np.int16)
    r = dict(count=np.zeros(npairs, np.int64), count_k=np.zeros((npairs, N), np.int64),
             P=np.zeros(npairs, D), H=np.zeros((npairs, N), D), naive=np.zeros(he, D), cond=np.zeros(he, D),
             indep=np.zeros(he, D), hits=np.zeros(he, np.int32), attr_obj=np.zeros(n_obj, D),
             attr_step=np.zeros(N, D), scalars=np.zeros(3, D), escape=np.zeros(he, np.int32))
    ne = ctypes.c_int(0)
    rc = L.orc_risk(ctypes.c_int(n_obj), _p(off, _lp), ctypes.c_int(N), ctypes.c_int(e), ctypes.c_int(npairs),
                    _p(pa, _ip), _p(pb, _ip), _p(poff, _lp), _p(tab, _sp), _p(prob, _dp),
                    _p(r["count"], _lp), _p(r["count_k"], _lp), _p(r["P"], _dp), _p(r["H"], _dp),
                    _p(r["naive"], _dp), _p(r["cond"], _dp), _p(r["indep"], _dp), _p(r["hits"], _ip),
                    _p(r["attr_obj"], _dp), _p(r["attr_step"], _dp), _p(r["scalars"], _dp),
                    _p(r["escape"], _ip), ctypes.byref(ne))
    if rc != 0:
        raise MemoryError("oracle risk ran out of memory")
    r["escape"] = r["escape"][: ne.value].copy()
    r["p_cra"], r["p_cra_cond"], r["p_cra_indep"] = (float(v) for v in r["scalars"])
    r["prob"] = prob
    return r


def run(sc, weights=None) -> Dict[str, object]:
    """Whole method: generate -> table -> risk."""
    poses = generate(sc)
    tab, poff, pairs = table(sc, poses)
    return dict(poses=poses, table=tab, pair_off=poff, pairs=pairs, risk=risk(sc, tab, pairs, weights))
