"""Thin ctypes binding of the CUDA library (``include/mhc.h``).

Only argument marshalling lives here: scenarios become the C structs, torch tensors provide device memory
and the current CUDA stream, and every step of the method runs in the library's kernels.  Importing this
module loads ``_build/libmhc.so`` and raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int16, c_int32, c_int64, c_longlong, c_size_t, c_uint64, c_void_p
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

MHC_OK, MHC_PENDING = 0, 1
MHC_OPT_CULL = 1
MHC_OPT_PROFILE = 2
MHC_OPT_COLLIDE_VARIANT = 3
MHC_OPT_GEN_SCAN = 4
MHC_OPT_SCORE = 5
COUNTER_WORDS = 7
KERNEL_CLASSES = ("generate", "bounds", "collide", "risk")


class MhcError(RuntimeError):
    def __init__(self, code: int, where: str, reason: str):
        super().__init__(f"{where}: {_STATUS.get(code, code)} ({reason})")
        self.code = code


_STATUS = {0: "MHC_OK", 1: "MHC_PENDING", -1: "MHC_E_INVALID", -2: "MHC_E_NOMEM", -3: "MHC_E_CUDA",
           -4: "MHC_E_TIMEOUT", -5: "MHC_E_BUSY", -6: "MHC_E_NOTFOUND"}


class MhcObject(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("flags", c_int32), ("length", c_float), ("width", c_float),
                ("radius", c_float), ("x0", c_float), ("y0", c_float), ("psi0", c_float), ("v0", c_float),
                ("v_max", c_float), ("n_a", c_int32), ("n_b", c_int32), ("grid_a", POINTER(c_float)),
                ("grid_b", POINTER(c_float)), ("veh_params", POINTER(c_float)), ("n_vertices", c_int32),
                ("vertices", POINTER(c_float)), ("paths", POINTER(c_float))]


class MhcScenario(ctypes.Structure):
    _fields_ = [("n_objects", c_int32), ("objects", POINTER(MhcObject)), ("tau", c_float), ("n_steps", c_int32),
                ("substeps", c_int32), ("pair_mode", c_int32), ("ego", c_int32), ("model", c_int32)]


class MhcPoses(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("c", c_void_p), ("s", c_void_p)]


class MhcBatchInfo(ctypes.Structure):
    _fields_ = [("n_traj", c_int64), ("n_poses", c_int64), ("n_entries", c_int64), ("n_step_entries", c_int64),
                ("n_scen_steps", c_int64), ("h_ego", c_int64), ("n_pairs", c_int32), ("n_objects", c_int32),
                ("n_scenarios", c_int32), ("max_steps", c_int32), ("scratch", c_size_t), ("plan_bytes", c_size_t)]


class MhcBatchSlice(ctypes.Structure):
    _fields_ = [("obj0", c_int32), ("n_objects", c_int32), ("pair0", c_int32), ("n_pairs", c_int32),
                ("n_steps", c_int32), ("ego", c_int32), ("traj0", c_int64), ("pose0", c_int64),
                ("entry0", c_int64), ("step_entry0", c_int64), ("ego0", c_int64), ("step0", c_int64)]


MHC_PLAN_GRAPH = 1
MHC_PLAN_PIPELINE = 2


class MhcServeConfig(ctypes.Structure):
    _fields_ = [("small_slots", c_int32), ("large_slots", c_int32), ("max_batch", c_int32), ("max_queue", c_int32),
                ("small_tests", c_int64), ("max_batch_tests", c_int64)]


class MhcServeStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("batches", c_int64), ("queued", c_int64),
                ("running", c_int64), ("pool_free", c_size_t), ("pool_largest", c_size_t)]

RISK_FIELDS = ("count", "count_k", "P", "H", "naive", "cond", "indep", "hits", "attr_obj", "attr_step",
               "scalars", "escape", "n_escape")


class MhcRisk(ctypes.Structure):
    _fields_ = [(f, c_void_p) for f in RISK_FIELDS]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; call __graft_entry__.build() "
                          "(the method has no CPU fallback)")
    L = ctypes.CDLL(path)
    L.mhc_status_string.restype = ctypes.c_char_p
    L.mhc_last_error.restype = ctypes.c_char_p
    L.mhc_version.restype = ctypes.c_char_p
    L.mhc_create.argtypes = [POINTER(c_void_p), c_int, c_void_p, c_size_t]
    L.mhc_destroy.argtypes = [c_void_p]
    L.mhc_destroy.restype = None
    L.mhc_set_option.argtypes = [c_void_p, c_int, c_longlong]
    L.mhc_collision_counters.argtypes = [c_void_p, POINTER(c_uint64), c_int32, c_int, c_void_p]
    L.mhc_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int64), c_int]
    L.mhc_transfer_bytes.argtypes = [c_void_p, POINTER(c_int64), POINTER(c_int64)]
    L.mhc_layout.argtypes = [POINTER(MhcScenario), POINTER(c_int64), POINTER(c_int32), POINTER(c_int64),
                             POINTER(c_int32), POINTER(c_size_t)]
    L.mhc_pair_table.argtypes = [POINTER(MhcScenario), c_void_p, c_void_p, c_void_p]
    L.mhc_generate_trajectories.argtypes = [c_void_p, POINTER(MhcScenario), POINTER(MhcPoses), c_void_p]
    L.mhc_detect_collisions.argtypes = [c_void_p, POINTER(MhcScenario), POINTER(MhcPoses), c_void_p, c_void_p]
    L.mhc_assess_risk.argtypes = [c_void_p, POINTER(MhcScenario), c_void_p, c_void_p, POINTER(MhcRisk), c_void_p]
    L.mhc_evaluate.argtypes = [c_void_p, POINTER(MhcScenario), c_void_p, POINTER(MhcPoses), c_void_p,
                               POINTER(MhcRisk), c_void_p]
    L.mhc_autotune.argtypes = [c_void_p, POINTER(MhcScenario), POINTER(MhcPoses), c_void_p, c_int,
                               POINTER(c_int32), POINTER(c_int32), c_void_p]
    L.mhc_run_bytes.argtypes = [POINTER(MhcScenario), POINTER(c_size_t)]
    L.mhc_batch_layout.argtypes = [POINTER(MhcScenario), c_int32, POINTER(MhcBatchInfo), c_void_p]
    L.mhc_batch_pair_table.argtypes = [POINTER(MhcScenario), c_int32, c_void_p, c_void_p, c_void_p]
    L.mhc_evaluate_batch.argtypes = [c_void_p, POINTER(MhcScenario), c_int32, c_void_p, POINTER(MhcPoses),
                                     c_void_p, POINTER(MhcRisk), c_void_p]
    L.mhc_autotune_batch.argtypes = [c_void_p, POINTER(MhcScenario), c_int32, POINTER(MhcPoses), c_void_p, c_int,
                                     POINTER(c_int32), POINTER(c_int32), c_void_p]
    L.mhc_plan_create.argtypes = [c_void_p, POINTER(MhcScenario), c_int32, c_void_p, POINTER(MhcPoses), c_void_p,
                                  POINTER(MhcRisk), c_void_p, c_size_t, c_int32, POINTER(c_void_p)]
    L.mhc_plan_update.argtypes = [c_void_p, POINTER(MhcScenario), c_int32]
    L.mhc_plan_launch.argtypes = [c_void_p, c_void_p]
    L.mhc_plan_destroy.argtypes = [c_void_p]
    L.mhc_plan_destroy.restype = None
    L.mhc_serve_start.argtypes = [c_void_p, c_void_p, c_size_t, POINTER(MhcServeConfig)]
    L.mhc_serve_stop.argtypes = [c_void_p]
    L.mhc_submit.argtypes = [c_void_p, POINTER(MhcScenario), c_void_p, POINTER(c_uint64)]
    L.mhc_poll.argtypes = [c_void_p, c_uint64, POINTER(MhcRisk), c_int32]
    L.mhc_release.argtypes = [c_void_p, c_uint64]
    L.mhc_request_buffers.argtypes = [c_void_p, c_uint64, POINTER(MhcPoses), POINTER(c_void_p), POINTER(MhcRisk)]
    L.mhc_request_times.argtypes = [c_void_p, c_uint64, POINTER(c_int64), POINTER(c_int32)]
    L.mhc_serve_stats_read.argtypes = [c_void_p, POINTER(MhcServeStats)]
    L.mhc_serve_pause.argtypes = [c_void_p, c_int32]
    L.mhc_pool_create.argtypes = [c_size_t, POINTER(c_void_p)]
    L.mhc_pool_alloc.argtypes = [c_void_p, c_size_t, POINTER(c_size_t)]
    L.mhc_pool_free.argtypes = [c_void_p, c_size_t]
    L.mhc_pool_info.argtypes = [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_int32)]
    L.mhc_pool_destroy.argtypes = [c_void_p]
    L.mhc_pool_destroy.restype = None
    L.mhc_run.argtypes = [c_void_p, POINTER(MhcScenario), c_void_p, POINTER(MhcRisk), c_void_p]
    return L


lib = _load()


def _check(code: int, where: str):
    if code != MHC_OK:
        raise MhcError(code, where, lib.mhc_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class CScenario:
    """A scenario marshalled into the C structs (keeps every host array alive)."""

    def __init__(self, sc):
        self.sc = sc
        self._keep: List[np.ndarray] = []
        objs = (MhcObject * len(sc.objects))()
        for q, o in enumerate(sc.objects):
            ga = np.ascontiguousarray(o.grid_a, np.float32)
            gb = np.ascontiguousarray(o.grid_b, np.float32)
            self._keep += [ga, gb]
            d = objs[q]
            d.kind, d.flags = int(o.kind), int(getattr(o, "flags", 0))
            d.length, d.width, d.radius = o.length, o.width, o.radius
            d.x0, d.y0, d.psi0, d.v0, d.v_max = o.x0, o.y0, o.psi0, o.v0, getattr(o, "v_max", 0.0)
            d.n_a, d.n_b = ga.size, gb.size
            d.grid_a = ga.ctypes.data_as(POINTER(c_float))
            d.grid_b = gb.ctypes.data_as(POINTER(c_float))
            if o.params is not None:
                pp = np.ascontiguousarray(o.params, np.float32)
                self._keep.append(pp)
                d.veh_params = pp.ctypes.data_as(POINTER(c_float))
            outline = getattr(o, "outline", None)
            if outline is not None:
                vv = np.ascontiguousarray(np.asarray(outline, np.float32).reshape(-1))
                self._keep.append(vv)
                d.n_vertices = vv.size // 2
                d.vertices = vv.ctypes.data_as(POINTER(c_float))
            paths = getattr(o, "paths", None)
            if paths is not None:
                pp = np.ascontiguousarray(np.asarray(paths, np.float32).reshape(-1))
                if pp.size != 9 * gb.size:
                    raise ValueError("paths must hold n_b x 3 sections x (x, y, psi)")
                self._keep.append(pp)
                d.paths = pp.ctypes.data_as(POINTER(c_float))
        self._objs = objs
        self.c = MhcScenario(len(sc.objects), objs, sc.tau, int(sc.n_steps), int(sc.substeps), int(sc.pair_mode),
                             int(sc.ego), int(sc.model))
        self.ref = ctypes.byref(self.c)


def as_c(sc) -> CScenario:
    return sc if isinstance(sc, CScenario) else CScenario(sc)


def lane_paths(dividers, x0: float, y0: float, psi0: float, v0: float, ego: bool = False) -> np.ndarray:
    """Paths of one vehicle from its lane dividers (mhc_lane_paths): dividers [n_div, 3, 2] in the
    vehicle frame, right to left.  Returns [n_paths, 3, 3] float32 (x, y, psi), ready for Obj.paths."""
    dv = np.ascontiguousarray(np.asarray(dividers, np.float32).reshape(-1))
    n = c_int32(0)
    fp = POINTER(c_float)
    _check(lib.mhc_lane_paths(dv.ctypes.data_as(fp), c_int32(dv.size // 6), c_float(x0), c_float(y0), c_float(psi0),
                              c_float(v0), c_int32(int(ego)), None, ctypes.byref(n)), "mhc_lane_paths")
    out = np.zeros((n.value, 3, 3), np.float32)
    _check(lib.mhc_lane_paths(dv.ctypes.data_as(fp), c_int32(dv.size // 6), c_float(x0), c_float(y0), c_float(psi0),
                              c_float(v0), c_int32(int(ego)), out.ctypes.data_as(fp), ctypes.byref(n)), "mhc_lane_paths")
    return out


def layout(sc) -> Dict[str, int]:
    cs = as_c(sc)
    nt, ne = c_int64(), c_int64()
    npair, he = c_int32(), c_int32()
    scratch = c_size_t()
    _check(lib.mhc_layout(cs.ref, ctypes.byref(nt), ctypes.byref(npair), ctypes.byref(ne), ctypes.byref(he),
                          ctypes.byref(scratch)), "mhc_layout")
    rb = c_size_t()
    _check(lib.mhc_run_bytes(cs.ref, ctypes.byref(rb)), "mhc_run_bytes")
    return dict(n_traj=nt.value, n_pairs=npair.value, n_entries=ne.value, h_ego=he.value, scratch=scratch.value,
                run_bytes=rb.value)


def pair_table(sc):
    cs = as_c(sc)
    n = layout(cs)["n_pairs"]
    pa, pb = np.zeros(n, np.int32), np.zeros(n, np.int32)
    poff = np.zeros(n + 1, np.int64)
    _check(lib.mhc_pair_table(cs.ref, pa.ctypes.data, pb.ctypes.data, poff.ctypes.data), "mhc_pair_table")
    return pa, pb, poff


class Context:
    """A library context whose arena is a torch-allocated device buffer."""

    def __init__(self, device: int = 0, arena_bytes: int = 256 << 20):
        self.device = device
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        h = c_void_p()
        _check(lib.mhc_create(ctypes.byref(h), device, self.arena.data_ptr(), self.arena.numel()), "mhc_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.mhc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        _check(lib.mhc_set_option(self.h, option, value), "mhc_set_option")

    def counters(self, reset: bool = False, stream=None):
        """(broad-phase tests executed, narrow-phase tests) since the last reset."""
        w = self.work(reset, stream)
        return w["executed"], w["narrow"]

    def work(self, reset: bool = False, stream=None) -> Dict[str, int]:
        """All collision work counters: executed broad-phase tests, narrow-phase tests and those by shape
        class (rect_rect, rect_disc, disc_disc, outline_outline, outline_disc)."""
        out = (c_uint64 * COUNTER_WORDS)()
        _check(lib.mhc_collision_counters(self.h, out, COUNTER_WORDS, int(reset), _stream(stream)),
               "mhc_collision_counters")
        return dict(zip(("executed", "narrow", "rect_rect", "rect_disc", "disc_disc", "outline_outline",
                         "outline_disc"),
                        (int(v) for v in out)))


    def profile(self, enable: bool = True):
        self.set_option(MHC_OPT_PROFILE, int(enable))

    def profile_read(self, reset: bool = False):
        ms = (c_double * 4)()
        n = (c_int64 * 4)()
        _check(lib.mhc_profile_read(self.h, ms, n, int(reset)), "mhc_profile_read")
        return {k: (float(ms[q]), int(n[q])) for q, k in enumerate(KERNEL_CLASSES)}

    def transfer_bytes(self):
        a, b = c_int64(), c_int64()
        _check(lib.mhc_transfer_bytes(self.h, ctypes.byref(a), ctypes.byref(b)), "mhc_transfer_bytes")
        return int(a.value), int(b.value)


def alloc_poses(sc, device="cuda") -> Dict[str, torch.Tensor]:
    n = layout(sc)["n_traj"] * int(sc.n_steps if not isinstance(sc, CScenario) else sc.sc.n_steps)
    return {k: torch.empty(n, dtype=torch.float32, device=device) for k in ("x", "y", "c", "s")}


def _poses_struct(p: Dict[str, torch.Tensor]) -> MhcPoses:
    return MhcPoses(p["x"].data_ptr(), p["y"].data_ptr(), p["c"].data_ptr(), p["s"].data_ptr())


def generate(ctx: Context, sc, poses=None, stream=None) -> Dict[str, torch.Tensor]:
    cs = as_c(sc)
    poses = alloc_poses(cs.sc) if poses is None else poses
    ps = _poses_struct(poses)
    _check(lib.mhc_generate_trajectories(ctx.h, cs.ref, ctypes.byref(ps), _stream(stream)),
           "mhc_generate_trajectories")
    return poses


def detect(ctx: Context, sc, poses, table=None, stream=None) -> torch.Tensor:
    cs = as_c(sc)
    if table is None:
        table = torch.empty(layout(cs)["n_entries"], dtype=torch.int16, device=poses["x"].device)
    ps = _poses_struct(poses)
    _check(lib.mhc_detect_collisions(ctx.h, cs.ref, ctypes.byref(ps), table.data_ptr(), _stream(stream)),
           "mhc_detect_collisions")
    return table


def risk_shapes(sc) -> Dict[str, tuple]:
    lay = layout(sc)
    s = sc.sc if isinstance(sc, CScenario) else sc
    np_, N, he, no = lay["n_pairs"], int(s.n_steps), lay["h_ego"], len(s.objects)
    return dict(count=((np_,), torch.int64), count_k=((np_, N), torch.int64), P=((np_,), torch.float64),
                H=((np_, N), torch.float64), naive=((he,), torch.float64), cond=((he,), torch.float64),
                indep=((he,), torch.float64), hits=((he,), torch.int32), attr_obj=((no,), torch.float64),
                attr_step=((N,), torch.float64), scalars=((4,), torch.float64), escape=((he,), torch.int32),
                n_escape=((1,), torch.int32))


def alloc_risk(sc, device="cuda", pin: bool = False) -> Dict[str, torch.Tensor]:
    out = {}
    for k, (shape, dt) in risk_shapes(sc).items():
        if device == "cpu":
            out[k] = torch.zeros(shape, dtype=dt, pin_memory=pin)
        else:
            out[k] = torch.zeros(shape, dtype=dt, device=device)
    return out


def _risk_struct(out: Dict[str, torch.Tensor]) -> MhcRisk:
    return MhcRisk(*[_ptr(out.get(f)) for f in RISK_FIELDS])


class CWeights:
    def __init__(self, weights: Optional[Sequence]):
        self.keep = []
        if weights is None:
            self.ptr = None
            return
        arr = (POINTER(c_float) * len(weights))()
        for q, w in enumerate(weights):
            if w is None:
                continue
            a = np.ascontiguousarray(w, np.float32)
            self.keep.append(a)
            arr[q] = a.ctypes.data_as(POINTER(c_float))
        self.arr = arr
        self.ptr = ctypes.cast(arr, c_void_p)


def assess(ctx: Context, sc, table: torch.Tensor, weights=None, out=None, stream=None) -> Dict[str, torch.Tensor]:
    cs = as_c(sc)
    out = alloc_risk(cs, device=table.device) if out is None else out
    rs = _risk_struct(out)
    w = weights if isinstance(weights, CWeights) else CWeights(weights)
    _check(lib.mhc_assess_risk(ctx.h, cs.ref, table.data_ptr(), w.ptr, ctypes.byref(rs), _stream(stream)),
           "mhc_assess_risk")
    return out


def autotune(ctx: Context, sc, poses, table=None, fused: bool = True, stream=None):
    """Times the collision kernel's layouts (and culling on / off) on this scenario, in the fused path of
    evaluate / run (fused=True) or of detect; later calls on `ctx` use the fastest for its size class.
    Returns (variant, cull)."""
    cs = as_c(sc)
    if table is None:
        table = torch.empty(layout(cs)["n_entries"], dtype=torch.int16, device=poses["x"].device)
    ps = _poses_struct(poses)
    v, c = c_int32(), c_int32()
    _check(lib.mhc_autotune(ctx.h, cs.ref, ctypes.byref(ps), table.data_ptr(), int(fused), ctypes.byref(v),
                            ctypes.byref(c), _stream(stream)), "mhc_autotune")
    return v.value, c.value


def evaluate(ctx: Context, sc, poses=None, table=None, weights=None, out=None, stream=None):
    """The whole method on device buffers in one call (fused collision + risk accumulation).
    Returns (poses, table, risk outputs)."""
    cs = as_c(sc)
    poses = alloc_poses(cs.sc) if poses is None else poses
    if table is None:
        table = torch.empty(layout(cs)["n_entries"], dtype=torch.int16, device=poses["x"].device)
    out = alloc_risk(cs, device=table.device) if out is None else out
    ps = _poses_struct(poses)
    rs = _risk_struct(out)
    w = weights if isinstance(weights, CWeights) else CWeights(weights)
    _check(lib.mhc_evaluate(ctx.h, cs.ref, w.ptr, ctypes.byref(ps), table.data_ptr(), ctypes.byref(rs),
                            _stream(stream)), "mhc_evaluate")
    return poses, table, out


def run(ctx: Context, sc, weights=None, out=None, stream=None, out_struct=None) -> Dict[str, torch.Tensor]:
    """Host inputs -> host risk outputs through mhc_run (synchronises the stream).  `out_struct` may carry
    the prebuilt MhcRisk of `out` (risk_struct(out)) to skip rebuilding it on every call."""
    cs = as_c(sc)
    out = alloc_risk(cs, device="cpu", pin=True) if out is None else out
    rs = out_struct if out_struct is not None else _risk_struct(out)
    wptr = None if weights is None else (weights if isinstance(weights, CWeights) else CWeights(weights)).ptr
    _check(lib.mhc_run(ctx.h, cs.ref, wptr, ctypes.byref(rs), _stream(stream)), "mhc_run")
    return out


def risk_struct(out: Dict[str, torch.Tensor]) -> MhcRisk:
    """The C struct of a dict of risk output buffers (for repeated calls)."""
    return _risk_struct(out)


def poses_by_trajectory(sc, plane: torch.Tensor) -> np.ndarray:
    """Device pose plane ([object][step][hypothesis]) as a host array [n_traj, N] (trajectory-major)."""
    s = sc.sc if isinstance(sc, CScenario) else sc
    N = int(s.n_steps)
    host = plane.detach().cpu().numpy()
    out, base = [], 0
    for o in s.objects:
        h = int(np.asarray(o.grid_a).size * np.asarray(o.grid_b).size)
        out.append(host[base: base + N * h].reshape(N, h).T)
        base += N * h
    return np.concatenate(out, axis=0)


def poses_to_device(sc, arr: np.ndarray, device="cuda") -> torch.Tensor:
    """Inverse of poses_by_trajectory: a [n_traj, N] host array into one device pose plane."""
    s = sc.sc if isinstance(sc, CScenario) else sc
    parts, t = [], 0
    for o in s.objects:
        h = int(np.asarray(o.grid_a).size * np.asarray(o.grid_b).size)
        parts.append(np.ascontiguousarray(arr[t: t + h].T).reshape(-1))
        t += h
    return torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(device)


# ---------------------------------------------------------------------------------------------------------
# batches of scenarios

class CBatch:
    """A list of scenarios marshalled into one contiguous C array (keeps every host array alive)."""

    def __init__(self, scenarios):
        self.items = [as_c(sc) for sc in scenarios]
        if not self.items:
            raise ValueError("a batch needs at least one scenario")
        arr = (MhcScenario * len(self.items))()
        for q, cs in enumerate(self.items):
            arr[q] = cs.c
        self.arr = arr
        self.n = len(self.items)
        self.ref = ctypes.cast(arr, POINTER(MhcScenario))

    @property
    def scenarios(self):
        return [cs.sc for cs in self.items]


def as_batch(scenarios) -> CBatch:
    return scenarios if isinstance(scenarios, CBatch) else CBatch(scenarios)


SLICE_FIELDS = [f for f, _ in MhcBatchSlice._fields_]


def batch_layout(scenarios):
    """(info dict, slices: list of dicts) of a batch, from mhc_batch_layout."""
    cb = as_batch(scenarios)
    info = MhcBatchInfo()
    sl = (MhcBatchSlice * cb.n)()
    _check(lib.mhc_batch_layout(cb.ref, cb.n, ctypes.byref(info), ctypes.cast(sl, c_void_p)), "mhc_batch_layout")
    d = {f: int(getattr(info, f)) for f, _ in MhcBatchInfo._fields_}
    return d, [{f: int(getattr(x, f)) for f in SLICE_FIELDS} for x in sl]


def batch_pair_table(scenarios):
    cb = as_batch(scenarios)
    n = batch_layout(cb)[0]["n_pairs"]
    pa, pb = np.zeros(n, np.int32), np.zeros(n, np.int32)
    poff = np.zeros(n + 1, np.int64)
    _check(lib.mhc_batch_pair_table(cb.ref, cb.n, pa.ctypes.data, pb.ctypes.data, poff.ctypes.data),
           "mhc_batch_pair_table")
    return pa, pb, poff


def batch_risk_shapes(info) -> Dict[str, tuple]:
    np_, nk, he, no, ns = info["n_pairs"], info["n_step_entries"], info["h_ego"], info["n_objects"], info["n_scenarios"]
    return dict(count=((np_,), torch.int64), count_k=((nk,), torch.int64), P=((np_,), torch.float64),
                H=((nk,), torch.float64), naive=((he,), torch.float64), cond=((he,), torch.float64),
                indep=((he,), torch.float64), hits=((he,), torch.int32), attr_obj=((no,), torch.float64),
                attr_step=((info["n_scen_steps"],), torch.float64), scalars=((4 * ns,), torch.float64),
                escape=((he,), torch.int32), n_escape=((ns,), torch.int32))


def alloc_batch(info, device="cuda"):
    """(poses, table, risk outputs) device buffers of a batch."""
    poses = {k: torch.empty(info["n_poses"], dtype=torch.float32, device=device) for k in ("x", "y", "c", "s")}
    table = torch.empty(info["n_entries"], dtype=torch.int16, device=device)
    out = {k: torch.zeros(shape, dtype=dt, device=device) for k, (shape, dt) in batch_risk_shapes(info).items()}
    return poses, table, out


def scenario_view(out: Dict[str, torch.Tensor], sl: dict) -> Dict[str, torch.Tensor]:
    """Scenario `sl`'s part (a slice from batch_slices) of batch risk outputs, shaped like the
    single-scenario outputs."""
    p0, npair, N = sl["pair0"], sl["n_pairs"], sl["n_steps"]
    k0, e0, he, q = sl["step_entry0"], sl["ego0"], sl["h_ego"], sl["index"]
    return dict(count=out["count"][p0: p0 + npair], count_k=out["count_k"][k0: k0 + npair * N].view(npair, N),
                P=out["P"][p0: p0 + npair], H=out["H"][k0: k0 + npair * N].view(npair, N),
                naive=out["naive"][e0: e0 + he], cond=out["cond"][e0: e0 + he], indep=out["indep"][e0: e0 + he],
                hits=out["hits"][e0: e0 + he], attr_obj=out["attr_obj"][sl["obj0"]: sl["obj0"] + sl["n_objects"]],
                attr_step=out["attr_step"][sl["step0"]: sl["step0"] + N], scalars=out["scalars"][4 * q: 4 * q + 4],
                escape=out["escape"][e0: e0 + he], n_escape=out["n_escape"][q: q + 1])


def batch_slices(scenarios):
    """Per-scenario slices with the scenario's index and EGO hypothesis count added."""
    cb = as_batch(scenarios)
    info, sls = batch_layout(cb)
    for q, (sl, sc) in enumerate(zip(sls, cb.scenarios)):
        sl["index"] = q
        e = sc.objects[sc.ego]
        sl["h_ego"] = int(np.asarray(e.grid_a).size * np.asarray(e.grid_b).size)
    return info, sls


def evaluate_batch(ctx: Context, scenarios, poses=None, table=None, weights=None, out=None, stream=None):
    """The whole method over a batch in one launch sequence.  Returns (poses, table, risk outputs)."""
    cb = as_batch(scenarios)
    info, _ = batch_layout(cb)
    if poses is None or table is None or out is None:
        p2, t2, o2 = alloc_batch(info)
        poses = p2 if poses is None else poses
        table = t2 if table is None else table
        out = o2 if out is None else out
    ps = _poses_struct(poses)
    rs = _risk_struct(out)
    w = weights if isinstance(weights, CWeights) else CWeights(weights)
    _check(lib.mhc_evaluate_batch(ctx.h, cb.ref, cb.n, w.ptr, ctypes.byref(ps), table.data_ptr(), ctypes.byref(rs),
                                  _stream(stream)), "mhc_evaluate_batch")
    return poses, table, out


def autotune_batch(ctx: Context, scenarios, poses, table, fused: bool = True, stream=None):
    cb = as_batch(scenarios)
    ps = _poses_struct(poses)
    v, c = c_int32(), c_int32()
    _check(lib.mhc_autotune_batch(ctx.h, cb.ref, cb.n, ctypes.byref(ps), table.data_ptr(), int(fused),
                                  ctypes.byref(v), ctypes.byref(c), _stream(stream)), "mhc_autotune_batch")
    return v.value, c.value


class Plan:
    """A batch laid out once (descriptors in a torch-owned scratch buffer) and, with graph=True, its launch
    sequence captured as a CUDA graph; launch() replays it, update() swaps in scenarios of the same
    structure (new initial states)."""

    def __init__(self, ctx: Context, scenarios, weights=None, graph: bool = True, buffers=None, pipeline: bool = False):
        self.ctx = ctx
        self.batch = as_batch(scenarios)
        self.info, _ = batch_layout(self.batch)
        dev = f"cuda:{ctx.device}"
        self.poses, self.table, self.out = alloc_batch(self.info, dev) if buffers is None else buffers
        self.scratch = torch.empty(int(self.info["plan_bytes"]) + 256, dtype=torch.uint8, device=dev)
        base = self.scratch.data_ptr()
        off = (-base) % 256
        self._w = weights if isinstance(weights, CWeights) else CWeights(weights)
        ps = _poses_struct(self.poses)
        rs = _risk_struct(self.out)
        h = c_void_p()
        _check(lib.mhc_plan_create(ctx.h, self.batch.ref, self.batch.n, self._w.ptr, ctypes.byref(ps),
                                   self.table.data_ptr(), ctypes.byref(rs), base + off,
                                   self.scratch.numel() - off,
                                   (MHC_PLAN_GRAPH if graph else 0) | (MHC_PLAN_PIPELINE if pipeline else 0),
                                   ctypes.byref(h)),
               "mhc_plan_create")
        self.h = h

    def update(self, scenarios):
        cb = as_batch(scenarios)
        _check(lib.mhc_plan_update(self.h, cb.ref, cb.n), "mhc_plan_update")
        self.batch = cb

    def launch(self, stream=None):
        _check(lib.mhc_plan_launch(self.h, _stream(stream)), "mhc_plan_launch")
        return self.poses, self.table, self.out

    def close(self):
        if getattr(self, "h", None):
            lib.mhc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------------------------
# serving loop

class Server:
    """Continuous batching on a context (mhc_serve_start ... mhc_serve_stop) with a torch-owned device pool."""

    def __init__(self, ctx: Context, pool_bytes: int, small_slots=3, large_slots=1, max_batch=64, max_queue=4096,
                 small_tests=1 << 31, max_batch_tests=1 << 34):
        self.ctx = ctx
        self.pool = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=f"cuda:{ctx.device}")
        base = self.pool.data_ptr()
        off = (-base) % 256
        self.cfg = MhcServeConfig(small_slots, large_slots, max_batch, max_queue, small_tests, max_batch_tests)
        _check(lib.mhc_serve_start(ctx.h, base + off, int(pool_bytes), ctypes.byref(self.cfg)), "mhc_serve_start")
        self.running = True
        self._keep = {}

    def submit(self, sc, weights=None) -> int:
        cs = as_c(sc)
        w = weights if isinstance(weights, CWeights) else CWeights(weights)
        t = c_uint64()
        _check(lib.mhc_submit(self.ctx.h, cs.ref, w.ptr, ctypes.byref(t)), "mhc_submit")
        return int(t.value)

    def poll(self, ticket: int, out=None, timeout_us: int = -1) -> bool:
        """True when done (outputs copied into `out`, host tensors of the single-scenario shapes), False if
        still pending after timeout_us."""
        rs = _risk_struct(out) if out is not None else None
        code = lib.mhc_poll(self.ctx.h, ticket, ctypes.byref(rs) if rs is not None else None, int(timeout_us))
        if code == MHC_PENDING:
            return False
        _check(code, "mhc_poll")
        return True

    def release(self, ticket: int):
        _check(lib.mhc_release(self.ctx.h, ticket), "mhc_release")

    def times(self, ticket: int):
        ns = (c_int64 * 3)()
        bs = c_int32()
        _check(lib.mhc_request_times(self.ctx.h, ticket, ns, ctypes.byref(bs)), "mhc_request_times")
        return (int(ns[0]), int(ns[1]), int(ns[2])), int(bs.value)

    def buffers(self, ticket: int):
        """Raw device addresses of a finished request: ({x, y, c, s}, table, MhcRisk of device pointers)."""
        ps = MhcPoses()
        tb = c_void_p()
        rs = MhcRisk()
        _check(lib.mhc_request_buffers(self.ctx.h, ticket, ctypes.byref(ps), ctypes.byref(tb), ctypes.byref(rs)),
               "mhc_request_buffers")
        return {k: getattr(ps, k) for k in ("x", "y", "c", "s")}, tb.value, rs

    def stats(self):
        st = MhcServeStats()
        _check(lib.mhc_serve_stats_read(self.ctx.h, ctypes.byref(st)), "mhc_serve_stats_read")
        return {f: int(getattr(st, f)) for f, _ in MhcServeStats._fields_}

    def pause(self, paused: bool = True):
        _check(lib.mhc_serve_pause(self.ctx.h, int(paused)), "mhc_serve_pause")

    def stop(self):
        if self.running:
            _check(lib.mhc_serve_stop(self.ctx.h), "mhc_serve_stop")
            self.running = False

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class _DevArray:
    _TYPESTR = {torch.float32: "<f4", torch.float64: "<f8", torch.int16: "<i2", torch.int32: "<i4",
                torch.int64: "<i8"}

    def __init__(self, addr: int, n: int, dtype):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": self._TYPESTR[dtype],
                                         "data": (int(addr), False), "version": 3, "strides": None}


def device_view(addr: int, n: int, dtype) -> torch.Tensor:
    """A torch tensor over n elements of library-owned device memory at addr (no copy; valid as long as
    that memory is, e.g. until mhc_release of a served request)."""
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DevArray(addr, n, dtype), device="cuda")


class Pool:
    """The serving loop's first-fit allocator on its own (host offsets)."""

    def __init__(self, nbytes: int):
        h = c_void_p()
        _check(lib.mhc_pool_create(int(nbytes), ctypes.byref(h)), "mhc_pool_create")
        self.h = h

    def alloc(self, nbytes: int) -> int:
        off = c_size_t()
        _check(lib.mhc_pool_alloc(self.h, int(nbytes), ctypes.byref(off)), "mhc_pool_alloc")
        return int(off.value)

    def free(self, offset: int):
        _check(lib.mhc_pool_free(self.h, int(offset)), "mhc_pool_free")

    def info(self):
        f, l, n = c_size_t(), c_size_t(), c_int32()
        _check(lib.mhc_pool_info(self.h, ctypes.byref(f), ctypes.byref(l), ctypes.byref(n)), "mhc_pool_info")
        return int(f.value), int(l.value), int(n.value)

    def close(self):
        if getattr(self, "h", None):
            lib.mhc_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
