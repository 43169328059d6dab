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
                ("grid_b", POINTER(c_float)), ("veh_params", POINTER(c_float))]


class MhcScenario(ctypes.Structure):
    _fields_ = [("n_objects", c_int32), ("objects", POINTER(MhcObject)), ("tau", c_float), ("n_steps", c_int32),
                ("substeps", c_int32), ("pair_mode", c_int32), ("ego", c_int32), ("model", c_int32)]


class MhcPoses(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("c", c_void_p), ("s", c_void_p)]


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
    L.mhc_collision_counters.argtypes = [c_void_p, POINTER(c_uint64), c_int, c_void_p]
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
        self._objs = objs
        self.c = MhcScenario(len(sc.objects), objs, sc.tau, int(sc.n_steps), int(sc.substeps), int(sc.pair_mode),
                             int(sc.ego), int(sc.model))
        self.ref = ctypes.byref(self.c)


def as_c(sc) -> CScenario:
    return sc if isinstance(sc, CScenario) else CScenario(sc)


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
        out = (c_uint64 * 2)()
        _check(lib.mhc_collision_counters(self.h, out, int(reset), _stream(stream)), "mhc_collision_counters")
        return int(out[0]), int(out[1])


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


def run(ctx: Context, sc, weights=None, out=None, stream=None) -> Dict[str, torch.Tensor]:
    """Host inputs -> host risk outputs through mhc_run (synchronises the stream)."""
    cs = as_c(sc)
    out = alloc_risk(cs, device="cpu", pin=True) if out is None else out
    rs = _risk_struct(out)
    w = weights if isinstance(weights, CWeights) else CWeights(weights)
    _check(lib.mhc_run(ctx.h, cs.ref, w.ptr, ctypes.byref(rs), _stream(stream)), "mhc_run")
    return out


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
