#!/usr/bin/env python
"""Benchmark of the multi-hypothesis collision-criticality hot path on GB300.

One step = the whole hot path on one 11-object intersection (7 cars x 441 hypotheses + 4 pedestrians
x 121, 30 steps of 0.1 s, every object pair: 1.70e8 pose-pair tests): trajectory generation, collision
recognition and risk assessment, all through the C ABI, inputs resident in HBM.  The L2 cache is
flushed (256 MiB write) before every timed step, outside the step's CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mhc|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU) every rank runs its own
scenario replica (independent placements, weak scaling) and the time is the maximum over ranks.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time
from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pose-pair tests/s"
UNIT = "tests/s"
# committed ncu summaries of the collision stage on the benchmark scene, per collision layout
PROFILE_NOTES = {5: os.path.join(ROOT, "profiles", "collide_tile_kernel_intersection11.md"),
                 6: os.path.join(ROOT, "profiles", "items_kernels_intersection11.md"),
                 7: os.path.join(ROOT, "profiles", "block_kernel_intersection11.md")}
COLLIDE_SRC = [os.path.join(ROOT, "paper_2005_06773_gb300", "csrc", f) for f in ("collide.cu", "mhc_internal.cuh")]
# Algorithmic lane instructions (FP32 pipe + ALU) per unit of collision work:
#   broad-phase test: dx, dy (2 FADD), d^2 (FMUL + FFMA), compare = 4 FP32 + 1 ALU = 5;
#   narrow-phase test by shape pair: rectangle-rectangle separating axes (relative rotation 4, frame
#   transforms 8, projected radii 8, abs 4, compares 4) = 24 FP32 + 8 ALU = 32; rectangle-disc (frame
#   transform 4, clamps 4, distance 2, compare) = 10 FP32 + 6 ALU = 16; disc-disc (dx, dy, d^2, compare) = 5;
#   convex outlines of n vertices: outline-outline 2 n^2 + 16 n (each edge against every vertex of the
#   other, both ways), outline-disc 5 n + 4.
OPS_PER_BROAD_TEST = 5.0
OPS_PER_NARROW = {"rect_rect": 32.0, "rect_disc": 16.0, "disc_disc": 5.0}
FP32_LANES_PER_SM = 128


def collide_ops(work: dict, n_vertices: float = 0.0) -> float:
    """Algorithmic lane instructions of the collision work counted by the kernels (mhc_collision_counters)."""
    nv = float(n_vertices)
    ops = OPS_PER_BROAD_TEST * work["executed"]
    ops += sum(c * work[k] for k, c in OPS_PER_NARROW.items())
    ops += (2 * nv * nv + 16 * nv) * work.get("outline_outline", 0) + (5 * nv + 4) * work.get("outline_disc", 0)
    return ops


def mean_vertices(sc) -> float:
    nv = [len(o.outline) for o in sc.objects if getattr(o, "outline", None) is not None]
    return sum(nv) / len(nv) if nv else 0.0
# the kernel behind each collision layout (MHC_OPT_COLLIDE_VARIANT)
COLLIDE_KERNELS = {1: "collide_kernel<256, 4, 4, 16>", 2: "collide_kernel<64, 8, 8, 8>", 3: "collide_warp_kernel<4, 8>",
                   4: "collide_tile_kernel<4, 64>", 5: "collide_tile_kernel<1, 32>",
                   6: "items_list_kernel + items_kernel + items_table_kernel (per-launch figures average the three)",
                   7: "block_kernel<4>", 8: "block_list_kernel + block_rec_kernel<4> (per-launch figures average the two)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mhc", choices=["mhc", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the stress32 / paper_s2 / batch / serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="window of the serving measurement at 2000/s")
    ap.add_argument("--serve-rates", default="4000,8000",
                    help="further offered rates (requests/s) of the serving sweep, 2 s windows each ('' for none)")
    ap.add_argument("--collide-variant", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6, 7, 8],
                    help="collision kernel layout; 0 = chosen by mhc_autotune in the set-up (profiling fixes one)")
    ap.add_argument("--workload", default="intersection11", choices=sorted(WORKLOADS),
                    help="the timed workload (the default is the benchmark's; the others serve profiling)")
    return ap.parse_args()


WORKLOADS = {
    "intersection11": "intersection11: 7 cars (4.5x1.8 m, 441 hypotheses = 21 accel x 21 steer) + 4 pedestrians "
                      "(r 0.4 m, 121 = 11 speeds x 11 headings), 30 steps of 0.1 s (5 sub-steps), all 55 object pairs",
    "stress32": "stress32: 32 cars x 2048 hypotheses (64 accel x 32 steer), 50 steps of 0.1 s, 496 object pairs",
    "stress12": "stress12: 12 cars x 2048 hypotheses (64 accel x 32 steer), 50 steps of 0.1 s, 66 object pairs",
    "paper_s2": "paper_s2: EGO 2058 (6 x 343) + 10 COs x 42 (6 x 7), 100 steps of 20 ms, EGO-only pairs",
    "outline11": "outline11: intersection11 with every car drawn as a convex octagon (4.5x1.8 m, corners cut 0.35 m)",
    "paths11": "paths11: intersection11 with every car following lane paths under the lateral controller "
               "(441 hypotheses = 63 accel x 7 paths)",
}
WORKLOAD = "intersection11"


def workload(rank: int = 0):
    from paper_2005_06773_gb300 import scenarios as S
    if WORKLOAD == "stress32":
        return S.stress32(4 + rank)
    if WORKLOAD == "stress12":
        return S.stress32(4 + rank, n_cars=12)
    if WORKLOAD == "paper_s2":
        return S.paper_s1s2(10, 6, seed=6 + rank)
    if WORKLOAD == "outline11":
        return S.with_outlines(S.intersection11(replica_seed(rank)), cut=0.35)
    if WORKLOAD == "paths11":
        return S.with_lane_paths(S.intersection11(replica_seed(rank), n_acc=63))
    return S.intersection11(replica_seed(rank))


def config_of(sc, rank0_seed=2):
    return {
        "workload": WORKLOADS[WORKLOAD],
        "seed": rank0_seed,
        "tests_per_step": sc.n_tests(),
        "trajectory_pairs_per_step": sc.n_traj_pairs(),
        "hypotheses": sum(sc.hyp_counts),
        "l2": "flushed before every timed step (256 MiB write, outside the step's events)",
    }


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def collide_code_sha256() -> str:
    """Hash of the collision kernels' code: collide.cu and the descriptor header with `//` comments and
    blank lines removed (neither file has `//` inside a string), so that a comment edit keeps a profile."""
    h = hashlib.sha256()
    for path in COLLIDE_SRC:
        for line in open(path, encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def traffic_from_profile(variant: int):
    """DRAM bytes per collide launch from the committed ncu summary, if it was taken on this code and
    this collision layout."""
    if variant not in PROFILE_NOTES:
        return None
    try:
        text = open(PROFILE_NOTES[variant]).read()
        sha = collide_code_sha256()
    except OSError:
        return None
    m_sha = re.search(r"collide_code_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_v = re.search(r"collide_variant:\s*([0-9]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha or not m_v or int(m_v.group(1)) != variant:
        return None
    return float(m_b.group(1))


class NvmlClocks:
    """SM clock, its maximum, power and clock-event reasons polled through NVML (read-only queries, driver
    library via ctypes) every `period_s` in a thread while the timed region runs, so that even a region of a
    few milliseconds has samples inside it."""
    BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, uuid: Optional[str], index: int, period_s: float = 0.002):
        import ctypes as C
        import threading
        self.C, self.period, self.rows, self.stop_flag = C, period_s, [], threading.Event()
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.lib, self.h = lib, C.c_void_p()
        found = False
        for u in ([uuid, "GPU-" + uuid] if uuid else []):
            if lib.nvmlDeviceGetHandleByUUID(C.c_char_p(u.encode()), C.byref(self.h)) == 0:
                found = True
                break
        if not found and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = C.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(self.h, C.c_int(1), C.byref(mx))     # NVML_CLOCK_SM
        self.max_mhz = float(mx.value)
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _sample(self):
        C, lib = self.C, self.lib
        mhz, mw, rs = C.c_uint(0), C.c_uint(0), C.c_ulonglong(0)
        if lib.nvmlDeviceGetClockInfo(self.h, C.c_int(1), C.byref(mhz)) != 0:
            return
        lib.nvmlDeviceGetPowerUsage(self.h, C.byref(mw))
        self.reasons_fn(self.h, C.byref(rs))
        self.rows.append((float(mhz.value), mw.value / 1e3, int(rs.value)))

    def _run(self):
        while not self.stop_flag.is_set():
            self._sample()
            time.sleep(self.period)

    def start(self):
        self._sample()
        self.thread.start()

    def stop(self):
        self.stop_flag.set()
        self.thread.join(timeout=5)
        self._sample()
        sm = [r[0] for r in self.rows]
        reasons = sorted({name for r in self.rows for bit, name in self.BITS.items() if r[2] & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(self.rows), "power_w_max": max((r[1] for r in self.rows), default=None),
                "source": f"NVML every {self.period * 1e3:g} ms during the timed region"}


class Clocks:
    """nvidia-smi sampler (200 ms) around the timed region: the fallback when NVML cannot be loaded."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self.tmp.close()
            os.unlink(self.tmp.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.tmp.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = {5: "hw_slowdown", 6: "hw_thermal_slowdown", 7: "sw_thermal_slowdown", 8: "sw_power_cap"}
        for r in rows:
            for col, name in names.items():
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if re.match(r"^[0-9.]+$", r[3])), default=None)}


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    return v[min(len(v) - 1, int(math.ceil(q / 100.0 * len(v))) - 1)]


def cpu_baseline(sc, budget_s: float):
    """The FP64 oracle, as it stands, on whole passes of the same scene (single thread)."""
    from oracle import oracle
    oracle.build()
    passes, t0 = 0, time.perf_counter()
    while True:
        out = oracle.run(sc)
        passes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    assert out["table"].size == sc.n_traj_pairs()
    return {"value": passes * sc.n_tests() / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{passes} full pass(es) of the 11-object scene (generate + table + risk, "
                      f"{sc.n_tests():.3e} tests each) in {dt:.1f} s on 1 host thread",
            "seconds": dt}, out


_ORACLE_STATE = {}


def _oracle_pool_init(root, sc, poses):
    sys.path.insert(0, root)
    from oracle import oracle
    _ORACLE_STATE.update(oracle=oracle, sc=sc, poses=poses)


def _oracle_pool_task(chunk):
    o = _ORACLE_STATE["oracle"]
    return int((o.first_steps(_ORACLE_STATE["sc"], _ORACLE_STATE["poses"], *chunk) >= 0).sum())


def _oracle_batch_init(root, scens):
    sys.path.insert(0, root)
    from oracle import oracle
    _ORACLE_STATE.update(oracle=oracle, scens=scens, poses=[oracle.generate(sc) for sc in scens])


def _oracle_batch_task(chunk):
    o = _ORACLE_STATE["oracle"]
    q = chunk[0]
    return int((o.first_steps(_ORACLE_STATE["scens"][q], _ORACLE_STATE["poses"][q], *chunk[1:]) >= 0).sum())


def cpu_oracle_batch(batch, target_tests: float = 1e8, n_scen: int = 16, seed: int = 11):
    """The oracle (its functions unchanged) on a fixed sample of the uneven batch: n_scen scenarios drawn
    by their share of the batch's pose tests, their trajectories generated, then random trajectory pairs of
    those scenarios (drawn by pair size) up to about target_tests pose tests, on one host thread and on
    every core (spawned workers generate the same scenarios); the rates extrapolated to the whole batch."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    from oracle import oracle
    oracle.build()
    tests_s = np.array([sc.n_tests() for sc in batch], dtype=np.float64)
    rng = np.random.default_rng(seed)
    pick = sorted(rng.choice(len(batch), size=min(n_scen, len(batch)), replace=False, p=tests_s / tests_s.sum()).tolist())
    scens = [batch[q] for q in pick]
    t0 = time.perf_counter()
    poses = [oracle.generate(sc) for sc in scens]
    t_gen = time.perf_counter() - t0
    hyps = sum(int(oracle.traj_offsets(sc)[-1]) for sc in scens)
    share = tests_s[pick] / tests_s[pick].sum()
    chunks, tests = [], 0
    for q, sc in enumerate(scens):
        off = oracle.traj_offsets(sc)
        pairs = oracle.pair_list(sc)
        h = np.diff(off)
        sizes = np.array([h[a] * h[b] for a, b in pairs], dtype=np.float64)
        n = max(1, int(target_tests * share[q] / sc.n_steps))
        k = rng.choice(len(pairs), size=n, p=sizes / sizes.sum())
        oa = np.array([pairs[x][0] for x in k]); ob = np.array([pairs[x][1] for x in k])
        ta = off[oa] + (rng.random(n) * h[oa]).astype(np.int64)
        tb = off[ob] + (rng.random(n) * h[ob]).astype(np.int64)
        tests += n * sc.n_steps
        for s in np.array_split(np.arange(n), max(1, n // 100_000)):
            chunks.append((q, oa[s], ta[s], ob[s], tb[s]))
    t0 = time.perf_counter()
    for c in chunks:
        oracle.first_steps(scens[c[0]], poses[c[0]], *c[1:])
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                initializer=_oracle_batch_init, initargs=(ROOT, scens)) as ex:
        list(ex.map(_oracle_batch_task, chunks[:cores]))          # workers started, scenarios generated
        t0 = time.perf_counter()
        list(ex.map(_oracle_batch_task, chunks))
        tn = time.perf_counter() - t0
    all_tests = float(tests_s.sum())
    all_hyps = sum(sc_h for sc_h in (sum(o.n_hyp for o in sc.objects) for sc in batch))
    gen_s = t_gen * all_hyps / max(hyps, 1)
    return {"tests": tests, "sample": f"{len(scens)} of {len(batch)} scenarios (drawn by their share of the tests), "
                                      f"{sum(len(c[1]) for c in chunks)} random trajectory pairs (first-collision steps only)",
            "one_thread_tests_per_s": tests / t1, "all_cores_tests_per_s": tests / tn, "cores": cores,
            "batch_tests": all_tests, "generation_s_one_thread": gen_s,
            "batch_s_one_thread": all_tests * t1 / tests + gen_s, "batch_s_all_cores": all_tests * tn / tests + gen_s / cores,
            "cpu": cpu_model()}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_oracle_cores(sc, n_pairs: int, seed: int = 7):
    """The oracle's first-collision steps (its functions unchanged) on n_pairs random trajectory pairs of the
    scene (or all of them), on one host thread and on every core (a spawn-started process pool over slices
    of the pairs): pose tests per second each way."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    from oracle import oracle
    oracle.build()
    poses = oracle.generate(sc)
    off = oracle.traj_offsets(sc)
    pairs = oracle.pair_list(sc)
    h = np.diff(off)
    sizes = np.array([h[a] * h[b] for a, b in pairs], dtype=np.float64)
    rng = np.random.default_rng(seed)
    if n_pairs >= sizes.sum():           # every trajectory pair of the scene
        oa, ta, ob, tb = [], [], [], []
        for a, b in pairs:
            i, j = np.meshgrid(np.arange(h[a]), np.arange(h[b]), indexing="ij")
            oa.append(np.full(i.size, a)); ob.append(np.full(i.size, b))
            ta.append(off[a] + i.ravel()); tb.append(off[b] + j.ravel())
        oa, ta, ob, tb = (np.concatenate(v) for v in (oa, ta, ob, tb))
        what = f"all {oa.size} trajectory pairs"
    else:
        q = rng.choice(len(pairs), size=n_pairs, p=sizes / sizes.sum())
        oa = np.array([pairs[x][0] for x in q]); ob = np.array([pairs[x][1] for x in q])
        ta = off[oa] + (rng.random(n_pairs) * h[oa]).astype(np.int64)
        tb = off[ob] + (rng.random(n_pairs) * h[ob]).astype(np.int64)
        what = f"{n_pairs} random trajectory pairs"
    tests = oa.size * sc.n_steps
    t0 = time.perf_counter()
    oracle.first_steps(sc, poses, oa, ta, ob, tb)
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    chunks = [(oa[s], ta[s], ob[s], tb[s]) for s in np.array_split(np.arange(oa.size), 4 * cores)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                initializer=_oracle_pool_init, initargs=(ROOT, sc, poses)) as ex:
        list(ex.map(_oracle_pool_task, chunks[:cores]))          # workers started and warm
        t0 = time.perf_counter()
        list(ex.map(_oracle_pool_task, chunks))
        tn = time.perf_counter() - t0
    return {"tests": tests, "sample": what + f" x {sc.n_steps} steps (first-collision steps only)",
            "one_thread_tests_per_s": tests / t1, "all_cores_tests_per_s": tests / tn, "cores": cores,
            "cpu": cpu_model()}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, each step a bounded random sample of the
    scene's trajectory pairs (plus the full trajectory generation)."""
    import numpy as np
    from oracle import oracle
    from paper_2005_06773_gb300 import scenarios as S
    oracle.build()
    sc = workload(0)
    off = oracle.traj_offsets(sc)
    pairs = oracle.pair_list(sc)
    h = np.diff(off)
    sizes = np.array([h[a] * h[b] for a, b in pairs], dtype=np.float64)
    rng = np.random.default_rng(12345)

    def draw(n):
        q = rng.choice(len(pairs), size=n, p=sizes / sizes.sum())
        pa = np.array([pairs[x][0] for x in q]); pb = np.array([pairs[x][1] for x in q])
        i = (rng.random(n) * h[pa]).astype(np.int64); j = (rng.random(n) * h[pb]).astype(np.int64)
        return pa, off[pa] + i, pb, off[pb] + j

    poses = oracle.generate(sc)
    t0 = time.perf_counter()
    oracle.first_steps(sc, poses, *draw(20000))
    rate = 20000 / max(time.perf_counter() - t0, 1e-6)          # trajectory pairs per second
    per_step = max(0.05, 120.0 / max(1, args.steps + args.warmup))
    n = int(max(2000, min(rate * per_step, sc.n_traj_pairs())))
    samples = [draw(n) for _ in range(args.steps + args.warmup)]
    times = []
    for s in range(args.steps + args.warmup):
        t = time.perf_counter()
        p = oracle.generate(sc)
        oracle.first_steps(sc, p, *samples[s])
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    tests = n * sc.n_steps
    total = sum(times)
    value = tests * len(times) / total
    sample = (f"each step: full trajectory generation + first-collision steps of {n} random trajectory pairs "
              f"({tests:.3e} pose tests) of the 11-object scene, 1 host thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(sc),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def measure_workload(mhc, torch, sc, dev, steps, flush, peak):
    """Device time of the whole hot path (mhc_evaluate) on one more workload, L2 flushed per step."""
    cs = mhc.as_c(sc)
    lay = mhc.layout(cs)
    ctx = mhc.Context(dev.index or 0, 512 << 20)
    poses = mhc.alloc_poses(sc, dev)
    table = torch.empty(lay["n_entries"], dtype=torch.int16, device=dev)
    risk = mhc.alloc_risk(cs, device=dev)
    stream = torch.cuda.current_stream(dev)
    mhc.generate(ctx, cs, poses, stream=stream)
    tuned = mhc.autotune(ctx, cs, poses, table, stream=stream)
    for _ in range(2):
        mhc.evaluate(ctx, cs, poses, table, out=risk, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s_ in range(steps):
        flush.zero_()
        ev[s_][0].record(stream)
        mhc.evaluate(ctx, cs, poses, table, out=risk, stream=stream)
        ev[s_][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    ctx.counters(reset=True)             # kernel split and work counters from further, profiled steps
    ctx.profile_read(reset=True)
    ctx.profile(True)
    for s_ in range(steps):
        flush.zero_()
        mhc.evaluate(ctx, cs, poses, table, out=risk, stream=stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read(reset=True)
    work = ctx.work(reset=True)
    coll_ms, coll_n = prof["collide"]
    coll_s = coll_ms / 1e3 / max(coll_n, 1)
    ops = collide_ops(work, mean_vertices(sc)) / max(coll_n, 1)
    out = {"tests_per_step": sc.n_tests(), "ms_per_step": ms, "tests_per_s": sc.n_tests() / (ms / 1e3),
           "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
           "work_per_step": {k: work[k] / steps for k in ("executed", "narrow")},
           "collide_roofline_frac": ops / coll_s / 1e12 / peak, "collide_achieved": ops / coll_s / 1e12,
           "collide_layout": [tuned[0], tuned[1]]}
    ctx.close()
    del table
    torch.cuda.empty_cache()
    return out


def measure_batch(mhc, torch, dev, steps, flush, batch_peak, count=256):
    """The uneven batch (256 scenarios, 2-24 objects, 64-1024 hypotheses, 20-50 steps) three ways, device
    time per batch with CUDA events (L2 flushed before each): a plan replayed as one CUDA graph, one
    mhc_evaluate_batch call, and the plain path of one mhc_evaluate call per scenario."""
    from paper_2005_06773_gb300 import scenarios as S
    batch = S.batch_scenarios(seed=3, count=count)
    cb = mhc.as_batch(batch)
    info, sls = mhc.batch_slices(cb)
    tests = sum(sc.n_tests() for sc in batch)
    stream = torch.cuda.current_stream(dev)
    ctx = mhc.Context(dev.index or 0, int(info["scratch"]) + (64 << 20))
    poses, table, out = mhc.alloc_batch(info, dev)
    mhc.evaluate_batch(ctx, cb, poses, table, out=out, stream=stream)     # poses for the autotuner
    tuned = mhc.autotune_batch(ctx, cb, poses, table, stream=stream)
    plan = mhc.Plan(ctx, cb, graph=True, buffers=(poses, table, out))

    def timed(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        walls = []
        for q in range(n):
            flush.zero_()
            t0 = time.perf_counter()
            ev[q][0].record(stream)
            fn()
            ev[q][1].record(stream)
            walls.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return statistics.median(ms), 1e3 * statistics.median(walls)

    g_ms, g_host = timed(lambda: plan.launch(stream), steps)
    b_ms, b_host = timed(lambda: mhc.evaluate_batch(ctx, cb, poses, table, out=out, stream=stream), steps)
    ctx.counters(reset=True)             # kernel split and work counters from further, profiled calls
    ctx.profile_read(reset=True)
    ctx.profile(True)
    n_calls = 3
    for _ in range(n_calls):
        flush.zero_()
        mhc.evaluate_batch(ctx, cb, poses, table, out=out, stream=stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read(reset=True)
    work = ctx.work(reset=True)
    # plain path: one mhc_evaluate per scenario into its own slice of the same buffers
    singles = []
    for sc, sl in zip(cb.items, sls):
        n_pose = int(sum(o.n_hyp for o in sc.sc.objects)) * sc.sc.n_steps
        singles.append((sc, {k: v[sl["pose0"]: sl["pose0"] + n_pose] for k, v in poses.items()},
                        table[sl["entry0"]:], mhc.alloc_risk(sc, device=dev)))

    def plain():
        for sc, p, t, r in singles:
            mhc.evaluate(ctx, sc, p, t, out=r, stream=stream)
    p_ms, p_host = timed(plain, max(3, steps // 2))
    plan.close()
    ctx.close()
    del poses, table, out, singles
    torch.cuda.empty_cache()
    return {
        "workload": f"{count} uneven scenarios (seed 3): 2-24 objects (70 % cars), 64-1024 hypotheses "
                    "(log-uniform), 20-50 steps of 0.1 s, all object pairs",
        "tests_per_batch": tests, "entries": info["n_entries"], "hypotheses": info["n_traj"],
        "collide_layout": {"variant": tuned[0], "cull": tuned[1], "chosen_by": "mhc_autotune_batch"},
        "graph": {"ms_per_batch": g_ms, "scenarios_per_s": count / (g_ms / 1e3), "tests_per_s": tests / (g_ms / 1e3),
                  "host_ms_per_launch": g_host},
        "batch_call": {"ms_per_batch": b_ms, "scenarios_per_s": count / (b_ms / 1e3),
                       "tests_per_s": tests / (b_ms / 1e3), "host_ms_per_call": b_host,
                       "kernels_ms_per_batch": {k: v[0] / n_calls for k, v in prof.items()},
                       "work_per_batch": {k: work[k] / n_calls for k in ("executed", "narrow")},
                       "collide_roofline_frac": collide_ops(work) / n_calls / (prof["collide"][0] / n_calls / 1e3) / 1e12
                                                / batch_peak},
        "plain_per_scenario": {"ms_per_batch": p_ms, "scenarios_per_s": count / (p_ms / 1e3),
                               "tests_per_s": tests / (p_ms / 1e3), "host_ms_per_batch": p_host},
    }


def arrivals(rate: float, seconds: float, large_share: float, seed: int = 5):
    """Poisson arrival times (s) and request kinds (0 = 11-object scene, 1 = 32-vehicle scene)."""
    from paper_2005_06773_gb300 import scenarios as S
    rng = S.SplitMix64(seed)
    t, out = 0.0, []
    while True:
        t += -math.log(1.0 - rng.uniform(0.0, 1.0)) / rate
        if t >= seconds:
            return out
        out.append((t, 1 if rng.uniform(0.0, 1.0) < large_share else 0))


def measure_serving(mhc, torch, dev, seconds: float, rates: str = "", rate: float = 2000.0, large_share: float = 0.05):
    """Served requests (continuous batching, mhc_submit / mhc_poll) against the plain path (one synchronous
    mhc_run per request in arrival order) at the same offered load: Poisson arrivals, 95 % shaped like the
    11-object scene (64 placements, cycled) and 5 % like the 32-vehicle scene (4 placements).  The main
    window runs `seconds` at `rate`; the sweep runs 2 s windows at each further rate in `rates`.  Latency =
    arrival (submission) to the risk outputs on the host; the queue of the plain path counts.  Sustained
    load = requests / (last completion - first arrival)."""
    import threading
    from paper_2005_06773_gb300 import scenarios as S
    small = [mhc.as_c(S.intersection11(100 + q)) for q in range(64)]
    large = [mhc.as_c(S.stress32(200 + q)) for q in range(4)]
    ctx = mhc.Context(dev.index or 0, 256 << 20)
    run_ctx = mhc.Context(dev.index or 0, max(mhc.layout(large[0])["run_bytes"], mhc.layout(small[0])["run_bytes"]) + (64 << 20))
    for c in (ctx, run_ctx):   # the collision layouts of both shapes, tuned once per context
        for cs in (small[0], large[0]):
            p = mhc.alloc_poses(cs.sc, dev)
            tb = torch.empty(mhc.layout(cs)["n_entries"], dtype=torch.int16, device=dev)
            mhc.generate(c, cs, p)
            mhc.autotune(c, cs, p, tb)
            del p, tb
    torch.cuda.empty_cache()
    outs = {id(cs): mhc.alloc_risk(cs, device="cpu", pin=True) for cs in small + large}
    for cs in small[:4] + large[:1]:
        mhc.run(run_ctx, cs, out=outs[id(cs)])
    srv = mhc.Server(ctx, 48 << 30)
    for cs in small[:8] + large[:1]:                    # warm-up (stream, pinned buffers, module load)
        t = srv.submit(cs)
        if not srv.poll(t, None, timeout_us=120_000_000):
            raise RuntimeError("warm-up request not finished after 120 s")
        srv.release(t)

    def summary(v):
        return {"n": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99), "max_ms": max(v) if v else None}

    def one_rate(r, secs, seed):
        plan = arrivals(r, secs, large_share, seed)
        reqs = [(t, kind, (large[q % 4] if kind else small[q % 64])) for q, (t, kind) in enumerate(plan)]
        tickets = [None] * len(reqs)
        t0 = time.perf_counter()

        def submitter():
            for q, (t, kind, cs) in enumerate(reqs):
                d = t0 + t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[q] = srv.submit(cs)

        th = threading.Thread(target=submitter)
        th.start()
        lat = {0: [], 1: []}
        first_sub, last_done, batch_sizes = None, 0, []
        # finished results are released per kind in arrival order (each lane of the server admits its queue in
        # order): a finished request holds its resident table until released, so waiting on all of them in
        # arrival order could leave the pool full of finished small requests while a queued large one waits
        # for memory
        import collections
        pending = {0: collections.deque(), 1: collections.deque()}
        nxt, idle_since = 0, time.perf_counter()
        while nxt < len(reqs) or pending[0] or pending[1]:
            while nxt < len(reqs) and tickets[nxt] is not None:
                pending[reqs[nxt][1]].append(nxt)
                nxt += 1
            progressed = False
            for kind in (0, 1):
                dq = pending[kind]
                while dq and srv.poll(tickets[dq[0]], None, timeout_us=0):
                    q = dq.popleft()
                    ns, bs = srv.times(tickets[q])
                    srv.release(tickets[q])
                    lat[kind].append((ns[2] - ns[0]) / 1e6)
                    first_sub = ns[0] if first_sub is None else min(first_sub, ns[0])
                    last_done = max(last_done, ns[2])
                    batch_sizes.append(bs)
                    progressed = True
            if progressed:
                idle_since = time.perf_counter()
            elif time.perf_counter() - idle_since > 60.0:
                raise RuntimeError(f"{len(pending[0]) + len(pending[1])} served requests made no progress for 60 s")
            else:
                time.sleep(0.0002)
        th.join()
        served_s = (last_done - first_sub) / 1e9
        # plain path: one mhc_run per request, in arrival order, on one host thread
        plat = {0: [], 1: []}
        t0 = time.perf_counter()
        for t, kind, cs in reqs:
            d = t0 + t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            mhc.run(run_ctx, cs, out=outs[id(cs)])
            plat[kind].append(1e3 * (time.perf_counter() - (t0 + t)))
        plain_s = time.perf_counter() - t0 - reqs[0][0]
        n = len(reqs)
        return {"offered_per_s": r, "window_s": secs, "requests": n,
                "served": {"sustained_per_s": n / served_s, "small": summary(lat[0]), "large": summary(lat[1]),
                           "mean_batch": statistics.mean(batch_sizes) if batch_sizes else None},
                "plain": {"sustained_per_s": n / plain_s, "small": summary(plat[0]), "large": summary(plat[1])}}

    out = {"shape": "95 % 11-object scenes (1.70e8 tests, 64 placements), 5 % 32-vehicle scenes (1.04e11 tests, "
                    "4.2 GB table, 4 placements); plain = mhc_run per request in arrival order, synchronous",
           "main": one_rate(rate, seconds, 5)}
    sweep = [float(x) for x in rates.split(",") if x.strip()]
    if sweep:
        out["sweep"] = [one_rate(r, 2.0, 6 + q) for q, r in enumerate(sweep)]
    out["batches"] = srv.stats()["batches"]
    srv.stop()
    run_ctx.close()
    ctx.close()
    torch.cuda.empty_cache()
    return out


def aggregate(units: float, seconds: float, world: int, device):
    """Whole-job throughput of a weak-scaling run: every rank's units (its own replica's pose tests) summed,
    divided by the slowest rank's time.  Returns (units per second, total units, max seconds)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    t_max, total = float(t.item()), float(u.item())
    return total / t_max, total, t_max


def replica_seed(rank: int) -> int:
    """Each rank runs its own scene replica: the benchmark scene's placement seed plus the rank."""
    return 2 + rank


def run_mhc(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2005_06773_gb300 import mhc

    sc = workload(rank)
    cs = mhc.as_c(sc)
    lay = mhc.layout(cs)
    ctx = mhc.Context(local, 512 << 20)
    poses = mhc.alloc_poses(sc, dev)
    table = torch.empty(lay["n_entries"], dtype=torch.int16, device=dev)
    risk = mhc.alloc_risk(cs, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():   # the whole hot path in one C-ABI call (fused collision + risk accumulation)
        mhc.evaluate(ctx, cs, poses, table, out=risk, stream=stream)

    mhc.generate(ctx, cs, poses, stream=stream)
    if args.collide_variant:
        ctx.set_option(mhc.MHC_OPT_COLLIDE_VARIANT, args.collide_variant)
        tuned = (args.collide_variant, 1)
    else:
        tuned = mhc.autotune(ctx, cs, poses, table, stream=stream)   # untimed set-up: picks the layout

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    try:   # NVML (samples inside even a short timed region), else nvidia-smi
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            uuid = None
        clocks = NvmlClocks(uuid, local)
    except Exception:
        clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_region")   # lets a profiler keep to the timed steps
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    value, tests_all, t_max = aggregate(sc.n_tests() * args.steps, dev_s, world, dev)
    # kernel split, launch count and collision work from a separate pass with the library's per-kernel
    # events on (they add GPU time, so they stay out of the timed steps)
    prof_steps = min(args.steps, 50)
    ctx.counters(reset=True)
    ctx.profile_read(reset=True)
    ctx.profile(True)
    for _ in range(prof_steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read(reset=True)
    work = ctx.work(reset=True)
    # the same step replayed from a plan (the scenario laid out once, its launch sequence a CUDA graph)
    plan = mhc.Plan(ctx, [sc], graph=True)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(prof_steps)]
    for _ in range(3):
        plan.launch(stream)
    for q in range(prof_steps):
        flush.zero_()
        pev[q][0].record(stream)
        plan.launch(stream)
        pev[q][1].record(stream)
    torch.cuda.synchronize()
    plan_ms = [a.elapsed_time(b) for a, b in pev]
    plan.close()

    # end to end through mhc_run: host scenario in, host (pinned) risk out, copies inside the timed region
    host_out = mhc.alloc_risk(cs, device="cpu", pin=True)
    host_struct = mhc.risk_struct(host_out)
    e2e_ctx = mhc.Context(local, max(lay["run_bytes"] + (64 << 20), 256 << 20))
    raw_stream = stream.cuda_stream
    for _ in range(3):
        mhc.run(e2e_ctx, cs, out=host_out, stream=raw_stream, out_struct=host_struct)
    e2e_ms = []
    for _ in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mhc.run(e2e_ctx, cs, out=host_out, stream=raw_stream, out_struct=host_struct)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    h2d, d2h = e2e_ctx.transfer_bytes()
    e2e_ctx.close()
    e2e_value, _, _ = aggregate(sc.n_tests() * args.e2e_steps, sum(e2e_ms) / 1e3, world, dev)

    coll_ms, coll_n = prof["collide"]
    avg_coll_s = coll_ms / 1e3 / max(coll_n, 1)
    ops_per_launch = collide_ops(work, mean_vertices(sc)) / max(coll_n, 1)
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = ops_per_launch / avg_coll_s / 1e12
    traffic = traffic_from_profile(tuned[0])
    launches = sum(n for _, n in prof.values()) * args.steps // max(prof_steps, 1)   # per step x timed steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(sc),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "mhc_run: host scenario -> device -> host risk outputs (pinned), stream synchronised"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": COLLIDE_KERNELS.get(tuned[0], "collide"), "achieved": achieved, "peak": peak,
                     "unit": "T lane-instr/s", "frac": achieved / peak, "traffic": traffic,
                     "avg_launch_ms": 1e3 * avg_coll_s, "ops_per_launch": ops_per_launch,
                     "peak_source": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                                    "(sm_max_mhz of MEASURED_PEAKS.json)",
                     "ops": "5 per executed broad test + 32 rect-rect / 16 rect-disc / 5 disc-disc per narrow test"},
        "clocks": clk,
        "latency_ms": {"device_p50": pct(step_ms, 50), "device_p99": pct(step_ms, 99),
                       "e2e_p50": pct(e2e_ms, 50), "e2e_p99": pct(e2e_ms, 99)},
        "kernels_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()},
        "plan_graph_ms_p50": pct(plan_ms, 50),
        "collision_work": dict({k: v / max(coll_n, 1) for k, v in work.items()}, launches_per_step=coll_n / max(prof_steps, 1)),
        "collide_layout": [tuned[0], tuned[1], "--collide-variant" if args.collide_variant else "mhc_autotune"],
        "wall_s_timed_region": wall,
    }
    if not args.no_extra:
        from paper_2005_06773_gb300 import scenarios as S
        line["extra_workloads"] = {
            "stress32": measure_workload(mhc, torch, S.stress32(4), dev, 5, flush, peak),
            "paper_s2": measure_workload(mhc, torch, S.paper_s1s2(10, 6), dev, 50, flush, peak),
            "outline11": measure_workload(mhc, torch, S.with_outlines(S.intersection11(2), cut=0.35), dev, 50,
                                          flush, peak),
            "paths11": measure_workload(mhc, torch, S.with_lane_paths(S.intersection11(2, n_acc=63)), dev, 50,
                                        flush, peak),
        }
        line["batch"] = measure_batch(mhc, torch, dev, 10, flush, peak)
        line["serving"] = measure_serving(mhc, torch, dev, args.serve_seconds, rates=args.serve_rates)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and WORKLOAD == "intersection11":
        base, oracle_out = cpu_baseline(sc, args.cpu_seconds)
        # the oracle on every host core as well (the whole table of the scene), and on a sample of the
        # 32-vehicle stress scene
        scen_mod = __import__("paper_2005_06773_gb300.scenarios", fromlist=["x"])
        line["cpu_oracle_cores"] = {"intersection11": cpu_oracle_cores(sc, 1 << 40),
                                    "stress32": cpu_oracle_cores(scen_mod.stress32(4), 2_000_000),
                                    "batch256": cpu_oracle_batch(scen_mod.batch_scenarios(seed=3, count=256))}
        # the benchmarked step's own outputs (the last timed step's table and risk) against the oracle's
        line["parity"] = parity_vs_oracle(sc, table, risk, oracle_out)
        line["cpu_baseline"] = base
    if rank == 0:
        # the per-workload and batch figures and the parity check last, where a tail of the output keeps them
        tail = ("serving", "cpu_oracle_cores", "extra_workloads", "batch", "parity", "cpu_baseline")
        ordered = {k: v for k, v in line.items() if k not in tail}
        ordered.update((k, line[k]) for k in tail if k in line)
        print(json.dumps(compact(ordered)), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def compact(v, top=True):
    """The JSON line with nested figures at 4 significant digits (the contract's top-level numbers stay
    exact), so that the whole line stays short."""
    if isinstance(v, dict):
        return {k: (x if top and k in ("value", "ms_per_step") else compact(x, False)) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [compact(x, False) for x in v]
    if isinstance(v, float) and math.isfinite(v) and not top:
        return float(f"{v:.4g}")
    return v


def parity_vs_oracle(sc, table, risk, oracle_out):
    """The benchmarked step's table and risk outputs against the oracle's on the same scene: entries that
    differ, how many of them are borderline (excused: the oracle's margin within 1 mm of zero at every
    disagreeing step), the pose tests inside the +-1 mm band, and the largest relative difference of the
    risk probabilities (the oracle's risk taken from the GPU's own table)."""
    import numpy as np
    from oracle import oracle, parity
    t = table.cpu().numpy()
    poses, tab_o, pairs, poff = (oracle_out[k] for k in ("poses", "table", "pairs", "pair_off"))
    agree = parity.table_agreement(sc, t, tab_o, poses, pairs, poff)
    r_o = oracle.risk(sc, t, pairs)
    g = {k: v.cpu().numpy() for k, v in risk.items()}
    ints_equal = all(np.array_equal(g[k], r_o[k]) for k in ("count", "count_k", "hits"))
    rel = 0.0
    for k in ("P", "H", "naive", "cond", "indep", "attr_obj", "attr_step"):
        d = np.abs(g[k] - r_o[k]) / np.maximum(np.abs(r_o[k]), 1e-300)
        rel = max(rel, float(d[np.abs(r_o[k]) > 1e-15].max(initial=0.0)))
    return {"tables_equal": agree["n_disagree"] == 0, "n_disagree": agree["n_disagree"],
            "n_excused": agree["n_excused"], "n_bad": agree["n_bad"],
            "excused_per_test": agree["n_excused"] / sc.n_tests(),
            "band_tests_1mm": parity.band_count(sc, poses), "risk_ints_equal": ints_equal,
            "risk_max_rel_err": rel}


def main():
    global WORKLOAD
    args = parse()
    WORKLOAD = args.workload
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
        return
    run_mhc(args)


if __name__ == "__main__":
    main()
