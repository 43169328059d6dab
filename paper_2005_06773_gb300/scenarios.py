"""Seeded synthetic scenario generators shared by the CUDA path, the oracle tests and the benchmark.

This module only *describes inputs*: object shapes, initial states and the control grids each object's
hypotheses are drawn from.  It contains none of the method's arithmetic (no motion model, no overlap
test, no probability), so that the oracle and the CUDA path can both consume its output without sharing
code.  Every floating-point input is rounded to FP32 here, before either side sees it.

Workloads (shapes follow the paper's scenarios, §VI-B, and the five benchmark configurations):

* ``tiny_crossing``   two 4.5 x 1.8 m cars on a 90 degree crossing, 16 hypotheses each, 20 steps of 0.1 s.
* ``intersection11``  paper-shaped 11-object intersection: 7 cars (441 hypotheses) + 4 pedestrians (121),
  30 steps of 0.1 s, all object pairs.
* ``batch_scenarios`` many uneven intersections (2-24 objects, 64-1024 hypotheses, 20-50 steps).
* ``stress32``        32 cars x 2048 hypotheses, 50 steps.
* ``paper_s1s2``      the paper's S1/S2 shape (EGO 2058 = 6 x 343, each CO 42 = 6 x 7, 100 steps of 20 ms),
  EGO-only pairing (§IV-C.1, Table I).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), mapped to doubles in [0, 1) with 53 bits.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

VEHICLE = 0
PEDESTRIAN = 1

ALL_PAIRS = 0
EGO_ONLY = 1

MODEL_OT = 0   # one-track (linear bicycle) dynamics, Eq. (onetrack)
MODEL_KIN = 1  # kinematic bicycle

# pedestrian flag: grid_a holds accelerations (paper's sampling, §IV-B.3) instead of initial speeds
PED_ACCEL_GRID = 1

F32 = np.float32

# Default "mid-size car" one-track parameters (m, I_z, l_f, l_r, c_af, c_ar).  The paper takes them
# from cited tables that are not reproduced in it (§IV-B.1); these values are the project's choice.
DEFAULT_VEH_PARAMS = np.array([1500.0, 2500.0, 1.2, 1.5, 80000.0, 80000.0], dtype=F32)


class SplitMix64:
    """SplitMix64 generator; ``uniform()`` returns a double in [0, 1)."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on the closed range [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1)) % (hi - lo + 1)


@dataclasses.dataclass
class Obj:
    """One traffic object and the control grid its hypotheses are sampled from.

    Vehicles (rectangles centred on the pose point, body axis along psi, or the convex `outline` given in
    the body frame): hypothesis h = i_a * n_b + i_b uses acceleration grid_a[i_a] (m/s^2) and constant
    front steering angle grid_b[i_b] (rad).
    Pedestrians (discs): grid_a holds initial speeds (m/s) or, with PED_ACCEL_GRID, accelerations;
    grid_b holds heading offsets (rad) added to psi0.
    """
    kind: int
    length: float
    width: float
    radius: float
    x0: float
    y0: float
    psi0: float
    v0: float
    grid_a: np.ndarray
    grid_b: np.ndarray
    params: Optional[np.ndarray] = None
    v_max: float = 0.0
    flags: int = 0
    outline: Optional[np.ndarray] = None   # vehicles: convex outline, [n, 2] body-frame vertices (x ahead)
    paths: Optional[np.ndarray] = None     # vehicles: [n_b, 3, 3] path sections (x, y, psi) to follow

    def __post_init__(self):
        for f in ("length", "width", "radius", "x0", "y0", "psi0", "v0", "v_max"):
            setattr(self, f, float(F32(getattr(self, f))))
        self.grid_a = np.ascontiguousarray(self.grid_a, dtype=F32)
        self.grid_b = np.ascontiguousarray(self.grid_b, dtype=F32)
        if self.params is not None:
            self.params = np.ascontiguousarray(self.params, dtype=F32)
        if self.outline is not None:
            self.outline = np.ascontiguousarray(np.asarray(self.outline).reshape(-1, 2), dtype=F32)
        if self.paths is not None:
            self.paths = np.ascontiguousarray(np.asarray(self.paths).reshape(-1, 3, 3), dtype=F32)

    @property
    def n_hyp(self) -> int:
        return int(self.grid_a.size * self.grid_b.size)


@dataclasses.dataclass
class Scenario:
    objects: List[Obj]
    tau: float = 0.1
    n_steps: int = 20
    substeps: int = 5
    pair_mode: int = ALL_PAIRS
    ego: int = 0
    model: int = MODEL_OT
    name: str = ""

    def __post_init__(self):
        self.tau = float(F32(self.tau))

    @property
    def n_objects(self) -> int:
        return len(self.objects)

    @property
    def hyp_counts(self) -> List[int]:
        return [o.n_hyp for o in self.objects]

    def pairs(self) -> List[tuple]:
        """Object pairs in table order: (a, b) with a < b for ALL_PAIRS; (ego, b) for EGO_ONLY."""
        n = self.n_objects
        if self.pair_mode == EGO_ONLY:
            return [(self.ego, b) for b in range(n) if b != self.ego]
        return [(a, b) for a in range(n) for b in range(a + 1, n)]

    def n_tests(self) -> int:
        """Nominal pose-pair tests: sum over object pairs of h_a * h_b * N (the paper's 'pose combinations')."""
        h = self.hyp_counts
        return sum(h[a] * h[b] for a, b in self.pairs()) * self.n_steps

    def n_traj_pairs(self) -> int:
        h = self.hyp_counts
        return sum(h[a] * h[b] for a, b in self.pairs())


# ----------------------------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------------------------

def accel_grid_paper(n: int, lo: float, hi: float) -> np.ndarray:
    """Longitudinal sampling rule of §IV-B.2(a): the minimum, zero and the maximum of the range are
    samples; the remaining n - 3 samples are spread evenly over the open negative region (lo, 0).
    Returned in ascending order."""
    if n < 3:
        raise ValueError("the paper's acceleration rule needs at least 3 samples")
    r = n - 3
    neg = [lo * k / (r + 1) for k in range(r, 0, -1)]  # lo*r/(r+1) ... lo/(r+1), ascending
    return np.array([lo] + neg + [0.0, hi], dtype=F32)


def linspace(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n, dtype=np.float64).astype(F32)


# ----------------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------------

CAR_L, CAR_W = 4.5, 1.8
PED_R = 0.4
LANE_OFF = 1.75      # right-hand lane centre offset from the road axis, lane width 3.5 m
STOP_LINE = 7.0      # distance of the stop line from the intersection centre


def _car(x, y, psi, v, grid_a, grid_b, params=None) -> Obj:
    return Obj(VEHICLE, CAR_L, CAR_W, 0.0, x, y, psi, v, grid_a, grid_b,
               DEFAULT_VEH_PARAMS if params is None else params)


def tiny_crossing(seed: int = 1, start: float = 30.0) -> Scenario:
    """Two cars on a 90 degree crossing, `start` metres from the conflict point, speeds U[10, 15] m/s,
    4 accelerations {-6, -3, 0, 2} x 4 steering angles in [-0.1, 0.1]; 20 steps of 0.1 s."""
    rng = SplitMix64(seed)
    ga = accel_grid_paper(4, -6.0, 2.0)
    gb = linspace(-0.1, 0.1, 4)
    va, vb = rng.uniform(10.0, 15.0), rng.uniform(10.0, 15.0)
    objs = [_car(-start, 0.0, 0.0, va, ga, gb), _car(0.0, -start, math.pi / 2, vb, ga, gb)]
    return Scenario(objs, tau=0.1, n_steps=20, substeps=5, name=f"tiny_crossing_s{seed}_d{start:g}")


_ARMS = (  # (unit vector from centre to arm, heading toward centre, lateral unit vector of right lane)
    ((1.0, 0.0), math.pi, (0.0, 1.0)),          # east arm, driving west, right lane north of axis
    ((0.0, 1.0), -math.pi / 2, (-1.0, 0.0)),    # north arm, driving south
    ((-1.0, 0.0), 0.0, (0.0, -1.0)),            # west arm, driving east
    ((0.0, -1.0), math.pi / 2, (1.0, 0.0)),     # south arm, driving north
)


def _place_cars(rng: SplitMix64, n: int, per_arm: Optional[int], d_lo: float, d_hi: float,
                spacing: float, v_lo: float, v_hi: float):
    """Cars queued on the four approach arms, heading to the centre, centre-to-centre spacing >= spacing.
    A car whose drawn arm has no room left goes to the emptiest arm that has."""
    arms: List[List[float]] = [[], [], [], []]
    out = []
    for c in range(n):
        first = (c % 4) if per_arm is not None else rng.randint(0, 3)
        order = [first] + sorted((q for q in range(4) if q != first), key=lambda q: (len(arms[q]), q))
        for arm in order:
            hi = d_hi + (spacing * len(arms[arm]) if per_arm is not None else 0.0)
            d = None
            for _ in range(10000):
                cand = rng.uniform(d_lo, hi)
                if all(abs(cand - e) >= spacing for e in arms[arm]):
                    d = cand
                    break
            if d is not None:
                break
        else:
            raise RuntimeError("placement failed")
        arms[arm].append(d)
        (ux, uy), psi, (lx, ly) = _ARMS[arm]
        r = STOP_LINE + d
        v = rng.uniform(v_lo, v_hi)
        out.append((ux * r + lx * LANE_OFF, uy * r + ly * LANE_OFF, psi, v))
    return out


_CORNERS = ((1, 1, math.pi), (-1, 1, -math.pi / 2), (-1, -1, 0.0), (1, -1, math.pi / 2))


def _place_pedestrian(rng: SplitMix64, corner: int):
    sx, sy, psi = _CORNERS[corner % 4]
    return sx * rng.uniform(5.0, 8.0), sy * rng.uniform(5.0, 8.0), psi


def intersection11(seed: int = 2, n_steps: int = 30, n_acc: int = 21, n_str: int = 21,
                   n_ped_v: int = 11, n_ped_h: int = 11) -> Scenario:
    """Paper-shaped 11-object intersection (7 cars + 4 pedestrians), all object pairs, ego = object 0."""
    rng = SplitMix64(seed)
    ga = accel_grid_paper(n_acc, -8.0, 3.0)
    gb = linspace(-0.3, 0.3, n_str)
    objs = [_car(x, y, psi, v, ga, gb)
            for x, y, psi, v in _place_cars(rng, 7, None, 10.0, 40.0, 7.0, 8.0, 15.0)]
    pv = linspace(0.0, 3.0, n_ped_v)
    ph = linspace(-math.pi / 3, math.pi / 3, n_ped_h)
    for c in range(4):
        x, y, psi = _place_pedestrian(rng, c)
        objs.append(Obj(PEDESTRIAN, 0.0, 0.0, PED_R, x, y, psi, 0.0, pv, ph))
    return Scenario(objs, tau=0.1, n_steps=n_steps, substeps=5, name=f"intersection11_s{seed}")


def _split_hyp(h: int):
    na = max(1, int(round(math.sqrt(h))))
    nb = max(1, int(round(h / na)))
    return na, nb


def random_intersection(rng: SplitMix64, n_obj: int, h_lo: int = 64, h_hi: int = 1024,
                        n_steps: Optional[int] = None, p_vehicle: float = 0.7) -> Scenario:
    kinds = [VEHICLE if (i == 0 or rng.uniform() < p_vehicle) else PEDESTRIAN for i in range(n_obj)]
    n_car = sum(1 for k in kinds if k == VEHICLE)
    per_arm = (n_car + 3) // 4
    cars = iter(_place_cars(rng, n_car, per_arm, 10.0, 30.0, 7.0, 8.0, 15.0))
    objs = []
    corner = 0
    for k in kinds:
        h = int(round(math.exp(rng.uniform(math.log(h_lo), math.log(h_hi)))))
        na, nb = _split_hyp(h)
        if k == VEHICLE:
            x, y, psi, v = next(cars)
            objs.append(_car(x, y, psi, v, accel_grid_paper(max(na, 3), -8.0, 3.0), linspace(-0.3, 0.3, nb)))
        else:
            x, y, psi = _place_pedestrian(rng, corner)
            corner += 1
            objs.append(Obj(PEDESTRIAN, 0.0, 0.0, PED_R, x, y, psi, 0.0,
                            linspace(0.0, 3.0, na), linspace(-math.pi / 3, math.pi / 3, nb)))
    n = n_steps if n_steps is not None else rng.randint(20, 50)
    return Scenario(objs, tau=0.1, n_steps=n, substeps=5)


def batch_scenarios(seed: int = 3, count: int = 256, n_lo: int = 2, n_hi: int = 24,
                    h_lo: int = 64, h_hi: int = 1024) -> List[Scenario]:
    """Uneven scenario batch: n_obj ~ U{n_lo..n_hi}, 70 % cars, hypotheses log-uniform in [h_lo, h_hi],
    N ~ U{20..50} steps of 0.1 s."""
    rng = SplitMix64(seed)
    out = []
    for s in range(count):
        sc = random_intersection(rng, rng.randint(n_lo, n_hi), h_lo, h_hi)
        sc.name = f"batch_s{seed}_{s}"
        out.append(sc)
    return out


def stress32(seed: int = 4, n_cars: int = 32, n_acc: int = 64, n_str: int = 32, n_steps: int = 50) -> Scenario:
    """Throughput stress: 32 cars, 8 per arm, 64 x 32 = 2048 hypotheses each, 50 steps."""
    rng = SplitMix64(seed)
    ga = accel_grid_paper(n_acc, -8.0, 3.0)
    gb = linspace(-0.3, 0.3, n_str)
    objs = [_car(x, y, psi, v, ga, gb)
            for x, y, psi, v in _place_cars(rng, n_cars, n_cars // 4, 10.0, 30.0, 7.0, 8.0, 15.0)]
    return Scenario(objs, tau=0.1, n_steps=n_steps, substeps=5, name=f"stress32_s{seed}")


def paper_s1s2(n_co: int = 10, n_profiles: int = 6, seed: int = 6) -> Scenario:
    """The paper's Table I shape: EGO with n_profiles x 343 hypotheses, each CO n_profiles x 7,
    a 2 s horizon at 20 ms (100 steps), EGO-only pairing (§IV-C.1, §VI-B).  The 343 / 7 controller paths
    are stood in for by constant steering grids."""
    rng = SplitMix64(seed)
    ga = accel_grid_paper(n_profiles, -9.7, 9.7)
    ego = _car(-25.0, -LANE_OFF, 0.0, rng.uniform(10.0, 15.0), ga, linspace(-0.05, 0.05, 343))
    objs = [ego]
    for x, y, psi, v in _place_cars(rng, n_co, None, 5.0, 35.0, 7.0, 8.0, 15.0):
        objs.append(_car(x, y, psi, v, ga, linspace(-0.05, 0.05, 7)))
    return Scenario(objs, tau=0.02, n_steps=100, substeps=1, pair_mode=EGO_ONLY, ego=0,
                    name=f"paper_s{'2' if n_co == 10 else '1'}_p{n_profiles}")


def uniform_weights(sc: Scenario) -> List[np.ndarray]:
    return [np.ones(o.n_hyp, dtype=F32) for o in sc.objects]


def chamfered_outline(length: float, width: float, cut: float) -> np.ndarray:
    """Octagon outline of a length x width body with every corner cut `cut` metres along both sides
    (counter-clockwise, body frame, x ahead); cut = 0 gives the rectangle's corners."""
    hl, hw = length / 2.0, width / 2.0
    if cut <= 0.0:
        return np.array([[hl, hw], [-hl, hw], [-hl, -hw], [hl, -hw]], dtype=F32)
    return np.array([[hl, hw - cut], [hl - cut, hw], [-hl + cut, hw], [-hl, hw - cut],
                     [-hl, -hw + cut], [-hl + cut, -hw], [hl - cut, -hw], [hl, -hw + cut]], dtype=F32)


def with_outlines(sc: Scenario, cut: float = 0.35, every: int = 1) -> Scenario:
    """The scenario with every `every`-th vehicle drawn as its chamfered outline instead of a rectangle."""
    objs = []
    for i, o in enumerate(sc.objects):
        if o.kind == VEHICLE and i % every == 0:
            o = dataclasses.replace(o, outline=chamfered_outline(o.length, o.width, cut))
        objs.append(o)
    return dataclasses.replace(sc, objects=objs, name=f"{sc.name}_outline{cut:g}")


LANE_W = 3.5
PATH_OFFSETS = (-0.875, 0.0, 0.875, LANE_W - 0.6, LANE_W + 0.6, -LANE_W - 0.6, -LANE_W + 0.6)


def lane_paths(o: "Obj", offsets=PATH_OFFSETS, times=(1.0, 1.5, 2.0)) -> np.ndarray:
    """Paths of Section IV-B.2b for a car driving along its current lane: per lateral offset (three samples
    in the own lane, two in each neighbouring lane, relative to the car's current line), three sections
    parallel to the lane through the points the car would reach at the sampling instants at its current
    speed.  [len(offsets), 3, 3] of (x, y, psi)."""
    c, s_ = math.cos(o.psi0), math.sin(o.psi0)
    out = np.zeros((len(offsets), 3, 3), dtype=np.float64)
    for q, off in enumerate(offsets):
        for k, t in enumerate(times):
            along = o.v0 * t
            out[q, k] = (o.x0 + along * c - off * s_, o.y0 + along * s_ + off * c, o.psi0)
    return out.astype(F32)


def with_lane_paths(sc: Scenario, offsets=PATH_OFFSETS, every: int = 1) -> Scenario:
    """The scenario with every `every`-th car following lane paths (hypotheses = accelerations x paths)
    instead of constant steering angles."""
    objs = []
    for i, o in enumerate(sc.objects):
        if o.kind == VEHICLE and i % every == 0:
            o = dataclasses.replace(o, grid_b=np.zeros(len(offsets), dtype=F32), paths=lane_paths(o, offsets))
        objs.append(o)
    return dataclasses.replace(sc, objects=objs, name=f"{sc.name}_paths")


def paper_pedestrians(sc: Scenario, n_acc: int = 9, n_head: int = 12, seed: int = 15) -> Scenario:
    """The scenario with its pedestrians sampled as in Section IV-B.3: accelerations evenly over
    [-12, 12] m/s^2 from an initial walking speed U[0.5, 1.5] m/s, the speed held within [0, 2.7] m/s, and
    headings evenly over the full circle (psi0 + 2 pi q / n_head)."""
    rng = SplitMix64(seed)
    objs = []
    for o in sc.objects:
        if o.kind == PEDESTRIAN:
            o = dataclasses.replace(o, flags=o.flags | PED_ACCEL_GRID, v0=rng.uniform(0.5, 1.5), v_max=2.7,
                                    grid_a=linspace(-12.0, 12.0, n_acc),
                                    grid_b=np.array([2.0 * math.pi * q / n_head for q in range(n_head)], dtype=F32))
        objs.append(o)
    return dataclasses.replace(sc, objects=objs, name=f"{sc.name}_paperped")


def random_weights(sc: Scenario, seed: int) -> List[np.ndarray]:
    rng = SplitMix64(seed)
    return [np.array([rng.uniform(0.05, 1.0) for _ in range(o.n_hyp)], dtype=F32) for o in sc.objects]


def by_name(name: str) -> Scenario:
    table = {
        "tiny": lambda: tiny_crossing(1),
        "tiny_near": lambda: tiny_crossing(1, start=15.0),
        "intersection11": lambda: intersection11(2),
        "stress32": lambda: stress32(4),
        "paper_s2": lambda: paper_s1s2(10, 6),
        "paper_s1": lambda: paper_s1s2(3, 6),
    }
    return table[name]()
