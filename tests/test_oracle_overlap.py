"""Pins of the oracle's overlap test (Section IV-C.1) against brute-force polygon geometry, sampled boundary
distances and hand-computed cases.  The brute force here uses segment crossings and crossing-number
containment (cross products), not the oracle's projection arithmetic."""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300.scenarios import SplitMix64


def rect_corners(x, y, psi, L, W):
    c, s = math.cos(psi), math.sin(psi)
    out = []
    for a, b in ((1, 1), (1, -1), (-1, -1), (-1, 1)):
        out.append((x + a * L / 2 * c - b * W / 2 * s, y + a * L / 2 * s + b * W / 2 * c))
    return out


def cross(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def on_segment(p, a, b):
    return min(a[0], b[0]) - 1e-12 <= p[0] <= max(a[0], b[0]) + 1e-12 and \
        min(a[1], b[1]) - 1e-12 <= p[1] <= max(a[1], b[1]) + 1e-12


def segments_meet(p1, p2, q1, q2):
    d1, d2 = cross(q1, q2, p1), cross(q1, q2, p2)
    d3, d4 = cross(p1, p2, q1), cross(p1, p2, q2)
    if ((d1 > 0 > d2) or (d1 < 0 < d2)) and ((d3 > 0 > d4) or (d3 < 0 < d4)):
        return True
    return (d1 == 0 and on_segment(p1, q1, q2)) or (d2 == 0 and on_segment(p2, q1, q2)) or \
        (d3 == 0 and on_segment(q1, p1, p2)) or (d4 == 0 and on_segment(q2, p1, p2))


def point_in_polygon(p, poly):
    """Crossing-number test (Shimrat / Haines); points on the boundary are handled by the edge tests."""
    inside = False
    n = len(poly)
    for i in range(n):
        a, b = poly[i], poly[(i + 1) % n]
        if (a[1] > p[1]) != (b[1] > p[1]):
            xi = a[0] + (p[1] - a[1]) * (b[0] - a[0]) / (b[1] - a[1])
            if p[0] < xi:
                inside = not inside
    return inside


def brute_overlap(A, B):
    for i in range(4):
        for j in range(4):
            if segments_meet(A[i], A[(i + 1) % 4], B[j], B[(j + 1) % 4]):
                return True
    return point_in_polygon(A[0], B) or point_in_polygon(B[0], A)


def sampled_boundary(poly, n=400):
    pts = []
    for i in range(len(poly)):
        a, b = np.array(poly[i]), np.array(poly[(i + 1) % len(poly)])
        t = np.linspace(0, 1, n, endpoint=False)[:, None]
        pts.append(a + t * (b - a))
    return np.concatenate(pts)


def test_rect_rect_matches_brute_force(orc):
    rng = SplitMix64(11)
    decided = 0
    for _ in range(3000):
        La, Wa = rng.uniform(1.0, 6.0), rng.uniform(0.5, 2.5)
        Lb, Wb = rng.uniform(1.0, 6.0), rng.uniform(0.5, 2.5)
        xb, yb = rng.uniform(-6, 6), rng.uniform(-6, 6)
        pa, pb = rng.uniform(-math.pi, math.pi), rng.uniform(-math.pi, math.pi)
        m = orc.margin(0, La, Wa, 0, 0.0, 0.0, pa, 0, Lb, Wb, 0, xb, yb, pb)
        if abs(m) < 1e-9:
            continue
        decided += 1
        brute = brute_overlap(rect_corners(0, 0, pa, La, Wa), rect_corners(xb, yb, pb, Lb, Wb))
        assert (m <= 0) == brute, (La, Wa, Lb, Wb, xb, yb, pa, pb, m)
    assert decided > 2900


def test_rect_rect_distance_matches_sampled_boundary(orc):
    rng = SplitMix64(12)
    for _ in range(60):
        pa, pb = rng.uniform(-3, 3), rng.uniform(-3, 3)
        xb, yb = rng.uniform(-9, 9), rng.uniform(-9, 9)
        m = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, pa, 0, 4.5, 1.8, 0, xb, yb, pb)
        A, B = rect_corners(0, 0, pa, 4.5, 1.8), rect_corners(xb, yb, pb, 4.5, 1.8)
        if brute_overlap(A, B):
            assert m <= 0
            continue
        sa, sb = sampled_boundary(A), sampled_boundary(B)
        d = np.sqrt(((sa[:, None, :] - sb[None, :, :]) ** 2).sum(-1)).min()
        # sampling spacing is at most 4.5 / 400; the sampled distance over-estimates by < one spacing
        assert m <= d + 1e-9 and d - m < 4.5 / 400 + 1e-9


def test_plus_shape_overlaps_but_paper_vertex_test_misses_it(orc):
    """Two 4.5 x 1.8 m cars centred on the same point at 90 degrees: no vertex of either lies in the other,
    so the paper's vertex-in-polygon test (both directions) reports no overlap, but the rectangles do
    intersect.  The exact test counts it."""
    m = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, 0.0, 0, 4.5, 1.8, 0, 0.0, 0.0, math.pi / 2)
    assert m < -0.8
    assert not orc.overlap_pip(4.5, 1.8, 0.0, 0.0, 0.0, 4.5, 1.8, 0.0, 0.0, math.pi / 2)
    assert brute_overlap(rect_corners(0, 0, 0, 4.5, 1.8), rect_corners(0, 0, math.pi / 2, 4.5, 1.8))
    # ordinary corner overlap: both tests agree
    assert orc.overlap_pip(4.5, 1.8, 0.0, 0.0, 0.0, 4.5, 1.8, 4.0, 1.5, 0.0)
    assert orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, 0.0, 0, 4.5, 1.8, 0, 4.0, 1.5, 0.0) < 0


@pytest.mark.parametrize("dx,dy,expect", [
    (4.5 + 0.5, 0.0, 0.5),            # end to end, 0.5 m gap
    (0.0, 1.8 + 0.25, 0.25),          # side by side, 0.25 m gap
    (4.5, 0.0, 0.0),                  # touching end to end counts
    (4.5 - 0.3, 0.0, -0.3),           # 0.3 m longitudinal penetration
    (1.0, 1.8 - 0.2, -0.2),           # 0.2 m lateral penetration (smaller than longitudinal 3.5)
    (4.5 + 3.0, 1.8 + 4.0, 5.0),      # corner to corner: 3-4-5 triangle
])
def test_axis_aligned_margins(orc, dx, dy, expect):
    m = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, 0.0, 0, 4.5, 1.8, 0, dx, dy, 0.0)
    assert abs(m - expect) < 1e-12
    # a half-turn of either rectangle leaves the shape unchanged
    m2 = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, math.pi, 0, 4.5, 1.8, 0, dx, dy, 0.0)
    assert abs(m2 - expect) < 1e-12


@pytest.mark.parametrize("cx,cy,expect", [
    (2.25 + 0.4 + 0.1, 0.0, 0.1),     # in front of the nose
    (0.0, -(0.9 + 0.4), 0.0),         # touching the side
    (2.25 + 0.3, 0.9 + 0.4, 0.5 - 0.4),  # corner region: hypot(0.3, 0.4) - r
    (0.5, 0.2, -(0.4 + 0.7)),         # centre inside, nearest boundary 0.7 m away (side)
])
def test_rect_disc_margins(orc, cx, cy, expect):
    m = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, 0.0, 1, 0, 0, 0.4, cx, cy, 0.0)
    assert abs(m - expect) < 1e-12
    m2 = orc.margin(1, 0, 0, 0.4, cx, cy, 0.0, 0, 4.5, 1.8, 0, 0.0, 0.0, 0.0)
    assert abs(m2 - expect) < 1e-12


def test_rect_disc_matches_sampled_boundary(orc):
    rng = SplitMix64(13)
    for _ in range(200):
        psi = rng.uniform(-3, 3)
        cx, cy = rng.uniform(-4, 4), rng.uniform(-3, 3)
        m = orc.margin(0, 4.5, 1.8, 0, 0.0, 0.0, psi, 1, 0, 0, 0.4, cx, cy, 0.0)
        A = rect_corners(0, 0, psi, 4.5, 1.8)
        inside = point_in_polygon((cx, cy), A)
        d = np.sqrt(((sampled_boundary(A, 2000) - np.array([cx, cy])) ** 2).sum(-1)).min()
        if inside:
            assert m <= -0.4 and abs(m + 0.4 + d) < 4.5 / 2000 + 1e-9
        else:
            assert abs(m - (d - 0.4)) < 4.5 / 2000 + 1e-9


def test_disc_disc(orc):
    assert abs(orc.margin(1, 0, 0, 0.4, 0, 0, 0, 1, 0, 0, 0.4, 3.0, 4.0, 0) - 4.2) < 1e-12
    assert orc.margin(1, 0, 0, 0.4, 0, 0, 0, 1, 0, 0, 0.4, 0.8, 0.0, 0) == 0.0


def test_margin_symmetry_and_rigid_invariance(orc):
    rng = SplitMix64(14)
    for _ in range(300):
        ka, kb = rng.randint(0, 1), rng.randint(0, 1)
        xa, ya, pa = rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-3, 3)
        xb, yb, pb = rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-3, 3)
        m = orc.margin(ka, 4.5, 1.8, 0.4, xa, ya, pa, kb, 3.13, 1.46, 0.4, xb, yb, pb)
        m_sym = orc.margin(kb, 3.13, 1.46, 0.4, xb, yb, pb, ka, 4.5, 1.8, 0.4, xa, ya, pa)
        th, tx, ty = rng.uniform(-3, 3), rng.uniform(-50, 50), rng.uniform(-50, 50)
        c, s = math.cos(th), math.sin(th)
        rot = lambda x, y: (tx + c * x - s * y, ty + s * x + c * y)
        xa2, ya2 = rot(xa, ya)
        xb2, yb2 = rot(xb, yb)
        m_rot = orc.margin(ka, 4.5, 1.8, 0.4, xa2, ya2, pa + th, kb, 3.13, 1.46, 0.4, xb2, yb2, pb + th)
        assert abs(m - m_sym) < 1e-12
        assert abs(m - m_rot) < 1e-9
