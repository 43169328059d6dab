"""Pins of the oracle's convex-outline shapes (Section IV-C.1 allows an object's outline to be as detailed as
needed; the oracle takes any convex polygon).  The overlap flag is checked against brute-force segment
crossings and containment, the margin against sampled boundary distances and hand-computed cases, and
a rectangle given as a 4-gon against the rectangle code; at table level, an outline inside the
rectangle can only delay or remove a first collision."""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S
from paper_2005_06773_gb300.scenarios import SplitMix64


def world(outline, x, y, psi):
    c, s = math.cos(psi), math.sin(psi)
    return [(x + c * vx - s * vy, y + s * vx + c * vy) for vx, vy in np.asarray(outline, float)]


def cross(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def segments_meet(p1, p2, q1, q2):
    d1, d2 = cross(q1, q2, p1), cross(q1, q2, p2)
    d3, d4 = cross(p1, p2, q1), cross(p1, p2, q2)
    return ((d1 > 0 > d2) or (d1 < 0 < d2)) and ((d3 > 0 > d4) or (d3 < 0 < d4))


def point_in_polygon(p, poly):
    """Crossing-number test (Shimrat / Haines)."""
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
    for i in range(len(A)):
        for j in range(len(B)):
            if segments_meet(A[i], A[(i + 1) % len(A)], B[j], B[(j + 1) % len(B)]):
                return True
    return point_in_polygon(A[0], B) or point_in_polygon(B[0], A)


def sampled_boundary(poly, n=300):
    pts = []
    for i in range(len(poly)):
        a, b = np.array(poly[i]), np.array(poly[(i + 1) % len(poly)])
        t = np.linspace(0, 1, n, endpoint=False)[:, None]
        pts.append(a + t * (b - a))
    return np.concatenate(pts)


def random_convex(rng, n_lo=3, n_hi=8, r_lo=0.6, r_hi=2.5):
    """Convex polygon: vertices at sorted random angles on a random ellipse (strictly convex, CCW)."""
    n = rng.randint(n_lo, n_hi)
    while True:
        ang = sorted(rng.uniform(0.0, 2 * math.pi) for _ in range(n))
        gaps = [(ang[(i + 1) % n] - ang[i]) % (2 * math.pi) for i in range(n)]
        if min(gaps) > 0.15 and max(gaps) < math.pi - 0.1:
            break
    a, b = rng.uniform(r_lo, r_hi), rng.uniform(r_lo, r_hi)
    return np.array([[a * math.cos(t), b * math.sin(t)] for t in ang])


def shape(kind, x, y, psi, outline=None, length=0.0, width=0.0, radius=0.0):
    d = dict(kind=kind, x=x, y=y, psi=psi, length=length, width=width, radius=radius)
    if outline is not None:
        d["outline"] = outline
    return d


def test_polygon_overlap_matches_brute_force(orc):
    rng = SplitMix64(21)
    decided = 0
    for _ in range(2500):
        A, B = random_convex(rng), random_convex(rng)
        pa, pb = rng.uniform(-math.pi, math.pi), rng.uniform(-math.pi, math.pi)
        xb, yb = rng.uniform(-5, 5), rng.uniform(-5, 5)
        m, flag = orc.margin_shapes(shape(2, 0.0, 0.0, pa, A), shape(2, xb, yb, pb, B))
        assert flag == (m <= 0.0)
        if abs(m) < 1e-9:
            continue
        decided += 1
        assert (m <= 0) == brute_overlap(world(A, 0, 0, pa), world(B, xb, yb, pb))
    assert decided > 2400


def test_polygon_distance_matches_sampled_boundary(orc):
    rng = SplitMix64(22)
    checked = 0
    for _ in range(80):
        A, B = random_convex(rng), random_convex(rng)
        pa, pb = rng.uniform(-3, 3), rng.uniform(-3, 3)
        xb, yb = rng.uniform(-8, 8), rng.uniform(-8, 8)
        m, _ = orc.margin_shapes(shape(2, 0.0, 0.0, pa, A), shape(2, xb, yb, pb, B))
        WA, WB = world(A, 0, 0, pa), world(B, xb, yb, pb)
        if brute_overlap(WA, WB):
            assert m <= 0
            continue
        sa, sb = sampled_boundary(WA), sampled_boundary(WB)
        d = np.sqrt(((sa[:, None, :] - sb[None, :, :]) ** 2).sum(-1)).min()
        spacing = max(np.hypot(*np.subtract(P[(i + 1) % len(P)], P[i])) for P in (WA, WB) for i in range(len(P))) / 300
        assert m <= d + 1e-9 and d - m < spacing + 1e-9
        checked += 1
    assert checked > 40


def test_polygon_disc_matches_sampled_boundary(orc):
    rng = SplitMix64(23)
    for _ in range(200):
        A = random_convex(rng)
        psi = rng.uniform(-3, 3)
        cx, cy = rng.uniform(-3.5, 3.5), rng.uniform(-3.5, 3.5)
        m, flag = orc.margin_shapes(shape(2, 0.0, 0.0, psi, A), shape(1, cx, cy, 0.0, radius=0.4))
        m2, _ = orc.margin_shapes(shape(1, cx, cy, 0.0, radius=0.4), shape(2, 0.0, 0.0, psi, A))
        assert m == m2 and flag == (m <= 0)
        W = world(A, 0, 0, psi)
        pts = sampled_boundary(W, 2000)
        d = np.sqrt(((pts - np.array([cx, cy])) ** 2).sum(-1)).min()
        tol = max(np.hypot(*np.subtract(W[(i + 1) % len(W)], W[i])) for i in range(len(W))) / 2000 + 1e-9
        if point_in_polygon((cx, cy), W):
            assert abs(m + 0.4 + d) < tol
        else:
            assert abs(m - (d - 0.4)) < tol


def test_rectangle_as_four_gon_equals_rectangle(orc):
    rng = SplitMix64(24)
    quad = np.array([[2.25, 0.9], [-2.25, 0.9], [-2.25, -0.9], [2.25, -0.9]])
    for _ in range(500):
        pa, pb = rng.uniform(-3, 3), rng.uniform(-3, 3)
        xb, yb = rng.uniform(-7, 7), rng.uniform(-7, 7)
        m_rect, f_rect = orc.margin_shapes(shape(0, 0.0, 0.0, pa, length=4.5, width=1.8),
                                           shape(0, xb, yb, pb, length=3.13, width=1.46))
        m_poly, f_poly = orc.margin_shapes(shape(2, 0.0, 0.0, pa, quad),
                                           shape(0, xb, yb, pb, length=3.13, width=1.46))
        assert abs(m_rect - m_poly) < 1e-12 and f_rect == f_poly
        m_rd, _ = orc.margin_shapes(shape(0, 0.0, 0.0, pa, length=4.5, width=1.8), shape(1, xb / 2, yb / 2, 0.0, radius=0.4))
        m_pd, _ = orc.margin_shapes(shape(2, 0.0, 0.0, pa, quad), shape(1, xb / 2, yb / 2, 0.0, radius=0.4))
        assert abs(m_rd - m_pd) < 1e-12


@pytest.mark.parametrize("dx,dy,psi_b,expect", [
    (3.0, 0.0, 0.0, 1.0),                     # unit squares (half side 1) face to face, 1 m apart
    (2.0, 0.0, 0.0, 0.0),                     # touching faces count as overlap
    (1.5, 0.0, 0.0, -0.5),                    # 0.5 m penetration
    (3.0, 3.0, 0.0, math.sqrt(2.0)),          # corner to corner along the diagonal
    (1.0 + math.sqrt(2.0) + 0.5, 0.0, math.pi / 4, 0.5),   # a diamond's tip 0.5 m in front of a face
])
def test_square_closed_forms(orc, dx, dy, psi_b, expect):
    sq = np.array([[1.0, 1.0], [-1.0, 1.0], [-1.0, -1.0], [1.0, -1.0]])
    m, flag = orc.margin_shapes(shape(2, 0.0, 0.0, 0.0, sq), shape(2, dx, dy, psi_b, sq))
    assert abs(m - expect) < 1e-12 and flag == (expect <= 0)


def test_hexagon_disc_closed_forms(orc):
    """Regular hexagon of circumradius 1 (apothem sqrt(3)/2) against a disc of radius 0.25."""
    hexa = np.array([[math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)] for k in range(6)])
    ap = math.sqrt(3.0) / 2
    for k in range(6):
        t = (k + 0.5) * math.pi / 3                # toward the middle of an edge
        m, _ = orc.margin_shapes(shape(2, 0.0, 0.0, 0.0, hexa), shape(1, 2 * math.cos(t), 2 * math.sin(t), 0.0, radius=0.25))
        assert abs(m - (2 - ap - 0.25)) < 1e-12
        t = k * math.pi / 3                        # toward a vertex
        m, _ = orc.margin_shapes(shape(2, 0.0, 0.0, 0.0, hexa), shape(1, 2 * math.cos(t), 2 * math.sin(t), 0.0, radius=0.25))
        assert abs(m - (1 - 0.25)) < 1e-12
    m, flag = orc.margin_shapes(shape(2, 0.0, 0.0, 0.0, hexa), shape(1, 0.0, 0.0, 0.0, radius=0.25))
    assert abs(m - (-ap - 0.25)) < 1e-12 and flag


def test_polygon_symmetry_and_rigid_invariance(orc):
    rng = SplitMix64(25)
    for _ in range(300):
        A, B = random_convex(rng), random_convex(rng)
        xa, ya, pa = rng.uniform(-4, 4), rng.uniform(-4, 4), rng.uniform(-3, 3)
        xb, yb, pb = rng.uniform(-4, 4), rng.uniform(-4, 4), rng.uniform(-3, 3)
        m, _ = orc.margin_shapes(shape(2, xa, ya, pa, A), shape(2, xb, yb, pb, B))
        m_sym, _ = orc.margin_shapes(shape(2, xb, yb, pb, B), shape(2, xa, ya, pa, A))
        th, tx, ty = rng.uniform(-3, 3), rng.uniform(-50, 50), rng.uniform(-50, 50)
        c, s = math.cos(th), math.sin(th)
        m_rot, _ = orc.margin_shapes(shape(2, tx + c * xa - s * ya, ty + s * xa + c * ya, pa + th, A),
                                     shape(2, tx + c * xb - s * yb, ty + s * xb + c * yb, pb + th, B))
        assert abs(m - m_sym) < 1e-12
        assert abs(m - m_rot) < 1e-9


def test_outline_inside_rectangle_delays_first_collisions(orc):
    """A chamfered outline lies inside its rectangle, so wherever it overlaps the rectangle does: every
    first-collision step with outlines is at or after the rectangle's (or there is none), some strictly."""
    sc = S.tiny_crossing(1, start=15.0)
    poses = orc.generate(sc)
    tab_r, _, _ = orc.table(sc, poses)
    sc_o = S.with_outlines(sc, cut=0.6)
    tab_o, _, _ = orc.table(sc_o, poses)
    assert (tab_r >= 0).any()
    later = (tab_o == -1) | (tab_o >= tab_r)
    assert np.all(later[tab_r >= 0]) and np.all(tab_o[tab_r == -1] == -1)
    assert np.any(tab_o != tab_r)
    # a zero cut is the rectangle itself
    tab_q, _, _ = orc.table(S.with_outlines(sc, cut=0.0), poses)
    assert np.array_equal(tab_q, tab_r)
    # and the registry is cleared for scenes without outlines
    tab_again, _, _ = orc.table(sc, poses)
    assert np.array_equal(tab_again, tab_r)
