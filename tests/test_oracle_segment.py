"""Pins of the segment contact model (Eq. 3-7: a contact point anywhere on an element, its
displacement interpolated from the two nodal translations by N(xi) of Eq. 4-6, in the element's
frame): the shape functions, the closest points of a segment and a triangle against dense sampling
and constructed cases, and a small-deflection closed form of a cantilever resting on a narrow wall
patch between two nodes, which the node model cannot see."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import beam, contact, segment, solver

L, M = 0.12, 20
l0 = L / M
ROB = wl.robot_desc(L, M)
SEC = beam.section_constants(ROB)
EI = SEC["EI"]


def test_shape_functions():
    for xi in np.linspace(0.0, l0, 7):
        p1, p2, p3, p4 = segment.shape(xi, l0)
        assert p1 + p2 == pytest.approx(1.0, abs=1e-15) and p3 + p4 == pytest.approx(1.0, abs=1e-15)
        assert segment.shape(l0 - xi, l0)[2] == pytest.approx(p4, abs=1e-15)     # P3(l0 - xi) = P4(xi)
    assert segment.shape(0.0, l0) == (1.0, 0.0, 1.0, 0.0)
    assert segment.shape(l0, l0) == (0.0, 1.0, 0.0, 1.0)
    h = 1e-7 * l0                                   # cubic Hermite: zero slope at both ends
    for xi in (0.0, l0 - h):
        assert abs((segment.shape(xi + h, l0)[2] - segment.shape(xi, l0)[2]) / h) <= 1e-5 / l0
    Nm = segment.n_matrix(0.4 * l0, l0)
    assert Nm.shape == (3, 6) and Nm[0, 1] == 0.0 and Nm[1, 0] == 0.0


def test_row_weights_rigid_translation_and_ends():
    rng = np.random.default_rng(30)
    for _ in range(5):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Rr = q * np.sign(np.linalg.det(q))
        v = rng.normal(size=3)
        for xi in (0.0, 0.3 * l0, l0):
            Wm = segment.row_weights(Rr, xi, l0)
            assert np.allclose(Wm @ np.concatenate([v, v]), v, atol=1e-15)
        assert np.allclose(segment.row_weights(Rr, 0.0, l0), np.hstack([np.eye(3), np.zeros((3, 3))]), atol=1e-15)
        assert np.allclose(segment.row_weights(Rr, l0, l0), np.hstack([np.zeros((3, 3)), np.eye(3)]), atol=1e-15)


def test_closest_segment_triangle_vs_sampling_and_constructed_cases():
    rng = np.random.default_rng(31)
    for _ in range(30):
        a, b, c = rng.normal(size=(3, 3))
        p0, p1 = rng.normal(size=(2, 3)) * 1.5
        s, q, w, d, _ = segment.closest_segment_triangle(p0, p1, a, b, c)
        ts = np.linspace(0.0, 1.0, 1201)
        ds = min(np.linalg.norm(p0 + t * (p1 - p0) - contact.closest_point_on_triangle(p0 + t * (p1 - p0), a, b, c))
                 for t in ts)
        step = np.linalg.norm(p1 - p0) / 1200
        assert d <= ds + 1e-12 and d >= ds - step
        assert np.allclose(q, p0 + s * (p1 - p0), atol=1e-14) and abs(np.linalg.norm(q - w) - d) <= 1e-12
    a, b, c = np.array([0, 0, 0.0]), np.array([1, 0, 0.0]), np.array([0, 1, 0.0])
    # crossing the face: distance 0 at the crossing point
    s, q, w, d, interior = segment.closest_segment_triangle(np.array([0.2, 0.2, -1.0]), np.array([0.2, 0.2, 3.0]), a, b, c)
    assert d == 0.0 and interior and s == pytest.approx(0.25) and np.allclose(w, [0.2, 0.2, 0.0])
    # parallel to an edge outside the triangle: the gap to the edge line
    s, q, w, d, interior = segment.closest_segment_triangle(np.array([0.2, -0.5, 0.0]), np.array([0.6, -0.5, 0.0]), a, b, c)
    assert d == pytest.approx(0.5) and not interior and abs(w[1]) <= 1e-15
    # segment above the face, tilted: closest at its lower end, face point below it
    s, q, w, d, interior = segment.closest_segment_triangle(np.array([0.1, 0.1, 0.3]), np.array([0.3, 0.2, 0.9]), a, b, c)
    assert s == 0.0 and d == pytest.approx(0.3) and interior and np.allclose(w, [0.1, 0.1, 0.0])


def _delta(x, c):
    """Deflection at x of an Euler-Bernoulli cantilever (clamped at 0) under a unit load at c."""
    return x * x * (3 * c - x) / (6 * EI) if x <= c else c * c * (3 * x - c) / (6 * EI)


def test_cantilever_on_a_patch_between_nodes_closed_form():
    """Tip load P pushes the rod up against a 1 mm patch above the middle of element 10 (gap g):
    the node model finds no row (the nearest nodes are 2.5 mm away in x), the segment model rests
    on it.  At convergence the chord point sits on the wall, (1 - s) v_a + s v_b = g, and the force
    y enters the nodes with the weights P3, P4 of the row: nodal small-deflection superposition
    gives y in closed form."""
    g = 2e-6
    a = (10 + 0.5) * l0
    lum = wl.patch_lumen(a - 0.5e-3, a + 0.5e-3, ROB.outer_radius + g, z_half=1e-3, n=1)
    P = 2 * g * 6 * EI / (a * a * (3 * L - a))
    node = solver.Model(ROB, lum, solver.Options(step_limit=1.0))
    rn = node.solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert rn.status == solver.OK and rn.contacts == []
    seg = solver.Model(ROB, lum, solver.Options(step_limit=1.0, contact_model="segment"))
    r = seg.solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK and len(r.contacts) >= 1
    act = [c for c in r.contacts if c["force"] > 0.0]
    e, s = act[0]["elem"], act[0]["s"]          # the patch edge where the rising chord is highest
    assert e == 10 and all(c["elem"] == e and c["s"] == pytest.approx(s, abs=1e-12) for c in act)
    assert s == pytest.approx((0.5e-3 + 0.5 * l0) / l0, abs=1e-4)
    y = sum(c["force"] for c in act)
    xa, xb = e * l0, (e + 1) * l0
    _, _, p3, p4 = segment.shape(s * l0, l0)
    num = (1 - s) * P * _delta(xa, L) + s * P * _delta(xb, L) - g
    den = (1 - s) * (p3 * _delta(xa, xa) + p4 * _delta(xa, xb)) + s * (p3 * _delta(xb, xa) + p4 * _delta(xb, xb))
    assert y == pytest.approx(num / den, rel=1e-5)
    va = P * _delta(xa, L) - y * (p3 * _delta(xa, xa) + p4 * _delta(xa, xb))
    vb = P * _delta(xb, L) - y * (p3 * _delta(xb, xa) + p4 * _delta(xb, xb))
    assert r.node_pos[e, 1] == pytest.approx(va, rel=1e-5) and r.node_pos[e + 1, 1] == pytest.approx(vb, rel=1e-5)
    # the chord point at the wall (the normal to the patch edge tilts with the chord's slope, which
    # shifts the contact height by r_o (1 - cos) ~ 1e-11 m)
    assert (1 - s) * r.node_pos[e, 1] + s * r.node_pos[e + 1, 1] == pytest.approx(g, rel=1e-5)
