"""Segment contacts: the contact model of Eq. 3-7 as printed (test infrastructure, like all of the
oracle).  A contact point lies anywhere on an element, at distance xi in [0, l0] from the element's
node closer to the base, and its displacement is interpolated from the element's two nodal
translations by N(xi) of Eq. 4 with the shape functions of Eq. 5-6:
    P1 = 1 - xi/l0, P2 = xi/l0 (axial, linear),  P3 = 1 - 3 xi^2/l0^2 + 2 xi^3/l0^3, P4 = 1 - P3
(transverse, cubic); B_i of Eq. 7 picks the two translations.

Reading: the paper writes N against global x, y, z, but its first row is the axial (linear) and the
other two the transverse (cubic) interpolation, which is meaningful in the element's frame.  N is
applied to the translations in the element's corotated frame R_r (e1 along the chord, the frame of
the element force):
    du(xi) = R_r N(xi) [R_r^T du_a; R_r^T du_b].
With P1 + P2 = 1 and P3 + P4 = 1, a common translation of both nodes moves the point rigidly.  The
point itself lies on the chord, p(xi) = x_a + (xi / l0) (x_b - x_a)... written with the chord
fraction s = xi / l0 of the closest point between the chord and a triangle.

Rows: per element (nodes a = e, b = e + 1, at least one free), every triangle whose closest point
to the chord is within r_o + activation gap gives a row when the chord's closest point lies over
the triangle's face (plane projection inside the triangle enlarged by the barycentric margin
FACE_BAND) or the triangle is the element's closest; rows of one element with the same pair of
closest points (1e-12 m) are merged, and a contact at a shared node (s = 1 of element e, s = 0 of
element e + 1, same wall point) is kept once, on the lower element.
"""
import numpy as np

from .contact import FACE_BAND, closest_point_on_triangle

__all__ = ["shape", "n_matrix", "closest_segment_segment", "closest_segment_triangle", "detect_elements",
           "row_weights"]


def shape(xi, l0):
    """P1..P4 of Eq. 5-6."""
    r = xi / l0
    p3 = 1.0 - 3.0 * r * r + 2.0 * r ** 3
    return 1.0 - r, r, p3, 3.0 * r * r - 2.0 * r ** 3


def n_matrix(xi, l0):
    """N(xi) of Eq. 4 (3 x 6, acting on [u_a; u_b] in the element frame)."""
    p1, p2, p3, p4 = shape(xi, l0)
    return np.array([[p1, 0.0, 0.0, p2, 0.0, 0.0],
                     [0.0, p3, 0.0, 0.0, p4, 0.0],
                     [0.0, 0.0, p3, 0.0, 0.0, p4]])


def row_weights(Rr, xi, l0):
    """The 3 x 6 map [du_a; du_b] -> du(xi) = R_r N(xi) blockdiag(R_r^T, R_r^T)."""
    E = np.zeros((6, 6))
    E[:3, :3] = Rr.T
    E[3:, 3:] = Rr.T
    return Rr @ n_matrix(xi, l0) @ E


def closest_segment_segment(p0, p1, q0, q1):
    """Closest points of segments p0p1 and q0q1 (parameters s, t in [0, 1]), by minimising the
    quadratic |p0 + s d1 - q0 - t d2|^2 over the unit square: the interior stationary point if it
    lies inside, else the best of the four edges of the square (each a clamped 1-D minimum)."""
    d1, d2, r = p1 - p0, q1 - q0, p0 - q0
    a, e, b = d1 @ d1, d2 @ d2, d1 @ d2
    c, f = d1 @ r, d2 @ r
    cands = []
    den = a * e - b * b
    if den > 1e-30 * a * e:
        s = (b * f - c * e) / den
        t = (a * f - b * c) / den
        if 0.0 <= s <= 1.0 and 0.0 <= t <= 1.0:
            cands.append((s, t))
    for s in (0.0, 1.0):                            # edges s = 0, 1: t = clamp((b s + f) / e)
        cands.append((s, min(1.0, max(0.0, (b * s + f) / e)) if e > 0 else 0.0))
    for t in (0.0, 1.0):                            # edges t = 0, 1: s = clamp((b t - c) / a)
        cands.append((min(1.0, max(0.0, (b * t - c) / a)) if a > 0 else 0.0, t))
    best = None
    for s, t in cands:
        x, y = p0 + s * d1, q0 + t * d2
        d = np.linalg.norm(x - y)
        if best is None or d < best[4]:
            best = (s, t, x, y, d)
    return best


def closest_segment_triangle(p0, p1, a, b, c):
    """Closest points of segment p0p1 and triangle abc.  Returns (s, q, w, dist, interior): s the
    segment parameter, q the segment point, w the triangle point, interior whether w is inside the
    face (not on an edge).  By the plain case split: if the segment crosses the triangle, the
    crossing point at distance 0; otherwise the minimum distance pair has a segment endpoint
    against the triangle (point-triangle closest point) or the segment against a triangle edge
    (segment-segment closest points)."""
    p0, p1, a, b, c = (np.asarray(v, dtype=np.float64) for v in (p0, p1, a, b, c))
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n)
    h0, h1 = n @ (p0 - a), n @ (p1 - a)

    def inside(x):
        M = np.array([[(b - a) @ (b - a), (b - a) @ (c - a)], [(b - a) @ (c - a), (c - a) @ (c - a)]])
        v, w = np.linalg.solve(M, np.array([(b - a) @ (x - a), (c - a) @ (x - a)]))
        return v >= 0 and w >= 0 and v + w <= 1

    if h0 * h1 < 0.0:
        s = h0 / (h0 - h1)
        x = p0 + s * (p1 - p0)
        x = x - (n @ (x - a)) * n
        if inside(x):
            return s, p0 + s * (p1 - p0), x, 0.0, True
    best = None
    for s, pt in ((0.0, p0), (1.0, p1)):
        w = closest_point_on_triangle(pt, a, b, c)
        d = np.linalg.norm(pt - w)
        if best is None or d < best[3]:
            best = (s, pt, w, d, None)
    for e0, e1 in ((a, b), (b, c), (c, a)):
        s, t, x, y, d = closest_segment_segment(p0, p1, e0, e1)
        if d < best[3]:
            best = (s, x, y, d, False)
    s, q, w, d, interior = best
    if interior is None:                             # endpoint case: inside when the projection is
        proj = q - (n @ (q - a)) * n
        interior = bool(inside(proj)) and np.linalg.norm(proj - w) <= 1e-15 * max(1.0, np.abs(w).max())
    return s, q, w, d, interior


def _near(q, a, b, c):
    """Plane projection of q inside the triangle enlarged by FACE_BAND (barycentric margin)."""
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n)
    proj = q - (n @ (q - a)) * n
    M = np.array([[(b - a) @ (b - a), (b - a) @ (c - a)], [(b - a) @ (c - a), (c - a) @ (c - a)]])
    v, w = np.linalg.solve(M, np.array([(b - a) @ (proj - a), (c - a) @ (proj - a)]))
    return v >= -FACE_BAND and w >= -FACE_BAND and 1.0 - v - w >= -FACE_BAND


def detect_elements(x, k, V, T, r_o, act, nf=None):
    """Segment rows of the elements with a free node (elements k .. M - 1 for last prescribed node k),
    over all triangles.  Each row: element, triangle, chord fraction s, segment point, wall point,
    normal n (the face normal for an interior wall point, else along the wall point minus the
    segment point, outward), gap n.c - n.q - r_o."""
    M = len(x) - 1
    if nf is None:
        A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
        nf = np.cross(B - A, C - A)
        nf = nf / np.linalg.norm(nf, axis=1, keepdims=True)
    thr = r_o + act
    # a triangle lies within its bounding sphere (centroid, farthest vertex), so one whose sphere is
    # farther than thr from the chord has no point within thr of it and gives no row: skipping it
    # changes nothing (when every triangle is farther than thr, the element has no row anyway)
    cen = V[T].mean(axis=1)
    rad = np.max(np.linalg.norm(V[T] - cen[:, None, :], axis=2), axis=1)
    rows = []
    for e in range(max(k, 0), M):
        xa, xb = x[e], x[e + 1]
        ab = xb - xa
        sc = np.clip(((cen - xa) @ ab) / (ab @ ab), 0.0, 1.0)
        dc = np.linalg.norm(cen - (xa[None, :] + sc[:, None] * ab[None, :]), axis=1)
        cands = []
        for t in np.nonzero(dc - rad <= thr * (1.0 + 1e-9) + 1e-12)[0]:
            a, b, c = V[T[t, 0]], V[T[t, 1]], V[T[t, 2]]
            s, q, w, d, interior = closest_segment_triangle(xa, xb, a, b, c)
            cands.append((d, t, s, q, w, interior, a, b, c))
        if not cands:
            continue
        gd, gt = min((cd[0], cd[1]) for cd in cands)
        kept = []
        for d, t, s, q, w, interior, a, b, c in sorted(cands, key=lambda z: z[1]):
            if d > thr or not (t == gt or _near(q, a, b, c)):
                continue
            if any(np.linalg.norm(w - r["point"]) <= 1e-12 and np.linalg.norm(q - r["robot_point"]) <= 1e-12
                   for r in kept):
                continue
            if interior or d < 1e-12:
                n = nf[t].copy()
            else:
                n = (w - q) / d
                if n @ nf[t] < 0.0:
                    n = -n
            kept.append({"elem": e, "tri": t, "s": s, "robot_point": q, "point": w, "normal": n,
                         "gap": float(n @ w - n @ q - r_o), "face": bool(interior)})
        rows.extend(kept)
    # a contact at a shared node appears on both elements: keep the lower element's row
    out = []
    for r in rows:
        if r["s"] == 0.0 and any(o["elem"] == r["elem"] - 1 and o["s"] == 1.0 and
                                 np.linalg.norm(o["point"] - r["point"]) <= 1e-12 for o in out):
            continue
        out.append(r)
    return out
