"""Node-vs-triangle contact detection (Eq. 3-10; Sec. III.C "match the nodes with the triangles").

Contacts are node based: the contact point of Eq. 4 sits at xi = 0 of an element, so
N_i(0) B_i selects the translation of one node and row i of A_c is n_i^T on that node.

Per free node p, over ALL triangles (brute force), every locally closest feature within
r_o + activation gap is one constraint row (``detect_node``).  "Over the face" allows the plane
projection a barycentric margin FACE_BAND outside the triangle, so that a node near an edge shared
by two faces keeps a row for each (every triangle's distance constraint is a valid wall
constraint; the margin removes the row switching at face edges that stalls Newton iterations).  The contact normal n points
from the robot towards the far side of the wall (Eq. 3 wording) and the robot radius r_o
enters the gap of Eq. 10: b_i = n . c - n . p - r_o.
"""
import numpy as np

FACE_BAND = 0.1


def closest_point_on_triangle(p, a, b, c):
    """Closest point of triangle abc to p, by its plain definition: the orthogonal projection
    onto the plane when that projection lies in the triangle, otherwise the nearest of the
    closest points on the three edges (each a clamped projection onto a segment)."""
    p, a, b, c = (np.asarray(v, dtype=np.float64) for v in (p, a, b, c))
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n)
    proj = p - np.dot(n, p - a) * n
    # barycentric coordinates of proj: proj - a = v (b - a) + w (c - a)
    M = np.array([[np.dot(b - a, b - a), np.dot(b - a, c - a)], [np.dot(b - a, c - a), np.dot(c - a, c - a)]])
    rhs = np.array([np.dot(b - a, proj - a), np.dot(c - a, proj - a)])
    v, w = np.linalg.solve(M, rhs)
    if v >= 0 and w >= 0 and v + w <= 1:
        return proj
    best, bd = None, np.inf
    for s0, s1 in ((a, b), (b, c), (c, a)):
        e = s1 - s0
        t = min(1.0, max(0.0, np.dot(p - s0, e) / np.dot(e, e)))
        q = s0 + t * e
        d = np.linalg.norm(p - q)
        if d < bd:
            best, bd = q, d
    return best


def closest_points_all(p, A, B, C):
    """Vectorised ``closest_point_on_triangle`` over triangles (rows of A, B, C).
    Returns the closest points, distances, whether each point is interior to its face (the plane
    projection falls inside the triangle, edges included), and whether the plane projection falls
    inside the triangle enlarged by the barycentric margin FACE_BAND (all three barycentric
    coordinates >= -FACE_BAND)."""
    ab = B - A
    ac = C - A
    n = np.cross(ab, ac)
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    ap = p[None, :] - A
    proj = p[None, :] - np.sum(n * ap, axis=1, keepdims=True) * n
    m00 = np.sum(ab * ab, axis=1); m01 = np.sum(ab * ac, axis=1); m11 = np.sum(ac * ac, axis=1)
    r0 = np.sum(ab * (proj - A), axis=1); r1 = np.sum(ac * (proj - A), axis=1)
    det = m00 * m11 - m01 * m01
    v = (m11 * r0 - m01 * r1) / det
    w = (m00 * r1 - m01 * r0) / det
    inside = (v >= 0) & (w >= 0) & (v + w <= 1)
    near = (v >= -FACE_BAND) & (w >= -FACE_BAND) & (v + w <= 1 + FACE_BAND)
    best = proj.copy()
    bd = np.where(inside, np.linalg.norm(p[None, :] - proj, axis=1), np.inf)
    for S0, S1 in ((A, B), (B, C), (C, A)):
        e = S1 - S0
        t = np.clip(np.sum((p[None, :] - S0) * e, axis=1) / np.sum(e * e, axis=1), 0.0, 1.0)
        q = S0 + t[:, None] * e
        d = np.linalg.norm(p[None, :] - q, axis=1)
        upd = (~inside) & (d < bd)
        best[upd] = q[upd]
        bd = np.where(upd, d, bd)
    return best, bd, inside, near


def face_normals(V, T):
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(B - A, C - A)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def _record(p, t, c, dist, face, n_face, r_o):
    if face or dist < 1e-12:
        n = n_face                      # plane of the face, outward winding
    elif np.dot(n_face, c - p) > 0:
        n = (c - p) / dist              # edge / vertex point, node on the lumen side
    else:
        n = (p - c) / dist              # edge / vertex point, node across the wall
    return {"tri": int(t), "point": c, "normal": n, "gap": np.dot(n, c) - np.dot(n, p) - r_o,
            "dist": dist, "face": bool(face)}


def detect_node(p, V, T, r_o, activation_gap, nf=None, tri=None):
    """Contact constraints of one node against all triangles (Eq. 3, 8-10), or against the sorted
    triangle indices `tri` when given (see ``detect``).

    With c_t the closest point of triangle t, d_t = |c_t - p| and g the triangle of smallest
    d_t (lowest index on ties), the pair (node, t) is a constraint when d_t <= r_o + activation
    gap and c_t is a locally closest point of the mesh:
      * the node lies over t's face: its plane projection is inside the triangle enlarged by the
        barycentric margin FACE_BAND.  Interior projection (edges included): the face plane,
        n = outward face normal; projection in the margin: c_t on an edge, n as below;
      * t = g with c_t on an edge or a vertex (a convex feature): n along c_t - p, flipped
        to the outside when the node has crossed the wall.
    Faces meeting at a concave crease thus each contribute their plane (one plane per node
    cannot hold a node in a crease).  Pairs with the same closest point (within 1e-12 m) are
    one constraint, kept at the lowest triangle index.  Output ordered by triangle index."""
    if len(T) == 0:
        return []
    if nf is None:
        nf = face_normals(V, T)
    idx = np.arange(len(T)) if tri is None else np.asarray(tri, dtype=np.int64)
    if len(idx) == 0:
        return []
    A, B, C = V[T[idx, 0]], V[T[idx, 1]], V[T[idx, 2]]
    cp, d, inside, near = closest_points_all(p, A, B, C)
    g = int(idx[int(np.argmin(d))])
    thr = r_o + activation_gap
    recs = []
    for k in np.where(d <= thr)[0]:
        t = int(idx[k])
        if not (near[k] or t == g):
            continue
        rec = _record(p, t, cp[k], d[k], bool(inside[k]), nf[t], r_o)
        if any(np.linalg.norm(r["point"] - rec["point"]) <= 1e-12 for r in recs):
            continue
        recs.append(rec)
    return recs


def detect(positions, node_ids, V, T, r_o, activation_gap):
    """Contact constraints of the listed nodes, ordered by (node, triangle).

    A triangle lies within its bounding sphere (centroid, farthest vertex), so one whose sphere is
    farther than r_o + activation gap from the node has no point that near and gives no row; and
    the node's closest triangle g only matters when it is that near, in which case every triangle
    tied with it is kept too.  Each node is therefore tested against the triangles whose sphere
    reaches the activation distance (in increasing index order), which gives the rows of the
    all-triangle test."""
    if len(T) == 0:
        return []
    nf = face_normals(V, T)
    VT = V[T]
    cen = VT.mean(axis=1)
    rad = np.max(np.linalg.norm(VT - cen[:, None, :], axis=2), axis=1)
    thr = r_o + activation_gap
    out = []
    for i in node_ids:
        p = positions[i]
        tri = np.nonzero(np.linalg.norm(cen - p, axis=1) - rad <= thr * (1.0 + 1e-9) + 1e-12)[0]
        for rec in detect_node(p, V, T, r_o, activation_gap, nf, tri):
            rec["node"] = int(i)
            out.append(rec)
    return out
