"""Seeded synthetic inputs for the contact-FEM hot path (robot, lumen mesh, loads).

This module holds geometry and random draws only -- none of the method's
arithmetic (no element, contact or solver code).  Both the CPU oracle and the
CUDA path consume what it produces, so that the two sides see bit-identical
inputs.  Every draw uses ``numpy.random.default_rng(seed)``.

Workloads (sizes follow the paper's scale, Sec. IV.A: 100-400 nodes; the
bronchial MRI mesh of the paper is not available, synthetic tubes stand in):

* ``bent_tube_workload``  -- 120 mm rod, 20 elements, tube r = 5 mm made of a
  40 mm straight run and a 90 deg arc of bend radius 60 mm, 24 around x 1 mm
  axial; insertion 0 -> 100 mm; tensions U[0, 3] N.
* ``catmull_rom_workload`` -- 600 mm rod, 300 elements, tube r = 6 mm around a
  uniform Catmull-Rom centreline through 10 points 70 mm apart along x with
  lateral offsets U[-25, 25] mm, 48 around x 1 mm axial; insertion swept
  0 -> 600 mm in 60 steps; tensions U[0, 5] N per step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "RobotDesc", "LumenDesc", "Workload", "robot_desc", "tube_mesh",
    "bent_tube_centerline", "catmull_rom_centerline", "bent_tube_workload",
    "catmull_rom_workload", "plane_lumen", "random_tensions", "soft_tip_moduli", "with_soft_tip",
]


@dataclass
class RobotDesc:
    """Robot geometry and material (Sec. II.A-B; section constants are derived by each side)."""
    length: float
    outer_radius: float
    inner_radius: float
    youngs_modulus: float
    poisson_ratio: float
    n_elements: int
    n_cables: int = 3
    cable_radius: float = 1.5e-3
    cable_angles: np.ndarray = field(default_factory=lambda: np.array([0.0, 2 * math.pi / 3, 4 * math.pi / 3]))
    element_youngs: np.ndarray | None = None   # (n_elements,) per-element modulus, base to tip; None = uniform


@dataclass
class LumenDesc:
    """Triangle soup of the lumen wall (outward winding) and the clamp frame at its entrance."""
    vertices: np.ndarray          # (V, 3) float64, metres
    triangles: np.ndarray         # (T, 3) int32, counter-clockwise seen from outside the lumen
    entrance_point: np.ndarray    # (3,)
    entrance_dir: np.ndarray      # (3,) unit, insertion direction
    entrance_up: np.ndarray       # (3,) unit, orthogonal to entrance_dir


@dataclass
class Workload:
    name: str
    robot: RobotDesc
    lumen: LumenDesc
    insertions: np.ndarray        # (S,) insertion depth per solve, metres
    tensions: np.ndarray          # (S, n_cables) cable tension per solve, newtons


def robot_desc(length, n_elements, outer_radius=2e-3, inner_radius=1e-3, youngs_modulus=2.0e9,
               poisson_ratio=0.35, cable_radius=1.5e-3) -> RobotDesc:
    return RobotDesc(length=float(length), outer_radius=float(outer_radius), inner_radius=float(inner_radius),
                     youngs_modulus=float(youngs_modulus), poisson_ratio=float(poisson_ratio),
                     n_elements=int(n_elements), cable_radius=float(cable_radius))


def soft_tip_moduli(robot: RobotDesc, soft_length=0.07, soft_ratio=0.1) -> np.ndarray:
    """Per-element Young's moduli of a robot whose distal soft_length (70 mm on the robot of Sec. II.A)
    is softer by soft_ratio (the paper gives no value; 0.1 is this generator's choice).  An element
    is soft when its midpoint lies within soft_length of the tip."""
    M, l0 = robot.n_elements, robot.length / robot.n_elements
    mid = (np.arange(M) + 0.5) * l0
    E = np.full(M, robot.youngs_modulus)
    E[mid > robot.length - soft_length] *= soft_ratio
    return E


def with_soft_tip(robot: RobotDesc, soft_length=0.07, soft_ratio=0.1) -> RobotDesc:
    """A copy of robot with the soft distal section of soft_tip_moduli."""
    from dataclasses import replace
    return replace(robot, element_youngs=soft_tip_moduli(robot, soft_length, soft_ratio))


def _rmf(points: np.ndarray, t0_normal: np.ndarray):
    """Rotation-minimising frames along a polyline by the double-reflection rule
    (Wang, Juettler, Zheng, Liu 2008).  Returns tangents and normals per point."""
    n = len(points)
    tang = np.zeros_like(points)
    d = np.diff(points, axis=0)
    tang[1:-1] = points[2:] - points[:-2]
    tang[0] = d[0]
    tang[-1] = d[-1]
    tang /= np.linalg.norm(tang, axis=1, keepdims=True)
    norm = np.zeros_like(points)
    r0 = t0_normal - np.dot(t0_normal, tang[0]) * tang[0]
    norm[0] = r0 / np.linalg.norm(r0)
    for i in range(n - 1):
        v1 = points[i + 1] - points[i]
        c1 = np.dot(v1, v1)
        rl = norm[i] - (2.0 / c1) * np.dot(v1, norm[i]) * v1
        tl = tang[i] - (2.0 / c1) * np.dot(v1, tang[i]) * v1
        v2 = tang[i + 1] - tl
        c2 = np.dot(v2, v2)
        r = rl - (2.0 / c2) * np.dot(v2, rl) * v2 if c2 > 1e-30 else rl
        r = r - np.dot(r, tang[i + 1]) * tang[i + 1]
        norm[i + 1] = r / np.linalg.norm(r)
    return tang, norm


def tube_mesh(points: np.ndarray, radius: float, n_around: int, t0_normal=(0.0, 1.0, 0.0)):
    """Open tube of circular section around a sampled centreline.

    Ring k has ``n_around`` vertices at ``c_k + r (cos(phi) N_k + sin(phi) B_k)``;
    quads between rings are split into two triangles wound counter-clockwise
    when seen from outside (outward normals)."""
    points = np.asarray(points, dtype=np.float64)
    tang, norm = _rmf(points, np.asarray(t0_normal, dtype=np.float64))
    binorm = np.cross(tang, norm)
    phi = 2.0 * math.pi * np.arange(n_around) / n_around
    cph, sph = np.cos(phi), np.sin(phi)
    verts = (points[:, None, :] + radius * (cph[None, :, None] * norm[:, None, :]
                                             + sph[None, :, None] * binorm[:, None, :]))
    verts = verts.reshape(-1, 3)
    K = len(points)
    tris = []
    for k in range(K - 1):
        for j in range(n_around):
            a = k * n_around + j
            b = (k + 1) * n_around + j
            c = (k + 1) * n_around + (j + 1) % n_around
            d = k * n_around + (j + 1) % n_around
            tris.append((a, d, c))
            tris.append((a, c, b))
    return verts, np.asarray(tris, dtype=np.int32), tang, norm


def bent_tube_centerline(straight=0.040, arc_angle=math.pi / 2, bend_radius=0.060, ds=0.001):
    """Centreline: straight run along +x from the origin, then a circular arc bending towards +y."""
    n_s = int(round(straight / ds))
    pts = [np.array([i * ds, 0.0, 0.0]) for i in range(n_s + 1)]
    arc_len = arc_angle * bend_radius
    n_a = int(math.ceil(arc_len / ds))
    for i in range(1, n_a + 1):
        a = arc_angle * i / n_a
        pts.append(np.array([straight + bend_radius * math.sin(a), bend_radius * (1 - math.cos(a)), 0.0]))
    return np.asarray(pts)


def catmull_rom_centerline(seed: int, n_points=10, spacing=0.070, max_offset=0.025, ds=0.001):
    """Uniform Catmull-Rom curve through ``n_points`` control points ``spacing`` apart along x
    with lateral (y, z) offsets U[-max_offset, max_offset] (the first point sits at the origin),
    resampled every ``ds`` of arc length."""
    rng = np.random.default_rng(seed)
    P = np.zeros((n_points, 3))
    P[:, 0] = spacing * np.arange(n_points)
    P[1:, 1:] = rng.uniform(-max_offset, max_offset, size=(n_points - 1, 2))
    ext = np.vstack([2 * P[0] - P[1], P, 2 * P[-1] - P[-2]])
    dense = []
    sub = 400
    for i in range(1, n_points):
        p0, p1, p2, p3 = ext[i - 1], ext[i], ext[i + 1], ext[i + 2]
        for s in range(sub):
            t = s / sub
            dense.append(0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t
                                + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3))
    dense.append(P[-1])
    dense = np.asarray(dense)
    seg = np.linalg.norm(np.diff(dense, axis=0), axis=1)
    arc = np.concatenate([[0.0], np.cumsum(seg)])
    n_out = int(arc[-1] / ds)
    targets = ds * np.arange(n_out + 1)
    out = np.stack([np.interp(targets, arc, dense[:, k]) for k in range(3)], axis=1)
    return out


def _lumen_from_centerline(points, radius, n_around, up=(0.0, 1.0, 0.0)) -> LumenDesc:
    verts, tris, tang, norm = tube_mesh(points, radius, n_around, up)
    return LumenDesc(vertices=verts, triangles=tris, entrance_point=points[0].copy(),
                     entrance_dir=tang[0].copy(), entrance_up=norm[0].copy())


def random_tensions(seed: int, n_steps: int, t_max: float, n_cables: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, t_max, size=(n_steps, n_cables))


def bent_tube_workload(tension_seed: int = 0, n_steps: int = 10, insertion=0.100, n_elements=20,
                       length=0.120) -> Workload:
    """120 mm rod in a 5 mm tube with a 90 deg bend; insertion ramps to 100 mm in ``n_steps``
    equal steps under one seeded tension triple U[0, 3] N."""
    robot = robot_desc(length, n_elements)
    lumen = _lumen_from_centerline(bent_tube_centerline(), 0.005, 24)
    ins = insertion * np.arange(1, n_steps + 1) / n_steps
    t = random_tensions(tension_seed, 1, 3.0)
    return Workload("bent_tube_120mm_M%d" % n_elements, robot, lumen, ins, np.repeat(t, n_steps, axis=0))


def catmull_rom_workload(lumen_seed: int = 1, tension_seed: int = 2, n_steps: int = 60, length=0.600,
                         n_elements=300, max_insertion=None) -> Workload:
    """600 mm rod, 300 elements, in a 6 mm Catmull-Rom tube; insertion swept 0 -> 600 mm in
    ``n_steps`` warm-started steps with a fresh seeded tension triple U[0, 5] N per step."""
    robot = robot_desc(length, n_elements)
    lumen = _lumen_from_centerline(catmull_rom_centerline(lumen_seed), 0.006, 48)
    top = length if max_insertion is None else max_insertion
    ins = top * np.arange(1, n_steps + 1) / n_steps
    t = random_tensions(tension_seed, n_steps, 5.0)
    return Workload("catmull_rom_600mm_M%d" % n_elements, robot, lumen, ins, t)


def _straight_tube(start, d, length, radius, n_around, ds, back=0.0):
    """Tube mesh (as tube_mesh, vectorised) around the straight axis from start - back d to
    start + length d, rings every ds."""
    n = max(int(math.ceil((length + back) / ds)), 1)
    ts = -back + (length + back) * np.arange(n + 1) / n
    pts = start[None, :] + ts[:, None] * d[None, :]
    up = np.cross(d, [0.0, 0.0, 1.0])
    if np.linalg.norm(up) < 1e-6:
        up = np.cross(d, [0.0, 1.0, 0.0])
    up /= np.linalg.norm(up)
    bi = np.cross(d, up)
    phi = 2.0 * math.pi * np.arange(n_around) / n_around
    ring = np.cos(phi)[:, None] * up[None, :] + np.sin(phi)[:, None] * bi[None, :]
    verts = (pts[:, None, :] + radius * ring[None, :, :]).reshape(-1, 3)
    k = np.arange(n)[:, None]
    j = np.arange(n_around)[None, :]
    a_ = k * n_around + j
    b_ = (k + 1) * n_around + j
    c_ = (k + 1) * n_around + (j + 1) % n_around
    d_ = k * n_around + (j + 1) % n_around
    tris = np.stack([np.stack([a_, d_, c_], -1), np.stack([a_, c_, b_], -1)], axis=2).reshape(-1, 3)
    return verts, tris.astype(np.int32)


def _tree_segments(seed, radii):
    """Seeded 3-generation binary tree of straight segments: a root along +x from the origin; each
    segment ends in two children turned by U[25, 45] deg from its axis, on either side of a random
    plane through it; lengths U[60, 120] mm; radius by generation.  Entries (start, unit direction,
    length, radius, parent index)."""
    rng = np.random.default_rng(seed)
    segs = []

    def add(start, d, gen, parent):
        length = rng.uniform(0.060, 0.120)
        segs.append((start, d, length, radii[gen], parent))
        me = len(segs) - 1
        if gen < len(radii) - 1:
            end = start + length * d
            a = np.cross(d, rng.normal(size=3))
            a /= np.linalg.norm(a)
            for sgn in (1.0, -1.0):
                ang = math.radians(rng.uniform(25.0, 45.0))
                add(end, math.cos(ang) * d + sgn * math.sin(ang) * a, gen + 1, me)

    add(np.zeros(3), np.array([1.0, 0.0, 0.0]), 0, -1)
    return segs


def _capsule_field(segs, root_back):
    """Signed distance-like field of the lumen, the union of one capsule per segment (the set of
    points within the segment's radius of its axis segment): f(x) = min_j (|x - proj_j(x)| - r_j),
    negative inside.  The root capsule starts root_back before the origin, so the entrance plane
    x = 0 cuts a straight stretch.  Returns f(points) -> (values, gradients)."""
    A = np.array([s[0] - (root_back if s[4] < 0 else 0.0) * s[1] for s in segs])
    D = np.array([s[1] for s in segs])
    Lj = np.array([s[2] + (root_back if s[4] < 0 else 0.0) for s in segs])
    R = np.array([s[3] for s in segs])

    def f(P):
        best = np.full(len(P), np.inf)
        grad = np.zeros_like(P)
        for a, d, l, r in zip(A, D, Lj, R):
            t = np.clip((P - a) @ d, 0.0, l)
            q = a[None, :] + t[:, None] * d[None, :]
            v = P - q
            dist = np.linalg.norm(v, axis=1)
            val = dist - r
            upd = val < best
            best = np.where(upd, val, best)
            grad[upd] = v[upd] / np.maximum(dist[upd], 1e-300)[:, None]
        return best, grad
    return f, A, D, Lj, R


def branching_tree_lumen(seed: int = 3, radii=(0.008, 0.0055, 0.004), h=0.00038, root_back=0.030, entrance_cut=0.020):
    """Seeded 3-generation binary tube tree (segments as _tree_segments), meshed as one closed
    surface: the boundary of the union of the segments' capsules (hemispherical ends, so every
    junction is a clean, watertight intersection of tube walls and the leaves are capped), contoured
    by surface nets on a cubic grid of spacing h restricted to a narrow band around the tube walls:
    one vertex per grid cell that the surface crosses (the mean of its edge crossings, then moved onto
    the surface along the field's gradient), one quad (two triangles, the shorter diagonal) per grid
    edge that the surface crosses, wound outward; vertices closer than h / 10 are welded and the
    slivers left dropped.  The root starts root_back before the origin and triangles behind
    x = -entrance_cut are dropped, which opens the entrance.  Returns the lumen and
    the root-to-leaf path lengths (sum of segment lengths)."""
    segs = _tree_segments(seed, radii)
    f, A, D, Lj, R = _capsule_field(segs, root_back)
    pts_all = np.concatenate([A, A + Lj[:, None] * D])
    lo = pts_all.min(axis=0) - R.max() - 3 * h
    hi = pts_all.max(axis=0) + R.max() + 3 * h
    dims = np.ceil((hi - lo) / h).astype(np.int64) + 1
    # candidate cells: centres within sqrt(3) h of some capsule wall (narrow band), tube by tube
    band = math.sqrt(3.0) * h
    cells = []
    for a, d, l, r in zip(A, D, Lj, R):
        blo = np.floor((np.minimum(a, a + l * d) - r - 2 * h - lo) / h).astype(np.int64)
        bhi = np.ceil((np.maximum(a, a + l * d) + r + 2 * h - lo) / h).astype(np.int64)
        blo = np.maximum(blo, 0)
        bhi = np.minimum(bhi, dims - 2)
        ii = np.arange(blo[0], bhi[0] + 1)
        for j0 in range(blo[1], bhi[1] + 1, 64):
            jj = np.arange(j0, min(j0 + 64, bhi[1] + 1))
            kk = np.arange(blo[2], bhi[2] + 1)
            I, J, K = np.meshgrid(ii, jj, kk, indexing="ij")
            I, J, K = I.ravel(), J.ravel(), K.ravel()
            C = lo[None, :] + (np.stack([I, J, K], axis=1) + 0.5) * h
            t = np.clip((C - a) @ d, 0.0, l)
            dist = np.linalg.norm(C - (a[None, :] + t[:, None] * d[None, :]), axis=1)
            sel = np.abs(dist - r) <= band
            cells.append((I[sel] * dims[1] + J[sel]) * dims[2] + K[sel])
    cells = np.unique(np.concatenate(cells))
    ci, cj, ck = cells // (dims[1] * dims[2]), (cells // dims[2]) % dims[1], cells % dims[2]
    # field at the cells' corners (each grid point once)
    offs = np.array([[a_, b_, c_] for a_ in (0, 1) for b_ in (0, 1) for c_ in (0, 1)])
    corner = ((ci[:, None] + offs[None, :, 0]) * dims[1] + (cj[:, None] + offs[None, :, 1])) * dims[2] \
        + (ck[:, None] + offs[None, :, 2])
    gp, inv = np.unique(corner.ravel(), return_inverse=True)
    gi, gj, gk = gp // (dims[1] * dims[2]), (gp // dims[2]) % dims[1], gp % dims[2]
    fv = np.empty(len(gp))
    for c0 in range(0, len(gp), 1 << 20):
        P = lo[None, :] + np.stack([gi[c0:c0 + (1 << 20)], gj[c0:c0 + (1 << 20)], gk[c0:c0 + (1 << 20)]], axis=1) * h
        fv[c0:c0 + (1 << 20)] = f(P)[0]
    fv[fv == 0.0] = 1e-18                     # no grid point exactly on the surface
    fc = fv[inv].reshape(-1, 8)
    cross = (fc.min(axis=1) < 0.0) & (fc.max(axis=1) > 0.0)
    cells, ci, cj, ck, fc = cells[cross], ci[cross], cj[cross], ck[cross], fc[cross]
    # one vertex per crossed cell: mean of the crossings of its 12 edges
    edges = [(a_, b_) for a_ in range(8) for b_ in range(8) if a_ < b_ and np.sum(np.abs(offs[a_] - offs[b_])) == 1]
    acc = np.zeros((len(cells), 3))
    cnt = np.zeros(len(cells))
    for a_, b_ in edges:
        fa, fb = fc[:, a_], fc[:, b_]
        m = (fa < 0.0) != (fb < 0.0)
        t = np.where(m, fa / np.where(m, fa - fb, 1.0), 0.0)
        p = offs[a_][None, :] + t[:, None] * (offs[b_] - offs[a_])[None, :]
        acc[m] += p[m]
        cnt[m] += 1
    V = lo[None, :] + (np.stack([ci, cj, ck], axis=1) + acc / cnt[:, None]) * h
    for _ in range(3):                        # onto the surface along the gradient
        val, g = f(V)
        V = V - val[:, None] * g
    # one quad per crossed grid edge; the edge from grid point (i, j, k) along axis ax is the min-corner
    # edge of cell (i, j, k), which is then crossed, and of three more cells around it
    order = np.argsort(cells)
    cells_sorted = cells[order]

    def cell_index(I, J, K):
        key = (I * dims[1] + J) * dims[2] + K
        pos = np.searchsorted(cells_sorted, key)
        pos = np.minimum(pos, len(cells_sorted) - 1)
        ok = cells_sorted[pos] == key
        return order[pos], ok

    tris = []
    f0 = fc[:, 0]
    for ax, (u, w) in enumerate(((1, 2), (2, 0), (0, 1))):
        nb = [4, 2, 1][ax]                    # corner index of the far end of the axis edge
        f1 = fc[:, nb]
        m = (f0 < 0.0) != (f1 < 0.0)
        base = np.stack([ci[m], cj[m], ck[m]], axis=1)
        inside_first = f0[m] < 0.0
        quad = []
        ok_all = np.ones(len(base), dtype=bool)
        for du, dw in ((0, 0), (-1, 0), (-1, -1), (0, -1)):
            q = base.copy()
            q[:, u] += du
            q[:, w] += dw
            idx, ok = cell_index(q[:, 0], q[:, 1], q[:, 2])
            quad.append(idx)
            ok_all &= ok
        quad = np.stack(quad, axis=1)[ok_all]
        inside_first = inside_first[ok_all]
        # counter-clockwise around +axis; reversed when the outside lies towards -axis
        quad[~inside_first] = quad[~inside_first][:, ::-1]
        a_, b_, c_, d_ = quad.T
        diag_ac = np.linalg.norm(V[a_] - V[c_], axis=1) <= np.linalg.norm(V[b_] - V[d_], axis=1)
        t1 = np.where(diag_ac[:, None], np.stack([a_, b_, c_], 1), np.stack([a_, b_, d_], 1))
        t2 = np.where(diag_ac[:, None], np.stack([a_, c_, d_], 1), np.stack([b_, c_, d_], 1))
        tris += [t1, t2]
    T = np.concatenate(tris)
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    area2 = np.linalg.norm(nrm, axis=1)
    cen = V[T].mean(axis=1)
    # drop degenerate triangles, and the few slivers folded over by the projection at the sharp ridge
    # of a carina (their winding disagrees with the field's outward gradient; each is < 0.1 mm^2)
    _, gc = f(cen)
    T = T[(area2 > 1e-16) & (np.sum(nrm * gc, axis=1) > 0.0) & (cen[:, 0] >= -entrance_cut)]
    # weld vertices closer than h / 10 (edges that short come from projections landing together at
    # creases), drop the triangles that collapse and the needles left (area below h^2 / 300): such
    # slivers make the closest-feature tests of a node flip under sub-nanometre motions
    from scipy.spatial import cKDTree
    pairs = cKDTree(V).query_pairs(0.1 * h, output_type="ndarray")
    parent = np.arange(len(V))

    def root(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for a_, b_ in pairs:
        ra, rb = root(a_), root(b_)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    rep = np.array([root(i) for i in range(len(V))])
    T = rep[T]
    ok = (T[:, 0] != T[:, 1]) & (T[:, 1] != T[:, 2]) & (T[:, 0] != T[:, 2])
    T = T[ok]
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    T = T[area >= h * h / 300.0]
    used = np.unique(T)
    remap = np.full(len(V), -1, dtype=np.int64)
    remap[used] = np.arange(len(used))
    V = V[used]
    T = remap[T].astype(np.int32)
    paths = []
    for i, (start, d, length, r, parent) in enumerate(segs):
        if any(p == i for *_x, p in segs):
            continue
        total, k = 0.0, i
        while k >= 0:
            total += segs[k][2]
            k = segs[k][4]
        paths.append(total)
    lumen = LumenDesc(vertices=V, triangles=T, entrance_point=np.zeros(3), entrance_dir=np.array([1.0, 0.0, 0.0]),
                      entrance_up=np.array([0.0, 1.0, 0.0]))
    return lumen, paths


def tree_workload(seed: int = 3, n_elements=2000, length=0.600, step=0.010, t_max=5.0) -> Workload:
    """600 mm robot in the seeded branching tube tree; the robot is longer than every root-to-leaf
    path, so the insertion is swept up to 0.9 x the shortest path in ~10 mm warm-started steps, with a
    fresh tension triple U[0, t_max] N per step."""
    lumen, paths = branching_tree_lumen(seed)
    top = 0.9 * min(paths)
    n_steps = int(math.ceil(top / step - 1e-9))
    ins = top * np.arange(1, n_steps + 1) / n_steps
    t = random_tensions(seed + 7, n_steps, t_max)
    return Workload("tree%d_M%d" % (seed, n_elements), robot_desc(length, n_elements), lumen, ins, t)


def batch_workloads(n_instances: int = 256, seed: int = 3, step=0.010, length=0.600, m_min=50, m_max=2000,
                    t_max=5.0, first=0, count=None):
    """Uneven instances for batched solves: element count log-uniform in [m_min, m_max], a lumen
    from the Catmull-Rom generator with the instance's own seed (10000 + i), a target insertion
    U[0.3, 1] x length reached by warm-started steps of about ``step``, and a fresh tension triple
    U[0, t_max] N per step.  Instances first .. first + count - 1 are generated (all by default);
    instance i is the same whatever subset is asked for."""
    rng = np.random.default_rng(seed)
    M = np.round(np.exp(rng.uniform(np.log(m_min), np.log(m_max), n_instances))).astype(int)
    target = rng.uniform(0.3, 1.0, n_instances) * length
    count = n_instances - first if count is None else count
    out = []
    for i in range(first, first + count):
        n_steps = int(np.ceil(target[i] / step - 1e-9))
        robot = robot_desc(length, int(M[i]))
        lumen = _lumen_from_centerline(catmull_rom_centerline(10000 + i), 0.006, 48)
        ins = target[i] * np.arange(1, n_steps + 1) / n_steps
        t = random_tensions(seed * 100003 + i, n_steps, t_max)
        out.append(Workload("batch%d_M%d" % (i, M[i]), robot, lumen, ins, t))
    return out


def serve_trace(start_tensions, start_insertions, lengths, rate, duration, seed=4, dt_max=0.2, dins=0.0005):
    """Poisson request stream (``rate`` requests/s for ``duration`` s) over scenes whose commands
    start at ``start_tensions`` (S, k) and ``start_insertions`` (S,): each request picks a scene
    uniformly and is, with equal probability, a tension increment U[-dt_max, dt_max] N per cable
    (tensions kept >= 0) or an insertion step of +-dins (kept within [0.3, 1] x length).  Returns
    arrival times, scene indices, and the absolute tensions and insertion each request asks for."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate * duration)
    arrivals = np.sort(rng.uniform(0.0, duration, n))
    scenes = rng.integers(0, len(start_insertions), n)
    kinds = rng.integers(0, 2, n)
    dts = rng.uniform(-dt_max, dt_max, (n, np.asarray(start_tensions).shape[1]))
    signs = rng.choice([-1.0, 1.0], n)
    ten = np.array(start_tensions, dtype=np.float64).copy()
    ins = np.array(start_insertions, dtype=np.float64).copy()
    out_t = np.zeros((n, ten.shape[1]))
    out_i = np.zeros(n)
    for k in range(n):
        sc = scenes[k]
        if kinds[k] == 0:
            ten[sc] = np.maximum(ten[sc] + dts[k], 0.0)
        else:
            ins[sc] = min(max(ins[sc] + signs[k] * dins, 0.3 * lengths[sc]), lengths[sc])
        out_t[k] = ten[sc]
        out_i[k] = ins[sc]
    return arrivals, scenes, out_t, out_i


def plane_lumen(point, normal, size=0.2, n=8, entrance_point=(0.0, 0.0, 0.0), entrance_dir=(1.0, 0.0, 0.0),
                entrance_up=(0.0, 1.0, 0.0)) -> LumenDesc:
    """A flat square wall (``n`` x ``n`` quads, two triangles each) through ``point`` with unit
    ``normal`` pointing away from the robot; used for closed-form contact checks."""
    normal = np.asarray(normal, dtype=np.float64)
    normal = normal / np.linalg.norm(normal)
    a = np.cross(normal, [1.0, 0.0, 0.0])
    if np.linalg.norm(a) < 1e-6:
        a = np.cross(normal, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(normal, a)
    g = np.linspace(-size / 2, size / 2, n + 1)
    V = np.array([np.asarray(point) + u * a + v * b for u in g for v in g])
    T = []
    for i in range(n):
        for j in range(n):
            p00, p01, p10, p11 = i * (n + 1) + j, i * (n + 1) + j + 1, (i + 1) * (n + 1) + j, (i + 1) * (n + 1) + j + 1
            for tri in ((p00, p10, p11), (p00, p11, p01)):
                e1 = V[tri[1]] - V[tri[0]]
                e2 = V[tri[2]] - V[tri[0]]
                if np.dot(np.cross(e1, e2), normal) < 0:
                    tri = (tri[0], tri[2], tri[1])
                T.append(tri)
    return LumenDesc(vertices=V, triangles=np.asarray(T, dtype=np.int32),
                     entrance_point=np.asarray(entrance_point, float), entrance_dir=np.asarray(entrance_dir, float),
                     entrance_up=np.asarray(entrance_up, float))


def free_space_lumen(entrance_point=(0.0, 0.0, 0.0), entrance_dir=(1.0, 0.0, 0.0), entrance_up=(0.0, 1.0, 0.0)) -> LumenDesc:
    """No wall at all (zero triangles): the clamp frame only, for free-space load cases."""
    return LumenDesc(vertices=np.zeros((0, 3)), triangles=np.zeros((0, 3), np.int32),
                     entrance_point=np.asarray(entrance_point, float), entrance_dir=np.asarray(entrance_dir, float),
                     entrance_up=np.asarray(entrance_up, float))


def patch_lumen(x0, x1, y, z_half=0.01, n=2) -> LumenDesc:
    """A flat rectangular wall patch in the plane y = ``y`` over x in [x0, x1], |z| <= z_half,
    outward normal +y (the robot sits below it); clamp at the origin along +x."""
    xs = np.linspace(x0, x1, n + 1)
    zs = np.linspace(-z_half, z_half, n + 1)
    V = np.array([[x, y, z] for x in xs for z in zs])
    T = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = i * (n + 1) + j, i * (n + 1) + j + 1, (i + 1) * (n + 1) + j, (i + 1) * (n + 1) + j + 1
            for tri in ((a, c, d), (a, d, b)):
                e1 = V[tri[1]] - V[tri[0]]
                e2 = V[tri[2]] - V[tri[0]]
                if np.cross(e1, e2)[1] < 0:
                    tri = (tri[0], tri[2], tri[1])
                T.append(tri)
    return LumenDesc(vertices=V, triangles=np.asarray(T, np.int32), entrance_point=np.zeros(3),
                     entrance_dir=np.array([1.0, 0.0, 0.0]), entrance_up=np.array([0.0, 1.0, 0.0]))
