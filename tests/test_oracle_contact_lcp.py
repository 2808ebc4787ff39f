"""Pins of the oracle's collision detection (Eq. 3-10, Sec. III.C) and contact LCP (Eq. 12-13, 22-23):
dense sampling, constructed Voronoi regions, plane/crease/ridge closed forms, brute-force
enumeration of complementary sets."""
import numpy as np
import pytest

import workloads as wl
from oracle import contact, lcp


def _tri_samples(a, b, c, n):
    u = np.linspace(0, 1, n)
    U, V = np.meshgrid(u, u)
    m = U + V <= 1
    U, V = U[m], V[m]
    return a[None] + U[:, None] * (b - a)[None] + V[:, None] * (c - a)[None]


def test_closest_point_vs_dense_sampling():
    rng = np.random.default_rng(10)
    for _ in range(20):
        a, b, c = rng.normal(size=(3, 3))
        S = _tri_samples(a, b, c, 600)
        for _ in range(5):
            p = rng.normal(size=3) * 1.5
            q = contact.closest_point_on_triangle(p, a, b, c)
            d = np.linalg.norm(p - q)
            ds = np.linalg.norm(S - p[None], axis=1).min()
            h = max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(c - b)) / 599
            assert d <= ds + 1e-12
            assert d >= ds - 2 * h
            # q lies on the triangle: non-negative barycentric coordinates, in plane
            M = np.column_stack([b - a, c - a])
            vw, *_ = np.linalg.lstsq(M, q - a, rcond=None)
            assert vw.min() >= -1e-12 and vw.sum() <= 1 + 1e-12
            assert np.linalg.norm(M @ vw - (q - a)) <= 1e-12


def test_closest_point_all_seven_regions():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    cases = [((-1, -1, 0.3), a), ((2, -0.5, 1), b), ((-0.5, 2, -1), c),
             ((0.5, -1, 0.2), (0.5, 0, 0)), ((-1, 0.4, 0.7), (0, 0.4, 0)), ((1, 1, 0.5), (0.5, 0.5, 0)),
             ((0.2, 0.3, 0.9), (0.2, 0.3, 0))]
    for p, q in cases:
        assert np.allclose(contact.closest_point_on_triangle(np.array(p, float), a, b, c), q, atol=1e-15)
    P = np.array([p for p, _ in cases], float)
    for p, q in cases:
        cp, d, inside, _ = contact.closest_points_all(np.array(p, float), a[None], b[None], c[None])
        assert np.allclose(cp[0], q, atol=1e-15)
        assert inside[0] == (p == (0.2, 0.3, 0.9))


def test_vectorised_matches_scalar():
    rng = np.random.default_rng(11)
    A, B, C = rng.normal(size=(3, 200, 3))
    for _ in range(20):
        p = rng.normal(size=3)
        cp, d, _, _ = contact.closest_points_all(p, A, B, C)
        for t in range(0, 200, 17):
            q = contact.closest_point_on_triangle(p, A[t], B[t], C[t])
            assert np.allclose(cp[t], q, atol=1e-13)


def test_plane_wall_closed_form():
    """A node at height h over a flat wall: one face constraint n = wall normal, gap = h - r_o."""
    lum = wl.plane_lumen(point=(0.05, 0.01, 0.0), normal=(0.0, 1.0, 0.0), size=0.2, n=6)
    V, T = lum.vertices, lum.triangles
    r_o, act = 2e-3, 1e-3
    for h in (0.5e-3, 2.0e-3, 2.9e-3, 3.1e-3):
        p = np.array([0.0123, 0.01 - h, 0.0071])
        recs = contact.detect_node(p, V, T, r_o, act)
        if h <= r_o + act:
            assert len(recs) == 1
            assert np.allclose(recs[0]["normal"], [0, 1, 0], atol=1e-15)
            assert recs[0]["gap"] == pytest.approx(h - r_o, abs=1e-15)
            assert np.allclose(recs[0]["point"], [0.0123, 0.01, 0.0071], atol=1e-15)
        else:
            assert recs == []
    # penetrated node: same plane, negative gap
    p = np.array([0.0123, 0.01 + 0.5e-3, 0.0])
    recs = contact.detect_node(p, V, T, r_o, act)
    assert len(recs) == 1 and recs[0]["gap"] == pytest.approx(-0.5e-3 - r_o, abs=1e-15)


def test_crease_and_ridge_explicit():
    """Valley (concave crease seen from the lumen): both face planes; ridge (convex edge):
    one edge constraint with n along c - p (both faces reach the ridge point within the band,
    and rows with the same closest point are one)."""
    ca, sa = np.cos(0.3), np.sin(0.3)
    V = np.array([[0, 0, -1.0], [0, 0, 1.0], [ca, sa, 0.0], [-ca, sa, 0.0]])
    T = np.array([[0, 2, 1], [0, 1, 3]], np.int32)
    nf = contact.face_normals(V, T)
    assert nf[0, 1] < 0 and nf[1, 1] < 0          # outward = below the valley surface
    p = np.array([0.0, 0.25, 0.0])
    recs = contact.detect_node(p, V, T, 0.2, 0.2, nf)
    assert len(recs) == 2 and all(r["face"] for r in recs)
    for r, n in zip(recs, nf):
        assert np.allclose(r["normal"], n, atol=1e-15)
        assert r["gap"] == pytest.approx(abs(np.dot(n, p - V[0])) - 0.2, abs=1e-15)
    V2 = np.array([[0, 0, -1.0], [0, 0, 1.0], [ca, -sa, 0.0], [-ca, -sa, 0.0]])
    T2 = np.array([[0, 2, 1], [0, 1, 3]], np.int32)
    nf2 = contact.face_normals(V2, T2)
    assert nf2[0, 1] < 0 and nf2[1, 1] < 0
    p2 = np.array([0.0, 0.3, 0.0])
    recs2 = contact.detect_node(p2, V2, T2, 0.2, 0.2, nf2)
    assert len(recs2) == 1 and not recs2[0]["face"]
    assert np.allclose(recs2[0]["point"], [0, 0, 0], atol=1e-15)
    assert np.allclose(recs2[0]["normal"], [0, -1, 0], atol=1e-15)
    assert recs2[0]["gap"] == pytest.approx(0.3 - 0.2, abs=1e-15)


def test_face_band_rows_closed_form():
    """Two coplanar triangles sharing the diagonal of the unit square (z = 0).  A node over the
    first triangle within the barycentric band of the second has two rows: the first face's plane
    (foot of the perpendicular) and the second triangle's edge point (projection onto the shared
    diagonal, normal along c - p); farther from the diagonal it has the face row only."""
    V = np.array([[0, 0, 0.0], [1, 0, 0.0], [1, 1, 0.0], [0, 1, 0.0]])
    T = np.array([[0, 2, 1], [0, 3, 2]], np.int32)      # outward normal -z (the node is at z > 0)
    nf = contact.face_normals(V, T)
    assert np.allclose(nf, [[0, 0, -1], [0, 0, -1]])
    p = np.array([0.5, 0.45, 0.2])                       # second triangle's coordinate w = -0.05
    recs = contact.detect_node(p, V, T, 0.15, 0.1, nf)
    assert [r["tri"] for r in recs] == [0, 1]
    assert recs[0]["face"] and np.allclose(recs[0]["point"], [0.5, 0.45, 0.0], atol=1e-15)
    assert recs[0]["gap"] == pytest.approx(0.2 - 0.15, abs=1e-15)
    c = np.array([0.475, 0.475, 0.0])
    assert not recs[1]["face"] and np.allclose(recs[1]["point"], c, atol=1e-15)
    dist = np.linalg.norm(c - p)
    assert np.allclose(recs[1]["normal"], (c - p) / dist, atol=1e-15)
    assert recs[1]["gap"] == pytest.approx(dist - 0.15, abs=1e-15)
    p2 = np.array([0.5, 0.3, 0.2])                       # w = -0.2: outside the band
    recs2 = contact.detect_node(p2, V, T, 0.15, 0.1, nf)
    assert [r["tri"] for r in recs2] == [0] and recs2[0]["face"]


def test_detect_matches_naive_loop_on_small_mesh():
    """P10: brute force over a small random tube mesh with a plain per-triangle loop."""
    pts = wl.bent_tube_centerline(straight=0.01, arc_angle=0.5, bend_radius=0.02, ds=0.002)
    V, T, _, _ = wl.tube_mesh(pts, 0.005, 8)
    rng = np.random.default_rng(12)
    nf = contact.face_normals(V, T)
    for _ in range(40):
        p = pts[rng.integers(len(pts))] + rng.normal(size=3) * 0.002
        recs = contact.detect_node(p, V, T, 0.002, 0.001, nf)
        # naive: scalar closest point per triangle
        best = min(range(len(T)), key=lambda t: (np.linalg.norm(p - contact.closest_point_on_triangle(p, *V[T[t]])), t))
        cps = [contact.closest_point_on_triangle(p, *V[T[t]]) for t in range(len(T))]
        d = [np.linalg.norm(p - q) for q in cps]
        expect = []
        for t in range(len(T)):
            if d[t] > 0.003:
                continue
            # over the face: barycentric coordinates of the plane projection, each >= -FACE_BAND
            a0, a1, a2 = V[T[t, 0]], V[T[t, 1]], V[T[t, 2]]
            proj = p - np.dot(nf[t], p - a0) * nf[t]
            G = np.array([[np.dot(a1 - a0, a1 - a0), np.dot(a1 - a0, a2 - a0)],
                          [np.dot(a1 - a0, a2 - a0), np.dot(a2 - a0, a2 - a0)]])
            bv, bw = np.linalg.solve(G, [np.dot(a1 - a0, proj - a0), np.dot(a2 - a0, proj - a0)])
            band = contact.FACE_BAND
            over = bv >= -band and bw >= -band and 1.0 - bv - bw >= -band
            if over or t == best:
                if not any(np.linalg.norm(cps[t] - cps[u]) <= 1e-12 for u in expect):
                    expect.append(t)
        # triangle ids may differ only where several triangles share the closest point
        got = np.array([r["point"] for r in recs]).reshape(-1, 3)
        exp = np.array([cps[t] for t in expect]).reshape(-1, 3)
        assert got.shape == exp.shape and np.allclose(got, exp, atol=1e-12)


def test_detect_prefilter_equals_all_triangles():
    """detect tests each node only against the triangles whose bounding sphere reaches the
    activation distance: the rows (triangle, point, normal, gap) equal the all-triangle test of
    detect_node, for nodes near, on, beyond and far from the wall of a bent tube."""
    pts = wl.bent_tube_centerline(straight=0.01, arc_angle=0.5, bend_radius=0.02, ds=0.002)
    V, T, _, _ = wl.tube_mesh(pts, 0.005, 8)
    nf = contact.face_normals(V, T)
    rng = np.random.default_rng(31)
    x = np.array([pts[rng.integers(len(pts))] + rng.normal(size=3) * s
                  for s in (0.0005, 0.002, 0.004, 0.006, 0.02) for _ in range(12)])
    got = contact.detect(x, range(len(x)), V, T, 0.002, 0.001)
    exp = []
    for i in range(len(x)):
        for r in contact.detect_node(x[i], V, T, 0.002, 0.001, nf):
            r["node"] = i
            exp.append(r)
    assert len(exp) > 20 and len(got) == len(exp)
    for a, b in zip(got, exp):
        assert (a["node"], a["tri"]) == (b["node"], b["tri"])
        assert np.array_equal(a["point"], b["point"]) and np.array_equal(a["normal"], b["normal"])
        assert a["gap"] == b["gap"]


def _spd(rng, m):
    X = rng.normal(size=(m, m + 2))
    return X @ X.T / m + 0.05 * np.eye(m)


def test_murty_matches_enumeration():
    """P11: the LCP with SPD W has exactly one solution; pivoting finds it."""
    rng = np.random.default_rng(13)
    for m in range(1, 9):
        for _ in range(6):
            W = _spd(rng, m)
            q = rng.normal(size=m)
            sols = lcp.enumerate_lcp(W, q)
            assert len(sols) == 1
            y, w, _ = lcp.murty(W, q)
            assert np.allclose(y, sols[0][0], atol=1e-12)
            ww = W @ y + q
            assert y.min() >= 0 and ww.min() >= -1e-12 and abs(y @ ww) <= 1e-12


def test_qp_nnls_matches_murty_and_enumeration():
    """The QP (NNLS) form returns the unique LCP solution found by pivoting and enumeration."""
    rng = np.random.default_rng(15)
    for m in range(1, 9):
        for _ in range(6):
            W = _spd(rng, m)
            q = rng.normal(size=m)
            y, w, _ = lcp.qp_nnls(W, q)
            ye = lcp.enumerate_lcp(W, q)[0][0]
            assert np.allclose(y, ye, atol=1e-12)
    for m in (20, 60):
        W = _spd(rng, m)
        q = rng.normal(size=m)
        y, _, _ = lcp.qp_nnls(W, q)
        ym, _, _ = lcp.murty(W, q)
        assert np.allclose(y, ym, atol=1e-11)


def test_murty_kkt_larger():
    rng = np.random.default_rng(14)
    for m in (20, 60):
        W = _spd(rng, m)
        q = rng.normal(size=m)
        y, w, piv = lcp.murty(W, q)
        ww = W @ y + q
        assert y.min() >= 0 and ww.min() >= -1e-11 and np.abs(np.minimum(y, ww)).max() <= 1e-11


def test_admm_polish_matches_enumeration_and_pivoting():
    """OSQP-style ADMM on the contact-space QP, then the exact polish on its guess of the free rows:
    the unique LCP solution (enumeration for m <= 10, Murty's pivoting beyond), and the polish
    accepts the ADMM guess without falling back."""
    rng = np.random.default_rng(17)
    fallbacks = 0
    for m in list(range(1, 11)) + [20, 40]:
        for _ in range(5):
            W = _spd(rng, m)
            q = rng.normal(size=m)
            y, w, it, polished = lcp.admm_polish(W, q)
            ye = lcp.enumerate_lcp(W, q)[0][0] if m <= 10 else lcp.murty(W, q)[0]
            assert np.allclose(y, ye, atol=1e-11), (m, np.abs(y - ye).max())
            assert y.min() >= 0 and w.min() >= -1e-11 and abs(y @ w) <= 1e-10
            fallbacks += not polished
    assert fallbacks == 0


def test_admm_iterates_approach_the_solution():
    """The ADMM iterates themselves converge: at tighter tolerances y and z approach the exact
    solution and the multiplier lam approaches -w (the slack of the bound y >= 0)."""
    rng = np.random.default_rng(18)
    for m in (5, 12, 30):
        W = _spd(rng, m)
        q = rng.normal(size=m)
        ye, we, _ = lcp.murty(W, q)
        errs = []
        for eps in (1e-2, 1e-4, 1e-6):
            y, z, lam, _ = lcp.admm(W, q, eps_rel=eps, max_iter=100000)
            errs.append(np.abs(z - ye).max())
            assert np.abs(lam + we).max() <= 100 * eps * max(1.0, np.abs(q).max())
        assert errs[-1] <= 1e-4 * max(1.0, np.abs(ye).max()) and errs[-1] <= errs[0]


def test_primal_admm_on_eq23_matches_the_contact_space_solution():
    """OSQP's ADMM on the primal QP of Eq. 23 (variables dx, rows A dx <= b), polished exactly: the
    step and the multipliers of the exact contact-space solution; its iterates themselves approach
    it as the tolerance tightens."""
    rng = np.random.default_rng(19)
    for trial in range(25):
        n = int(rng.integers(4, 30))
        m = int(rng.integers(1, min(n, 12) + 1))
        X = rng.normal(size=(n, n + 3))
        K = X @ X.T / n + 0.1 * np.eye(n)
        g = rng.normal(size=n)
        A = rng.normal(size=(m, n))
        b = rng.normal(size=m) * 0.3
        rho = 0.1 * np.max(np.diag(K))
        Mi = np.linalg.inv(K + 1e-6 * np.eye(n) + rho * A.T @ A)
        Xk = np.linalg.solve(K, A.T)
        dxf = -np.linalg.solve(K, g)
        W = A @ Xk
        q = b - A @ dxf
        y, it, polished = lcp.primal_admm_polish(lambda r: Mi @ r, lambda v: K @ v, g, A, b, rho, W, q)
        ye = lcp.murty(W, q)[0]
        assert np.allclose(y, ye, atol=1e-10), trial
        dx = dxf - Xk @ y
        assert (A @ dx <= b + 1e-10).all()
        if trial < 5:
            xs, zs, lams, _ = lcp.primal_admm(lambda r: Mi @ r, lambda v: K @ v, g, A, b, rho, eps_rel=1e-9,
                                              max_iter=200000)
            assert np.abs(xs - (dxf - Xk @ ye)).max() <= 1e-6 * max(1.0, np.abs(dx).max())
            assert np.abs(lams - ye).max() <= 1e-6 * max(1.0, np.abs(ye).max())


def test_primal_admm_adaptive_rho():
    """OSQP's adaptive rho (refactor given): on problems whose K spans six decades on its diagonal
    (translational against rotational stiffness), the iterates still converge to the exact solution,
    in far fewer iterations than with the fixed rho = 0.1 max diag K, and rho is changed only by
    factors beyond 5."""
    rng = np.random.default_rng(23)
    fixed = adapt = 0
    for trial in range(10):
        n = int(rng.integers(12, 30))
        m = int(rng.integers(2, 8))
        sc = 10.0 ** rng.uniform(-3, 3, size=n)
        X = rng.normal(size=(n, n + 3))
        K = (X @ X.T / n + 0.1 * np.eye(n)) * np.sqrt(np.outer(sc, sc))
        g = rng.normal(size=n) * np.sqrt(sc)
        A = rng.normal(size=(m, n))
        b = rng.normal(size=m) * 0.3
        rho0 = 0.1 * np.max(np.diag(K))
        rhos = []

        def factor(rho):
            rhos.append(rho)
            Mi = np.linalg.inv(K + 1e-6 * np.eye(n) + rho * A.T @ A)
            return lambda r: Mi @ r
        Xk = np.linalg.solve(K, A.T)
        dxf = -np.linalg.solve(K, g)
        ye = lcp.murty(A @ Xk, b - A @ dxf)[0]
        x1, _, l1, it1 = lcp.primal_admm(factor(rho0), lambda v: K @ v, g, A, b, rho0, eps_rel=1e-6, max_iter=100000)
        rhos.clear()
        x2, _, l2, it2 = lcp.primal_admm(factor(rho0), lambda v: K @ v, g, A, b, rho0, eps_rel=1e-6, max_iter=100000,
                                         refactor=factor)
        for r0, r1 in zip(rhos, rhos[1:]):
            assert r1 > 5.0 * r0 or r1 < r0 / 5.0
        assert np.abs(l2 - ye).max() <= 1e-3 * max(1.0, np.abs(ye).max()), trial
        xe = dxf - Xk @ ye                        # in the energy norm: K's scales span six decades
        ex = x2 - xe
        assert np.sqrt(ex @ K @ ex) <= 1e-3 * np.sqrt(xe @ K @ xe), trial
        fixed += it1
        adapt += it2
    assert adapt < fixed / 2, (adapt, fixed)


def test_solver_with_primal_admm_equals_the_default():
    """The Newton solve with the primal ADMM as its QP solver reaches the same states in the same
    iterations as with the exact contact-space solver (bent tube, contacts from step 5)."""
    from oracle import solver
    w = wl.bent_tube_workload(0, n_steps=10)
    a = solver.Model(w.robot, w.lumen)
    b = solver.Model(w.robot, w.lumen, solver.Options(qp_solver="primal_admm"))
    rows = 0
    for s in range(len(w.insertions)):
        ra = a.solve(w.tensions[s], w.insertions[s])
        rb = b.solve(w.tensions[s], w.insertions[s])
        assert ra.status == rb.status == solver.OK and ra.newton_iters == rb.newton_iters, s
        assert np.abs(ra.node_pos - rb.node_pos).max() <= 1e-12 * np.abs(ra.node_pos).max(), s
        rows += len(rb.contacts)
    assert rows > 0
