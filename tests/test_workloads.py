"""Seeded input generators: the uneven batched instances, the serving trace and the branching tube
tree (properties that hold by construction, checked on the generated data)."""
import numpy as np

import workloads as wl


def test_batch_workloads_ranges_and_subsets():
    full = wl.batch_workloads(n_instances=8)
    sub = wl.batch_workloads(n_instances=8, first=3, count=2)
    for w in full:
        assert 50 <= w.robot.n_elements <= 2000
        target = w.insertions[-1]
        assert 0.3 * 0.6 - 1e-12 <= target <= 0.6 + 1e-12
        steps = np.diff(np.concatenate([[0.0], w.insertions]))
        assert np.all(steps > 0) and np.all(steps <= 0.010 + 1e-12)
        assert np.all((w.tensions >= 0) & (w.tensions <= 5.0))
    # instance i does not depend on which subset is generated
    for a, b in zip(full[3:5], sub):
        assert a.robot.n_elements == b.robot.n_elements
        assert np.array_equal(a.insertions, b.insertions) and np.array_equal(a.tensions, b.tensions)
        assert np.array_equal(a.lumen.vertices, b.lumen.vertices)


def test_serve_trace_commands():
    t0 = np.array([[1.0, 0.1, 2.0], [0.0, 0.0, 0.0]])
    i0 = np.array([0.30, 0.50])
    L = [0.6, 0.6]
    arr, sc, ten, ins = wl.serve_trace(t0, i0, L, rate=5000.0, duration=0.2, seed=9)
    assert len(arr) > 800 and np.all(np.diff(arr) >= 0) and arr[0] >= 0 and arr[-1] <= 0.2
    assert set(np.unique(sc)) <= {0, 1}
    assert np.all(ten >= 0.0)
    for s in (0, 1):
        k = np.nonzero(sc == s)[0]
        assert np.all((ins[k] >= 0.3 * L[s] - 1e-12) & (ins[k] <= L[s] + 1e-12))
        # consecutive requests of a scene change either the tensions (by at most 0.2 N each) or the insertion
        prev_t, prev_i = t0[s], i0[s]
        for j in k:
            dt = np.abs(ten[j] - prev_t)
            di = abs(ins[j] - prev_i)
            assert (np.all(dt <= 0.2 + 1e-12) and di == 0.0) or (np.all(dt == 0.0) and di <= 0.0005 + 1e-12)
            prev_t, prev_i = ten[j], ins[j]


def test_branching_tree_lumen():
    """The tree's wall is one closed surface (coarse grid here): every edge is shared by two triangles
    with opposite orientation, except the rim of the entrance cut, pinholes left by the folded slivers
    dropped at carina ridges, and a few pinched edges where two walls come within a grid cell; every vertex lies on the union of the capsules; every triangle is
    wound outward (normal along the field's outward gradient)."""
    lumen, paths = wl.branching_tree_lumen(3, h=0.001)
    V, T = lumen.vertices, lumen.triangles.astype(np.int64)
    assert len(paths) == 4 and all(0.18 <= p <= 0.36 for p in paths)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    assert np.linalg.norm(n, axis=1).min() > 0
    E = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    und, cnt = np.unique(np.minimum(E[:, 0], E[:, 1]) * len(V) + np.maximum(E[:, 0], E[:, 1]), return_counts=True)
    rim = und[cnt == 1]
    away = np.abs(V[rim // len(V), 0] + 0.020) > 0.001               # not on the entrance cut
    # elsewhere only the pinholes of the dropped folded slivers at carina ridges: a few edges, each
    # shorter than two grid cells (far below the robot's 2 mm radius)
    assert away.sum() <= 16
    assert np.all(np.linalg.norm(V[rim[away] // len(V)] - V[rim[away] % len(V)], axis=1) <= 0.002)
    assert np.sum(cnt == 2) >= 0.995 * len(und) and np.sum(cnt > 2) <= 0.001 * len(und)
    directed, dcnt = np.unique(E[:, 0] * len(V) + E[:, 1], return_counts=True)
    assert np.sum(dcnt > 1) <= 0.001 * len(directed)
    f, *_ = wl._capsule_field(wl._tree_segments(3, (0.008, 0.0055, 0.004)), 0.030)
    val, _ = f(V)
    assert np.abs(val).max() < 1e-12
    _, g = f(V[T].mean(axis=1))
    assert np.all(np.sum(n * g, axis=1) > 0)
    # the root's straight stretch is the 8 mm tube
    cen = V[T].mean(axis=1)
    root = (cen[:, 0] > 0.005) & (cen[:, 0] < 0.040)
    assert root.sum() > 100 and np.all(np.abs(np.hypot(cen[root, 1], cen[root, 2]) - 0.008) < 2e-4)


def test_tree_workload_insertion_cap():
    w = wl.tree_workload()
    lumen, paths = wl.branching_tree_lumen(3)
    assert abs(w.insertions[-1] - 0.9 * min(paths)) < 1e-12
    assert w.robot.n_elements == 2000 and len(w.lumen.triangles) > 350000
