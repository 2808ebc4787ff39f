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
    lumen, paths = wl.branching_tree_lumen(3, n_around=16, ds=0.002)
    V, T = lumen.vertices, lumen.triangles
    assert len(paths) == 4 and all(0.18 <= p <= 0.36 for p in paths)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    area2 = np.linalg.norm(n, axis=1)
    assert area2.min() > 0
    # outward winding: the face normal points away from the nearest tube axis point of the root tube
    # for triangles of the root tube's interior stretch (x in (5, 40) mm, radius 8 mm)
    cen = V[T].mean(axis=1)
    r = np.hypot(cen[:, 1], cen[:, 2])
    root = (cen[:, 0] > 0.005) & (cen[:, 0] < 0.040) & (np.abs(r - 0.008) < 1e-3)
    assert root.sum() > 100
    radial = np.stack([np.zeros(root.sum()), cen[root, 1], cen[root, 2]], axis=1)
    assert np.all(np.sum(n[root] * radial, axis=1) > 0)


def test_tree_workload_insertion_cap():
    w = wl.tree_workload()
    lumen, paths = wl.branching_tree_lumen(3)
    assert abs(w.insertions[-1] - 0.9 * min(paths)) < 1e-12
    assert w.robot.n_elements == 2000 and len(w.lumen.triangles) > 350000
