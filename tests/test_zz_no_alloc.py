"""The allocation-free collision query (accfem_detect_contacts_noalloc) against accfem_solve and the oracle.

Callers that must not allocate device memory once they run (a real-time loop that reserved its memory
at start-up, or an application that owns every allocation under a fixed budget) use this entry point:
its scratch is a fixed device array of the library, and the caller passes device buffers for the node
positions and the output rows.  Here it must report, for the same node positions, exactly the
constraint rows that accfem_solve detects at its start pose (one Newton iteration from a warm start)
and the rows of the oracle's all-triangle detection, on two calls in a row that reuse the shared
scratch; and the solve's per-node limit of 16 rows must hold (a node inside an icosahedral cell has
20 face rows: capacity status).  Tolerance: the one the collision parity test uses (points and normals
1e-12)."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import contact, solver
from oracle.rotation import to_quat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def af():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06922_gb300 import accfem
    if not os.path.exists(accfem.LIB_PATH):
        from paper_2503_06922_gb300 import build
        build.build()
    accfem.load()
    return accfem


def _poses(w, rng):
    ref = solver.Model(w.robot, w.lumen)
    x, R = ref.straight(0.1)
    quat = np.tile(to_quat(R[0]), (len(x), 1))
    pts = wl.bent_tube_centerline()
    k = solver.n_prescribed_last(w.robot.length, w.robot.n_elements, 0.1)
    for i in range(k + 1, w.robot.n_elements + 1):
        c = pts[rng.integers(20, len(pts) - 5)]
        off = rng.normal(size=3)
        x[i] = c + off / np.linalg.norm(off) * rng.uniform(2.0e-3, 3.4e-3)
    return x, quat, k


def test_noalloc_rows_match_solve_rows_twice(af):
    import torch
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen, max_newton_iters=1)
    rng = np.random.default_rng(21)
    cap = 256
    row_node = torch.zeros(cap, dtype=torch.int32, device="cuda")
    row_tri = torch.zeros(cap, dtype=torch.int32, device="cuda")
    row_pt = torch.zeros(cap * 3, dtype=torch.float64, device="cuda")
    row_n = torch.zeros(cap * 3, dtype=torch.float64, device="cuda")
    row_gap = torch.zeros(cap, dtype=torch.float64, device="cuda")
    n_rows = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call in range(2):
        x, quat, k = _poses(w, rng)
        g = gpu.accfem_solve(w.tensions[0], 0.1, warm=(x, quat))
        assert g["error"] in ("", "Newton iterations did not converge")
        pos = torch.tensor(x[k + 1:], dtype=torch.float64, device="cuda").contiguous()
        n = pos.shape[0]
        st = gpu.accfem_detect_contacts_noalloc(pos.data_ptr(), n, cap, row_node.data_ptr(), row_tri.data_ptr(),
                                                row_pt.data_ptr(), row_n.data_ptr(), row_gap.data_ptr(),
                                                n_rows.data_ptr())
        torch.cuda.synchronize()
        assert st == af.OK, gpu.accfem_last_error()
        m = int(n_rows.item())
        assert m == g["n_contacts"] and m > 0, (call, m, g["n_contacts"])
        nodes = row_node[:m].cpu().numpy() + k + 1
        tris = row_tri[:m].cpu().numpy()
        pts = row_pt[:3 * m].cpu().numpy().reshape(m, 3)
        nrm = row_n[:3 * m].cpu().numpy().reshape(m, 3)
        gaps = row_gap[:m].cpu().numpy()
        for i, c in enumerate(g["contacts"]):
            assert nodes[i] == c["node"] and tris[i] == c["tri"], (call, i)
            assert np.allclose(pts[i], c["point"], atol=1e-12)
            assert np.allclose(nrm[i], c["normal"], atol=1e-12)
            p = x[c["node"]]
            assert gaps[i] == pytest.approx(np.dot(c["normal"], c["point"] - p) - w.robot.outer_radius, abs=1e-12)
        # the oracle's detection over all triangles (no grid, no FP32 prefilter), same positions
        V = np.asarray(w.lumen.vertices, dtype=np.float64).reshape(-1, 3)
        T = np.asarray(w.lumen.triangles, dtype=np.int64).reshape(-1, 3)
        ref = contact.detect(x, range(k + 1, w.robot.n_elements + 1), V, T, w.robot.outer_radius, 1.0e-3)
        assert len(ref) == m, (call, len(ref), m)
        for i, r in enumerate(ref):
            assert nodes[i] == r["node"] and tris[i] == r["tri"], (call, i)
            assert np.allclose(pts[i], r["point"], atol=1e-12)
            assert np.allclose(nrm[i], r["normal"], atol=1e-12)
            assert gaps[i] == pytest.approx(r["gap"], abs=1e-12)
    # a size beyond the fixed maximum is rejected with a clear message
    st = gpu.accfem_detect_contacts_noalloc(pos.data_ptr(), 5000, cap, row_node.data_ptr(), row_tri.data_ptr(),
                                            row_pt.data_ptr(), row_n.data_ptr(), row_gap.data_ptr(), n_rows.data_ptr())
    assert st == af.E_INVALID_ARG and "4096" in gpu.accfem_last_error()
    gpu.close()


def _polyhedron_cell(kind, inradius):
    """Closed convex cell around the origin whose faces are all tangent to the sphere of the given
    radius, wound outward (the cell's inside is the lumen): an octahedron (8 faces) or an
    icosahedron (20 faces)."""
    if kind == "octahedron":
        V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
        edge = np.sqrt(2.0)
    else:
        ph = (1.0 + np.sqrt(5.0)) / 2.0
        V = []
        for a in (-1.0, 1.0):
            for b in (-ph, ph):
                V += [[0.0, a, b], [a, b, 0.0], [b, 0.0, a]]
        V = np.array(V)
        edge = 2.0
    T = []
    n = len(V)
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                if all(abs(np.linalg.norm(V[p] - V[q]) - edge) < 1e-9 for p, q in ((i, j), (j, k), (i, k))):
                    nrm = np.cross(V[j] - V[i], V[k] - V[i])
                    T.append([i, j, k] if np.dot(nrm, V[i] + V[j] + V[k]) > 0 else [i, k, j])
    T = np.array(T, dtype=np.int32)
    c = (V[T[0, 0]] + V[T[0, 1]] + V[T[0, 2]]) / 3.0
    V = V * (inradius / np.linalg.norm(c))
    return wl.LumenDesc(V, T, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0))


def test_noalloc_per_node_row_limit(af):
    """A node at the centre of a cell whose faces all lie 2.5 mm away (within r_o + gap = 3 mm) has one
    face row per face: 8 in an octahedron (equal to the oracle's rows, twice in a row), 20 in an
    icosahedron, beyond the per-node limit of 16 that accfem_solve also applies (capacity status)."""
    import torch
    w = wl.bent_tube_workload(0, n_steps=10)
    r_o = w.robot.outer_radius
    cap = 64
    bufs = [torch.zeros(cap, dtype=torch.int32, device="cuda"), torch.zeros(cap, dtype=torch.int32, device="cuda"),
            torch.zeros(cap * 3, dtype=torch.float64, device="cuda"), torch.zeros(cap * 3, dtype=torch.float64, device="cuda"),
            torch.zeros(cap, dtype=torch.float64, device="cuda")]
    n_rows = torch.zeros(1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3, dtype=torch.float64, device="cuda")
    for kind, faces in (("octahedron", 8), ("icosahedron", 20)):
        lum = _polyhedron_cell(kind, r_o + 0.5e-3)
        h = af.AccFem(w.robot, lum)
        for call in range(2):
            st = h.accfem_detect_contacts_noalloc(pos.data_ptr(), 1, cap, *[b.data_ptr() for b in bufs], n_rows.data_ptr())
            torch.cuda.synchronize()
            if faces <= 16:
                assert st == af.OK, h.accfem_last_error()
                m = int(n_rows.item())
                ref = contact.detect(np.zeros((1, 3)), [0], lum.vertices, lum.triangles.astype(np.int64), r_o, 1.0e-3)
                assert m == faces == len(ref)
                tris = bufs[1][:m].cpu().numpy()
                pts = bufs[2][:3 * m].cpu().numpy().reshape(m, 3)
                nrm = bufs[3][:3 * m].cpu().numpy().reshape(m, 3)
                for i, r in enumerate(ref):
                    assert tris[i] == r["tri"] and r["face"]
                    assert np.allclose(pts[i], r["point"], atol=1e-12) and np.allclose(nrm[i], r["normal"], atol=1e-12)
            else:
                assert st == af.E_CONTACT_CAPACITY and "16 rows" in h.accfem_last_error(), (st, h.accfem_last_error())
        h.close()
