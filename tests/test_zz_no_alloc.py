"""The allocation-free collision query (accfem_detect_contacts_noalloc) against accfem_solve.

Callers that cannot call cudaMalloc while they run (inside CUDA stream capture, or in a loop with a
fixed device-memory budget) use this entry point: its scratch is a fixed device array of the
library, and the caller passes device buffers for the node positions and the output rows.  Here it
must report, for the same node positions, exactly the constraint rows that accfem_solve detects at
its start pose (one Newton iteration from a warm start), on two calls in a row that reuse the
shared scratch.  Tolerance: the one the collision parity test uses (points and normals 1e-12)."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import solver
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
    # a size beyond the fixed maximum is rejected with a clear message
    st = gpu.accfem_detect_contacts_noalloc(pos.data_ptr(), 5000, cap, row_node.data_ptr(), row_tri.data_ptr(),
                                            row_pt.data_ptr(), row_n.data_ptr(), row_gap.data_ptr(), n_rows.data_ptr())
    assert st == af.E_INVALID_ARG and "4096" in gpu.accfem_last_error()
    gpu.close()
