"""Frame mode (accfem_set_frame_mode): the paper's real-time scheme, one linearisation of Eq. 20-23
per frame with the limited step of Eq. 25-27.  Every frame's state is compared with the oracle run
with the same iteration cap per solve (its arithmetic is the full-convergence solver's, stopped at
the cap): positions 1e-9 relative, the same contact nodes.  At fixed inputs the frames reach the
equilibrium of a converged solve."""
import numpy as np
import pytest

import workloads as wl
from oracle import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def af():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06922_gb300 import accfem
    import os
    if not os.path.exists(accfem.LIB_PATH):
        from paper_2503_06922_gb300 import build
        build.build()
    accfem.load()
    return accfem


def _frames(af, w, k, steps, per_step):
    gpu = af.AccFem(w.robot, w.lumen)
    assert gpu.accfem_set_frame_mode(k) == af.OK
    ref = solver.Model(w.robot, w.lumen, solver.Options(max_newton_iters=k))
    scale = 0.0
    worst = 0.0
    rows = 0
    for s in range(steps):
        for f in range(per_step):
            g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
            o = ref.solve(w.tensions[s], w.insertions[s])
            assert g["status"] == af.OK, (s, f, g["error"])
            assert 1 <= g["newton_iters"] <= k and g["newton_iters"] == o.newton_iters, (s, f)
            scale = max(scale, np.abs(o.node_pos).max())
            err = np.abs(g["node_pos"] - o.node_pos).max() / scale
            worst = max(worst, err)
            assert err <= 1e-9, (s, f, err)
            assert sorted({c["node"] for c in g["contacts"]}) == sorted({c["node"] for c in o.contacts}), (s, f)
            rows += len(g["contacts"])
    return gpu, ref, worst, rows


def test_one_iteration_frames_match_oracle(af):
    """Bent tube, 4 frames per 10 mm insertion step: the robot lags the insertion (each frame moves
    a node by at most the step limit) and meets the wall, frame by frame as in the oracle."""
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu, ref, worst, rows = _frames(af, w, 1, 10, 4)
    assert rows > 0
    # the lag: a converged solve of the last step ends elsewhere
    full = solver.Model(w.robot, w.lumen)
    for s in range(10):
        o = full.solve(w.tensions[s], w.insertions[s])
    g = gpu.accfem_solve(w.tensions[9], w.insertions[9])
    assert np.abs(g["node_pos"] - o.node_pos).max() > 1e-3
    # at fixed inputs the frames reach the equilibrium
    for _ in range(150):
        g = gpu.accfem_solve(w.tensions[9], w.insertions[9])
        assert g["status"] == af.OK
    assert np.abs(g["node_pos"] - o.node_pos).max() <= 1e-9 * np.abs(o.node_pos).max()
    gpu.close()


def test_three_iteration_frames_match_oracle(af):
    w = wl.bent_tube_workload(3, n_steps=10)
    gpu, ref, worst, rows = _frames(af, w, 3, 10, 2)
    gpu.close()


def test_batch_member_in_frame_mode_equals_alone(af):
    w = wl.bent_tube_workload(0, n_steps=10)
    alone = af.AccFem(w.robot, w.lumen)
    assert alone.accfem_set_frame_mode(2) == af.OK
    ra = [alone.accfem_solve(w.tensions[s], w.insertions[s]) for s in range(10)]
    h = af.AccFem(w.robot, w.lumen)
    assert h.accfem_set_frame_mode(2) == af.OK
    other = af.AccFem(w.robot, w.lumen)          # solves to convergence beside it
    b = af.AccFemBatch([h, other])
    for s in range(10):
        st, sts, res = b.accfem_batch_solve([w.tensions[s]] * 2, [w.insertions[s]] * 2)
        assert st == af.OK and sts[0] == af.OK and sts[1] == af.OK
        assert np.array_equal(res[0]["node_pos"], ra[s]["node_pos"]), s
        assert res[0]["newton_iters"] == ra[s]["newton_iters"] <= 2
    b.close()
    for x in (alone, h, other):
        x.close()


def test_frame_mode_arguments(af):
    w = wl.bent_tube_workload(0, n_steps=3)
    h = af.AccFem(w.robot, w.lumen)
    assert h.accfem_set_frame_mode(-1) == af.E_INVALID_ARG
    assert h.accfem_set_frame_mode(10 ** 7) == af.E_INVALID_ARG
    assert h.accfem_set_frame_mode(1) == af.OK
    r = h.accfem_solve(w.tensions[2], w.insertions[2])
    assert r["status"] == af.OK and r["newton_iters"] == 1
    # back to solves to convergence: the next solve converges from the frame's state
    assert h.accfem_set_frame_mode(0) == af.OK
    r = h.accfem_solve(w.tensions[2], w.insertions[2])
    assert r["status"] == af.OK and r["newton_iters"] > 1
    ref = solver.Model(w.robot, w.lumen)
    for s in range(3):
        o = ref.solve(w.tensions[s], w.insertions[s])
    assert np.abs(r["node_pos"] - o.node_pos).max() <= 1e-9 * np.abs(o.node_pos).max()
    h.close()
