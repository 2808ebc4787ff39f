"""GPU path (through the C ABI) vs the CPU FP64 oracle on the same seeded inputs.

Tolerances: nodal positions 1e-9 relative (the parity target of the path), contact rows identical
as (node, closest point) apart from rows within 1e-9 m of the activation distance, net contact force
per node (sum of y_i n_i) 1e-6 relative to the largest one (the multipliers solve an LCP whose
conditioning amplifies rounding; the per-node net force is unique even where rows are dependent)."""
import numpy as np
import pytest

import workloads as wl
from oracle import contact, solver

pytestmark = pytest.mark.gpu

REL_POS = 1e-9


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


def _compare(g, o, act_thr, tag=""):
    scale = np.abs(o.node_pos).max()
    err = np.abs(g["node_pos"] - o.node_pos).max() / scale
    assert err <= REL_POS, (tag, err)
    qg, qo = g["node_quat"], o.node_quat
    qerr = np.minimum(np.abs(qg - qo).max(axis=1), np.abs(qg + qo).max(axis=1)).max()
    assert qerr <= 1e-9, (tag, qerr)
    gk = [(c["node"], tuple(np.round(c["point"], 9))) for c in g["contacts"]]
    ok = [(c["node"], tuple(np.round(c["point"], 9))) for c in o.contacts]
    if gk != ok:
        # only rows at the activation boundary may differ
        diff = set(gk) ^ set(ok)
        for node, pt in diff:
            p = o.node_pos[node] if node < len(o.node_pos) else None
            d = np.linalg.norm(np.array(pt) - p)
            assert abs(d - act_thr) <= 1e-9, (tag, "contact set differs", node, d)
    # net contact force on each node, sum_i y_i n_i (unique even where rows of a node are dependent)
    fo, fg = {}, {}
    for c in o.contacts:
        fo[c["node"]] = fo.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
    for c in g["contacts"]:
        fg[c["node"]] = fg.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
    fmax = max([np.linalg.norm(v) for v in fo.values()] + [1e-300])
    for n in set(fo) | set(fg):
        assert np.linalg.norm(fo.get(n, 0.0) - fg.get(n, 0.0)) <= 1e-6 * fmax, (tag, n, fo.get(n), fg.get(n))
    return err


def test_bent_tube_sweep_matches_oracle(af):
    """120 mm rod, 20 elements, 5 mm tube with a 90 deg bend: insertion 10 -> 100 mm."""
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    ref = solver.Model(w.robot, w.lumen)
    thr = w.robot.outer_radius + 1e-3
    worst = 0.0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["status"], g["error"])
        worst = max(worst, _compare(g, o, thr, "step %d" % s))
        assert abs(g["newton_iters"] - o.newton_iters) <= 3
        # both solves stop within newton_tol of the equilibrium along different paths (the GPU
        # solves the contact problem over a working set): the clamp force may differ by the axial
        # stiffness times twice that tolerance
        l0 = w.robot.length / w.robot.n_elements
        EA = w.robot.youngs_modulus * np.pi * (w.robot.outer_radius ** 2 - w.robot.inner_radius ** 2)
        assert np.allclose(g["base_reaction"], o.base_reaction, rtol=0.0, atol=2.0 * EA / l0 * 1e-11)
    assert len(g["contacts"]) >= 4
    gpu.close()


def test_second_tension_seed(af):
    w = wl.bent_tube_workload(7, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    ref = solver.Model(w.robot, w.lumen)
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK
    _compare(g, o, w.robot.outer_radius + 1e-3, "seed 7")
    gpu.close()


def test_free_space_closed_forms(af):
    """Cantilever P L^3/3EI, tip torque T L/GJ and the end-moment arc, through accfem_solve_tip_load."""
    L, M = 0.12, 20
    rob = wl.robot_desc(L, M)
    from oracle import beam
    sec = beam.section_constants(rob)
    gpu = af.AccFem(rob, wl.free_space_lumen(), step_limit=1.0)
    P = 3 * sec["EI"] * 1.2e-6 / L ** 3
    g = gpu.accfem_solve_tip_load((0.0, P, 0.0), (0.0, 0.0, 0.0), False, L)
    assert g["status"] == af.OK
    assert g["node_pos"][-1, 1] == pytest.approx(P * L ** 3 / (3 * sec["EI"]), rel=1e-8)
    Mz = 0.5 * np.pi * sec["EI"] / L
    gpu2 = af.AccFem(rob, wl.free_space_lumen(), step_limit=5e-3)
    g = gpu2.accfem_solve_tip_load((0.0, 0.0, 0.0), (0.0, 0.0, Mz), False, L)
    o = solver.Model(rob, wl.free_space_lumen(), solver.Options(step_limit=5e-3)).solve(
        delta=L, tip_load=((0.0, 0.0, 0.0), (0.0, 0.0, Mz), False))
    assert g["status"] == af.OK
    l0 = L / M
    phi = Mz * l0 / sec["EI"]
    ang = (np.arange(M) + 0.5) * phi
    pos = np.vstack([np.zeros(3), np.cumsum(l0 * np.column_stack([np.cos(ang), np.sin(ang), np.zeros(M)]), axis=0)])
    assert np.abs(g["node_pos"] - pos).max() <= 1e-10 * L
    assert np.abs(g["node_pos"] - o.node_pos).max() <= 1e-10 * L
    # follower tip force in the tip frame bends and follows; compare with the oracle
    g = gpu2.accfem_solve_tip_load((0.0, 0.5, 0.0), (0.0, 0.0, 0.0), True, L)
    o = solver.Model(rob, wl.free_space_lumen(), solver.Options(step_limit=5e-3)).solve(
        delta=L, tip_load=((0.0, 0.5, 0.0), (0.0, 0.0, 0.0), True))
    assert g["status"] == af.OK and o.status == solver.OK
    assert np.abs(g["node_pos"] - o.node_pos).max() <= REL_POS * L
    gpu.close(); gpu2.close()


def test_collision_rows_match_brute_force(af):
    """One Newton iteration from random start poses near the wall: the rows the GPU reports are the
    oracle's all-pairs rows at those poses (ties on shared edges compared by closest point)."""
    w = wl.bent_tube_workload(0, n_steps=10)
    rng = np.random.default_rng(5)
    gpu = af.AccFem(w.robot, w.lumen, max_newton_iters=1)
    ref = solver.Model(w.robot, w.lumen)
    x0, R0 = ref.straight(0.1)
    quat = np.array([[1.0, 0, 0, 0]] * len(x0))
    from oracle.rotation import to_quat
    q0 = to_quat(R0[0])
    quat[:] = q0
    V, T = w.lumen.vertices, w.lumen.triangles
    pts = wl.bent_tube_centerline()
    k = solver.n_prescribed_last(w.robot.length, w.robot.n_elements, 0.1)
    for trial in range(6):
        x = x0.copy()
        for i in range(k + 1, w.robot.n_elements + 1):
            c = pts[rng.integers(20, len(pts) - 5)]
            off = rng.normal(size=3)
            x[i] = c + off / np.linalg.norm(off) * rng.uniform(2.0e-3, 3.4e-3)
        g = gpu.accfem_solve(w.tensions[0], 0.1, warm=(x, quat))
        rows = contact.detect(x, range(k + 1, w.robot.n_elements + 1), V, T, w.robot.outer_radius, 1e-3)
        gk = sorted((c["node"], tuple(np.round(c["point"], 10))) for c in g["contacts"])
        ok = sorted((r["node"], tuple(np.round(r["point"], 10))) for r in rows)
        assert gk == ok, trial
        for cg in g["contacts"]:
            r = [r for r in rows if r["node"] == cg["node"] and np.allclose(r["point"], cg["point"], atol=1e-12)][0]
            assert np.allclose(cg["normal"], r["normal"], atol=1e-12)
    gpu.close()


def test_empty_and_edge_cases(af):
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    g = gpu.accfem_solve(w.tensions[0], 0.0)          # no free node
    assert g["status"] == af.OK and g["newton_iters"] == 0 and g["n_contacts"] == 0
    g = gpu.accfem_solve(w.tensions[0], 0.2)          # beyond the robot length
    assert g["status"] == af.E_INVALID_ARG
    g = gpu.accfem_solve([-1.0, 0.0, 0.0], 0.05)      # negative tension
    assert g["status"] == af.E_INVALID_ARG
    g = gpu.accfem_solve(w.tensions[0], 0.006)        # exactly one free node
    o = solver.Model(w.robot, w.lumen).solve(w.tensions[0], 0.006)
    assert g["status"] == af.OK and np.abs(g["node_pos"] - o.node_pos).max() <= REL_POS * 0.12
    gpu.close()
