"""Per-element Young's modulus (accfem_set_element_modulus; Sec. II.A: a distal section much less
rigid than the rest) through the C ABI: closed forms of a beam with element-wise constant
stiffness, the oracle on a soft-tip sweep with contacts, bit-identity of the uniform array, the
batch and the argument checks."""
import math
from dataclasses import replace

import numpy as np
import pytest

import workloads as wl
from oracle import beam, solver

pytestmark = pytest.mark.gpu

L, M = 0.12, 20
l0 = L / M
BASE = wl.robot_desc(L, M)
RATIO = np.random.default_rng(40).uniform(0.2, 1.0, M)
ROB = replace(BASE, element_youngs=BASE.youngs_modulus * RATIO)


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


def _secs():
    s = beam.element_sections(ROB)
    return (np.array([x["EA"] for x in s]), np.array([x["EI"] for x in s]), np.array([x["GJ"] for x in s]))


def test_piecewise_closed_forms(af):
    EA, EI, GJ = _secs()
    gpu = af.AccFem(ROB, wl.free_space_lumen(), step_limit=1.0)
    # series axial compliance
    P = 50.0
    g = gpu.accfem_solve_tip_load((P, 0.0, 0.0), (0.0, 0.0, 0.0), False, L)
    assert g["status"] == af.OK
    x = np.concatenate([[0.0], np.cumsum(l0 + P * l0 / EA)])
    assert np.allclose(g["node_pos"][:, 0], x, rtol=1e-12, atol=0.0)
    # small-deflection cantilever: unit-load integral over element-wise EI
    gpu.accfem_reset()
    P = 3 * EI.min() * 1.2e-6 / L ** 3
    g = gpu.accfem_solve_tip_load((0.0, P, 0.0), (0.0, 0.0, 0.0), False, L)
    assert g["status"] == af.OK

    def v(xx):
        F = lambda s: L * xx * s - (L + xx) * s * s / 2.0 + s ** 3 / 3.0
        return sum(P * (F(min((e + 1) * l0, xx)) - F(e * l0)) / EI[e] for e in range(M) if e * l0 < xx)
    vv = np.array([v(i * l0) for i in range(M + 1)])
    assert np.allclose(g["node_pos"][:, 1], vv, rtol=1e-8, atol=1e-18)
    gpu.close()
    # pure end moment: chords of length l0 turning by Mz l0 / EI_e
    gpu = af.AccFem(ROB, wl.free_space_lumen(), step_limit=5e-3)
    Mz = 0.4 * math.pi / np.sum(l0 / EI)
    g = gpu.accfem_solve_tip_load((0.0, 0.0, 0.0), (0.0, 0.0, Mz), False, L)
    assert g["status"] == af.OK
    phi = Mz * l0 / EI
    psi = np.concatenate([[0.0], np.cumsum(phi)])
    ang = psi[:-1] + 0.5 * phi
    pos = np.vstack([np.zeros(3), np.cumsum(l0 * np.column_stack([np.cos(ang), np.sin(ang), np.zeros(M)]), axis=0)])
    assert np.abs(g["node_pos"] - pos).max() <= 1e-10 * L
    gpu.close()


def test_soft_tip_sweep_matches_oracle(af):
    """Bent tube with a 70 mm distal section at a tenth of the modulus, 10 insertion steps with
    contacts: positions 1e-9 relative, the same contact nodes, net contact force per node within
    1e-6 of the largest one or the force that the Newton tolerance leaves open, whichever is
    larger: both sides stop at a residual up to tol max(1, |F_a|, max y), and a residual moment of
    that size acting over one element length l0 moves a contact force by tol max(1, sum tau) / l0."""
    w = wl.bent_tube_workload(0, n_steps=10)
    rob = wl.with_soft_tip(w.robot)
    gpu = af.AccFem(rob, w.lumen)
    ref = solver.Model(rob, w.lumen)
    n_rows = 0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["error"])
        err = np.abs(g["node_pos"] - o.node_pos).max() / np.abs(o.node_pos).max()
        assert err <= 1e-9, (s, err)
        assert sorted({c["node"] for c in g["contacts"]}) == sorted({c["node"] for c in o.contacts}), s
        fo, fg = {}, {}
        for c in o.contacts:
            fo[c["node"]] = fo.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
        for c in g["contacts"]:
            fg[c["node"]] = fg.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
        fmax = max([np.linalg.norm(f) for f in fo.values()] + [1e-300])
        ftol = max(1e-6 * fmax, 1e-10 * max(1.0, float(np.sum(w.tensions[s]))) / (rob.length / rob.n_elements))
        for n in fo:
            assert np.linalg.norm(fo[n] - fg[n]) <= ftol, (s, n, np.linalg.norm(fo[n] - fg[n]), ftol)
        n_rows += len(g["contacts"])
    assert n_rows > 0
    # the soft tip changes the answer: the uniform robot ends elsewhere
    uni = af.AccFem(w.robot, w.lumen)
    for s in range(len(w.insertions)):
        u = uni.accfem_solve(w.tensions[s], w.insertions[s])
    assert np.abs(u["node_pos"][-1] - g["node_pos"][-1]).max() > 1e-5
    gpu.close(); uni.close()


def test_uniform_array_is_bit_identical_and_null_restores(af):
    w = wl.bent_tube_workload(0, n_steps=4)
    a = af.AccFem(w.robot, w.lumen)
    b = af.AccFem(w.robot, w.lumen)
    assert b.accfem_set_element_modulus(np.full(M, w.robot.youngs_modulus)) == af.OK
    for s in range(4):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert np.array_equal(ra["node_pos"], rb["node_pos"]) and ra["newton_iters"] == rb["newton_iters"]
    # soft, then NULL: back to the uniform robot's answer for the same warm start
    assert b.accfem_set_element_modulus(wl.soft_tip_moduli(w.robot)) == af.OK
    a.accfem_reset(); b.accfem_reset()
    rs = b.accfem_solve(w.tensions[3], w.insertions[3])
    b.accfem_reset()
    assert b.accfem_set_element_modulus(None) == af.OK
    rb = b.accfem_solve(w.tensions[3], w.insertions[3])
    ra = a.accfem_solve(w.tensions[3], w.insertions[3])
    assert np.array_equal(ra["node_pos"], rb["node_pos"])
    assert not np.array_equal(rs["node_pos"], rb["node_pos"])
    a.close(); b.close()


def test_batch_member_with_soft_tip_equals_alone(af):
    w = wl.bent_tube_workload(0, n_steps=6)
    rob = wl.with_soft_tip(w.robot)
    alone = af.AccFem(rob, w.lumen)
    ra = [alone.accfem_solve(w.tensions[s], w.insertions[s]) for s in range(6)]
    hs = [af.AccFem(rob, w.lumen), af.AccFem(w.robot, w.lumen)]
    b = af.AccFemBatch(hs)
    for s in range(6):
        st, sts, res = b.accfem_batch_solve([w.tensions[s]] * 2, [w.insertions[s]] * 2)
        assert st == af.OK and sts[0] == af.OK
        assert np.array_equal(res[0]["node_pos"], ra[s]["node_pos"]), s
        assert res[0]["newton_iters"] == ra[s]["newton_iters"], s
    b.close()
    for h in hs + [alone]:
        h.close()


def test_modulus_arguments(af):
    w = wl.bent_tube_workload(0, n_steps=2)
    h = af.AccFem(w.robot, w.lumen)
    r0 = h.accfem_solve(w.tensions[0], w.insertions[0])
    E = np.full(M, w.robot.youngs_modulus)
    assert h.accfem_set_element_modulus(E, M - 1) == af.E_INVALID_ARG
    assert h.accfem_set_element_modulus(np.full(M + 1, 1e9)) == af.E_INVALID_ARG
    for bad in (0.0, -1e9, np.nan, np.inf):
        E2 = E.copy()
        E2[7] = bad
        assert h.accfem_set_element_modulus(E2) == af.E_INVALID_ARG
    # nothing changed: the same solve again from the same start gives the same answer
    h.accfem_reset()
    r1 = h.accfem_solve(w.tensions[0], w.insertions[0])
    assert np.array_equal(r0["node_pos"], r1["node_pos"])
    h.close()
