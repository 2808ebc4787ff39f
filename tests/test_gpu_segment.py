"""Segment contacts on the GPU (accfem_set_contact_model(ACCFEM_CONTACT_SEGMENT); Eq. 3-7 at any point
of an element) against the oracle's segment model (oracle/segment.py, solver.Options(contact_model=
"segment")): nodal positions 1e-9 relative, the same rows (element, closest wall point within 1e-9 m;
only rows at the activation distance may differ) and per-row forces (1e-6 of the largest)."""
import numpy as np
import pytest

import workloads as wl
from oracle import segment, solver

pytestmark = pytest.mark.gpu

L, M = 0.12, 20
ROB = wl.robot_desc(L, M)


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


def _compare(g, o, r_o, act, tag, ftol=1e-6):
    scale = np.abs(o.node_pos).max()
    err = np.abs(g["node_pos"] - o.node_pos).max() / scale
    assert err <= 1e-9, (tag, err)
    # GPU rows: contact_node = the element's far node; oracle rows: elem
    gr = [(c["node"] - 1, np.asarray(c["point"]), c["force"]) for c in g["contacts"]]
    orr = [(c["elem"], np.asarray(c["point"]), c["force"]) for c in o.contacts]
    fmax = max([c[2] for c in orr] + [1e-300])

    def match(a, b):
        out = []
        for e, p, f in a:
            k = next((j for j, (e2, p2, f2) in enumerate(b) if e2 == e and np.linalg.norm(p2 - p) <= 1e-9), -1)
            out.append(k)
        return out
    for (e, p, f), k in zip(gr, match(gr, orr)):
        if k < 0:                                     # only a row at the activation distance may be missing
            continue
        assert abs(f - orr[k][2]) <= ftol * fmax, (tag, e, f, orr[k][2])
    unmatched = [i for i, k in enumerate(match(orr, gr)) if k < 0] + [i for i, k in enumerate(match(gr, orr)) if k < 0]
    assert len(unmatched) <= 0, (tag, "rows differ", len(gr), len(orr))
    return err


def _coarse_bent_tube():
    """The bent-tube workload with its tube meshed 16 around x 2 mm axial (2176 triangles): a 6 mm chord
    lying along the 24 x 1 mm tube is over more facets than the per-element row limit (16)."""
    b = wl.bent_tube_workload(0, n_steps=10)
    return wl.Workload(b.name, b.robot, wl._lumen_from_centerline(wl.bent_tube_centerline(ds=0.002), 0.005, 16),
                       b.insertions, b.tensions)


def test_patch_between_nodes(af):
    """A tip load pushes the rod against a 1 mm patch above the middle of element 10: the node model
    finds no row, the segment model rests on it; GPU and oracle agree on the state, rows and force."""
    sec_EI = 2.0e9 * np.pi * (2e-3 ** 4 - 1e-3 ** 4) / 4
    l0 = L / M
    g = 2e-6
    a = 10.5 * l0
    lum = wl.patch_lumen(a - 0.5e-3, a + 0.5e-3, ROB.outer_radius + g, z_half=1e-3, n=1)
    P = 2 * g * 6 * sec_EI / (a * a * (3 * L - a))
    load = ((0.0, P, 0.0), (0.0, 0.0, 0.0), False)
    node = af.AccFem(ROB, lum, step_limit=1.0)
    rn = node.accfem_solve_tip_load(load[0], load[1], False, L)
    assert rn["status"] == af.OK and rn["n_contacts"] == 0
    gpu = af.AccFem(ROB, lum, step_limit=1.0)
    assert gpu.accfem_set_contact_model(af.CONTACT_SEGMENT) == af.OK
    rg = gpu.accfem_solve_tip_load(load[0], load[1], False, L)
    ref = solver.Model(ROB, lum, solver.Options(step_limit=1.0, contact_model="segment"))
    ro = ref.solve(delta=L, tip_load=load)
    assert rg["status"] == af.OK and ro.status == solver.OK, rg["error"]
    assert rg["n_contacts"] >= 1 and any(c["force"] > 0.0 for c in rg["contacts"])
    assert all(c["node"] == 11 for c in rg["contacts"] if c["force"] > 0.0)       # element 10
    _compare(rg, ro, ROB.outer_radius, 1e-3, "patch")
    node.close()
    gpu.close()


def test_bent_tube_sweep_segment_model(af):
    """The 120 mm robot inserted through the bent tube (meshed 16 around x 2 mm axial, 2176 triangles,
    to keep the oracle's all-triangle segment test short) with segment contacts, step by step."""
    w = _coarse_bent_tube()
    gpu = af.AccFem(w.robot, w.lumen)
    assert gpu.accfem_set_contact_model(af.CONTACT_SEGMENT) == af.OK
    ref = solver.Model(w.robot, w.lumen, solver.Options(contact_model="segment"))
    worst, rows = 0.0, 0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["error"], o.status)
        worst = max(worst, _compare(g, o, w.robot.outer_radius, 1e-3, "step %d" % s))
        rows += g["n_contacts"]
    assert rows > 0
    # switching back gives the node model's result
    assert gpu.accfem_set_contact_model(af.CONTACT_NODE) == af.OK
    assert gpu.accfem_set_contact_model(2) == af.E_INVALID_ARG
    gpu.close()


def test_segment_member_in_a_batch_equals_alone(af):
    """A batch mixing a segment-model member with node-model members: the segment member's results
    equal its solves alone bit for bit."""
    w = _coarse_bent_tube()
    other = wl.bent_tube_workload(7, n_steps=10)
    alone = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    alone.accfem_set_contact_model(af.CONTACT_SEGMENT)
    ref = [alone.accfem_solve(w.tensions[s], w.insertions[s]) for s in range(len(w.insertions))]
    assert all(r["status"] == af.OK for r in ref) and ref[-1]["n_contacts"] > 0
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=4096), af.AccFem(other.robot, other.lumen)]
    hs[0].accfem_set_contact_model(af.CONTACT_SEGMENT)
    b = af.AccFemBatch(hs)
    for s in range(len(w.insertions)):
        st, sts, res = b.accfem_batch_solve([w.tensions[s], other.tensions[s]], [w.insertions[s], other.insertions[s]])
        assert sts[0] == af.OK and sts[1] == af.OK
        assert np.array_equal(res[0]["node_pos"], ref[s]["node_pos"]), s
        assert res[0]["newton_iters"] == ref[s]["newton_iters"], s
        assert [c["force"] for c in res[0]["contacts"]] == [c["force"] for c in ref[s]["contacts"]], s
    b.close()
    for h in hs + [alone]:
        h.close()
