"""Contact solver ACCFEM_CONTACT_ADMM (accfem_set_contact_solver): the paper's scheme for Eq. 23
(Sec. III.B: OSQP), OSQP's ADMM on the contact-space QP over the working set, then the exact
polish of its free-row guess.  The solution of each contact QP is unique, so the solves equal the
oracle's (positions 1e-9 relative, contact nodes, net forces) and the default solver's."""
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


def _forces(contacts):
    f = {}
    for c in contacts:
        f[c["node"]] = f.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
    return f


def test_admm_bent_tube_matches_oracle(af):
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    assert gpu.accfem_set_contact_solver(af.CONTACT_ADMM) == af.OK
    ref = solver.Model(w.robot, w.lumen)
    rows = 0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["error"])
        err = np.abs(g["node_pos"] - o.node_pos).max() / np.abs(o.node_pos).max()
        assert err <= 1e-9, (s, err)
        assert sorted({c["node"] for c in g["contacts"]}) == sorted({c["node"] for c in o.contacts}), s
        fo, fg = _forces(o.contacts), _forces(g["contacts"])
        fmax = max([np.linalg.norm(v) for v in fo.values()] + [1e-300])
        for n in fo:
            assert np.linalg.norm(fo[n] - fg[n]) <= 1e-6 * fmax, (s, n)
        rows += len(g["contacts"])
    assert rows > 0
    gpu.close()


def test_admm_equals_active_set_on_an_uneven_instance(af):
    """Instance 2 of the batched workload (961 elements, its own lumen), first 12 steps."""
    w = wl.batch_workloads(first=2, count=1)[0]
    a = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    b = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    assert b.accfem_set_contact_solver(af.CONTACT_ADMM) == af.OK
    for s in range(12):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert ra["status"] == af.OK and rb["status"] == af.OK, (s, rb["error"])
        err = np.abs(ra["node_pos"] - rb["node_pos"]).max() / np.abs(ra["node_pos"]).max()
        assert err <= 1e-9, (s, err)
        assert sorted({c["node"] for c in ra["contacts"]}) == sorted({c["node"] for c in rb["contacts"]}), s
    a.close()
    b.close()


def test_contact_solver_arguments(af):
    w = wl.bent_tube_workload(0, n_steps=2)
    h = af.AccFem(w.robot, w.lumen)
    assert h.accfem_set_contact_solver(3) == af.E_INVALID_ARG
    assert h.accfem_set_contact_solver(-1) == af.E_INVALID_ARG
    r0 = h.accfem_solve(w.tensions[1], w.insertions[1])
    h.accfem_reset()
    assert h.accfem_set_contact_solver(af.CONTACT_ADMM) == af.OK
    h.accfem_solve(w.tensions[1], w.insertions[1])
    h.accfem_reset()
    assert h.accfem_set_contact_solver(af.CONTACT_ACTIVE_SET) == af.OK
    r1 = h.accfem_solve(w.tensions[1], w.insertions[1])
    assert np.array_equal(r0["node_pos"], r1["node_pos"])
    h.close()


def test_admm_member_in_a_batch_equals_alone(af):
    """A batch mixing an ADMM member (the bent tube, rows from step 5 on) with an active-set member:
    the ADMM member's results equal its solves alone bit for bit, and it ran ADMM iterations."""
    w = wl.bent_tube_workload(0, n_steps=10)
    other = wl.bent_tube_workload(7, n_steps=10)
    alone = af.AccFem(w.robot, w.lumen)
    alone.accfem_set_contact_solver(af.CONTACT_ADMM)
    ref, admm = [], 0
    for s in range(len(w.insertions)):
        ref.append(alone.accfem_solve(w.tensions[s], w.insertions[s]))
        admm += alone.accfem_solve_admm_iterations()
    assert all(r["status"] == af.OK for r in ref) and admm > 0
    hs = [af.AccFem(w.robot, w.lumen), af.AccFem(other.robot, other.lumen)]
    hs[0].accfem_set_contact_solver(af.CONTACT_ADMM)
    b = af.AccFemBatch(hs)
    for s in range(len(w.insertions)):
        st, sts, res = b.accfem_batch_solve([w.tensions[s], other.tensions[s]], [w.insertions[s], other.insertions[s]])
        assert sts[0] == af.OK and sts[1] == af.OK
        assert np.array_equal(res[0]["node_pos"], ref[s]["node_pos"]), s
        assert res[0]["newton_iters"] == ref[s]["newton_iters"], s
    b.close()
    for h in hs + [alone]:
        h.close()


def test_primal_admm_bent_tube_matches_oracle(af):
    """ACCFEM_CONTACT_PRIMAL_ADMM (the paper's OSQP on the primal QP of Eq. 23, K + sigma I + rho A^T A
    factored by the one-CTA reduction) against the oracle's primal ADMM (solver.Options(qp_solver=
    "primal_admm")): the same states, contact nodes and net forces, and ADMM iterations were run."""
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    assert gpu.accfem_set_contact_solver(af.CONTACT_PRIMAL_ADMM) == af.OK
    ref = solver.Model(w.robot, w.lumen, solver.Options(qp_solver="primal_admm"))
    rows = iters = 0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["error"])
        err = np.abs(g["node_pos"] - o.node_pos).max() / np.abs(o.node_pos).max()
        assert err <= 1e-9, (s, err)
        assert sorted({c["node"] for c in g["contacts"]}) == sorted({c["node"] for c in o.contacts}), s
        fo, fg = _forces(o.contacts), _forces(g["contacts"])
        fmax = max([np.linalg.norm(v) for v in fo.values()] + [1e-300])
        for n in fo:
            assert np.linalg.norm(fo[n] - fg[n]) <= 1e-6 * fmax, (s, n)
        rows += len(g["contacts"])
        iters += gpu.accfem_solve_admm_iterations()
    assert rows > 0 and iters > 0
    gpu.close()


def test_primal_admm_equals_active_set_on_the_sweep_start(af):
    """The first 40 solves of the 600 mm sweep (up to 200 free nodes, rows from solve 8 on) with the
    primal ADMM and with the default solver: the same states (the exact polish gives the unique
    contact solution either way)."""
    w = wl.catmull_rom_workload(lumen_seed=1, tension_seed=2, n_steps=60)
    a = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    b = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    assert b.accfem_set_contact_solver(af.CONTACT_PRIMAL_ADMM) == af.OK
    for s in range(40):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert ra["status"] == af.OK and rb["status"] == af.OK, (s, rb["error"])
        err = np.abs(ra["node_pos"] - rb["node_pos"]).max() / np.abs(ra["node_pos"]).max()
        assert err <= 1e-9, (s, err)
    a.close()
    b.close()


def test_primal_admm_arguments(af):
    w = wl.bent_tube_workload(0, n_steps=2)
    h = af.AccFem(w.robot, w.lumen)
    assert h.accfem_set_contact_model(af.CONTACT_SEGMENT) == af.OK
    assert h.accfem_set_contact_solver(af.CONTACT_PRIMAL_ADMM) == af.E_INVALID_ARG   # node contacts only
    assert h.accfem_set_contact_model(af.CONTACT_NODE) == af.OK
    assert h.accfem_set_contact_solver(af.CONTACT_PRIMAL_ADMM) == af.OK
    assert h.accfem_set_contact_model(af.CONTACT_SEGMENT) == af.E_INVALID_ARG
    with pytest.raises(RuntimeError):                                                  # not in batches
        af.AccFemBatch([h])
    assert h.accfem_set_contact_solver(3) == af.E_INVALID_ARG
    h.close()
