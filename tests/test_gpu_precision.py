"""Mixed precision (accfem_set_precision): FP32 element tangent, FP64 residual, factor and contact
solve.  The tangent only steers the Newton iteration, so a converged mixed solve sits within the
Newton tolerance of the FP64 equilibrium: checked against the oracle (tip position 1e-6 m, contact
forces 1e-4 relative, identical contact sets) and against the FP64 GPU path."""
import numpy as np
import pytest

import workloads as wl
from oracle import solver

pytestmark = pytest.mark.gpu

TIP_TOL = 1e-6        # m
FORCE_RTOL = 1e-4


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


def _node_forces(contacts):
    f = {}
    for c in contacts:
        f[c["node"]] = f.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
    return f


def _same_rows(ga, gb, tol=1e-9):
    """The same rows: per node as many, pairing up by closest point within tol (m)."""
    def group(cs):
        out = {}
        for c in cs:
            out.setdefault(c["node"], []).append(np.asarray(c["point"], dtype=np.float64))
        return out
    a, b = group(ga), group(gb)
    if set(a) != set(b):
        return False
    for n in a:
        if len(a[n]) != len(b[n]):
            return False
        used = [False] * len(b[n])
        for pa in a[n]:
            k = next((j for j, pb in enumerate(b[n]) if not used[j] and np.linalg.norm(pa - pb) <= tol), -1)
            if k < 0:
                return False
            used[k] = True
    return True


def _check(g, o_pos, o_contacts, tag):
    tip = np.linalg.norm(g["node_pos"][-1] - o_pos[-1])
    assert tip <= TIP_TOL, (tag, tip)
    assert _same_rows(g["contacts"], o_contacts), (tag, "contact sets differ")
    fg, fo = _node_forces(g["contacts"]), _node_forces(o_contacts)
    fmax = max([np.linalg.norm(v) for v in fo.values()] + [1e-300])
    for n in fo:
        assert np.linalg.norm(fg[n] - fo[n]) <= FORCE_RTOL * fmax, (tag, n)
    return tip


def test_mixed_bent_tube_matches_oracle(af):
    w = wl.bent_tube_workload(0, n_steps=10)
    gpu = af.AccFem(w.robot, w.lumen)
    assert gpu.accfem_set_precision(af.PRECISION_MIXED) == af.OK
    ref = solver.Model(w.robot, w.lumen)
    worst = 0.0
    for s in range(len(w.insertions)):
        g = gpu.accfem_solve(w.tensions[s], w.insertions[s])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert g["status"] == af.OK and o.status == solver.OK, (s, g["error"])
        worst = max(worst, _check(g, o.node_pos, o.contacts, "step %d" % s))
    assert len(g["contacts"]) >= 4
    gpu.close()


def test_mixed_matches_fp64_on_an_uneven_instance(af):
    """Instance 2 of the batched workload (961 elements, own lumen), first 12 steps: mixed vs FP64
    GPU solves of the same sequence."""
    w = wl.batch_workloads(first=2, count=1)[0]
    a = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    b = af.AccFem(w.robot, w.lumen, max_contacts=4096)
    assert b.accfem_set_precision(af.PRECISION_MIXED) == af.OK
    for s in range(12):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert ra["status"] == af.OK and rb["status"] == af.OK, (s, ra["error"], rb["error"])
        _check(rb, ra["node_pos"], ra["contacts"], "step %d" % s)
    a.close()
    b.close()


def test_precision_mode_arguments(af):
    w = wl.bent_tube_workload(0, n_steps=2)
    h = af.AccFem(w.robot, w.lumen)
    assert h.accfem_set_precision(2) == af.E_INVALID_ARG
    assert h.accfem_set_precision(-1) == af.E_INVALID_ARG
    # switching modes between solves re-captures the Newton graph; FP64 after mixed gives the FP64 result
    r64 = h.accfem_solve(w.tensions[0], w.insertions[0])
    h.accfem_reset()
    assert h.accfem_set_precision(af.PRECISION_MIXED) == af.OK
    h.accfem_solve(w.tensions[0], w.insertions[0])
    h.accfem_reset()
    assert h.accfem_set_precision(af.PRECISION_FP64) == af.OK
    r64b = h.accfem_solve(w.tensions[0], w.insertions[0])
    assert np.array_equal(r64["node_pos"], r64b["node_pos"])
    h.close()
