"""The oracle's own floor, which sets how tight a parity tolerance can be (the self-consistency pin
of the hot-path scope): on the 120 mm bent-tube sweep with contacts,
  * rounding: moving every lumen vertex or every cable tension by one ulp moves the converged
    poses by about 1e-15 relative;
  * stopping point: a solve stopped at the default step tolerance (1e-11 m) and one carried on to
    1e-13 m differ by about 1e-11 relative.
Two correct implementations stop at different iterates, so they may differ by the second amount;
the GPU parity tolerance of 1e-9 relative sits two orders of magnitude above it."""
from dataclasses import replace

import numpy as np

import workloads as wl
from oracle import solver

PARITY_REL = 1e-9


def test_rounding_and_stopping_floors():
    w = wl.bent_tube_workload(0, n_steps=10)
    base = solver.Model(w.robot, w.lumen)
    ulp_mesh = solver.Model(w.robot, replace(w.lumen, vertices=np.nextafter(w.lumen.vertices, np.inf)))
    ulp_load = solver.Model(w.robot, w.lumen)
    tight = solver.Model(w.robot, w.lumen, solver.Options(newton_tol=1e-13))
    rounding = stopping = 0.0
    rows = 0
    for s in range(len(w.insertions)):
        r0 = base.solve(w.tensions[s], w.insertions[s])
        r1 = ulp_mesh.solve(w.tensions[s], w.insertions[s])
        r2 = ulp_load.solve(np.nextafter(w.tensions[s], np.inf), w.insertions[s])
        r3 = tight.solve(w.tensions[s], w.insertions[s])
        assert all(r.status == solver.OK for r in (r0, r1, r2, r3))
        sc = np.abs(r0.node_pos).max()
        rounding = max(rounding, np.abs(r1.node_pos - r0.node_pos).max() / sc,
                       np.abs(r2.node_pos - r0.node_pos).max() / sc)
        stopping = max(stopping, np.abs(r3.node_pos - r0.node_pos).max() / sc)
        rows += len(r0.contacts)
    assert rows > 0
    assert rounding <= 1e-13, rounding
    assert stopping <= 1e-10, stopping
    assert PARITY_REL >= 10 * stopping
