"""accfem_time_kernel and accfem_time_kernel_graph (measurement entry points): both time every
listed kernel on the resident state of the last solve and leave that state as it was, so the next
warm-started solve equals the one of a handle that timed nothing."""
import numpy as np
import pytest

import workloads as wl

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


KERNELS = ("KERNEL_ELEMENT", "KERNEL_COLLIDE", "KERNEL_ASSEMBLE", "KERNEL_CONTACT", "KERNEL_FACTOR")


def test_timing_keeps_the_resident_state(af):
    w = wl.bent_tube_workload(0, n_steps=10)
    a = af.AccFem(w.robot, w.lumen)
    b = af.AccFem(w.robot, w.lumen)
    for s in range(8):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert ra["status"] == af.OK
    assert len(ra["contacts"]) > 0
    pos0, quat0 = a.accfem_get_state()
    for name in KERNELS:
        k = getattr(af, name)
        host = a.accfem_time_kernel(k, 5)
        graph = a.accfem_time_kernel_graph(k, 5)
        assert host > 0.0 and graph > 0.0, name
    pos1, quat1 = a.accfem_get_state()
    assert np.array_equal(pos0, pos1) and np.array_equal(quat0, quat1)
    for s in range(8, 10):
        ra = a.accfem_solve(w.tensions[s], w.insertions[s])
        rb = b.accfem_solve(w.tensions[s], w.insertions[s])
        assert ra["status"] == af.OK
        assert ra["newton_iters"] == rb["newton_iters"]
        assert np.array_equal(ra["node_pos"], rb["node_pos"]) and np.array_equal(ra["node_quat"], rb["node_quat"])
    with pytest.raises(RuntimeError):
        a.accfem_time_kernel_graph(af.KERNEL_FACTOR, 0)
    a.close()
    b.close()
