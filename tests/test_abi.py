"""The C-ABI library loads and exports every entry point that include/accfem.h declares; host-side
argument validation answers with status codes (no GPU compute is called here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_06922_gb300 import accfem as af
    if not os.path.exists(af.LIB_PATH):
        from paper_2503_06922_gb300 import build
        build.build()
    return af.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "accfem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(accfem_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("accfem_create", "accfem_solve", "accfem_destroy", "accfem_default_options", "accfem_get_state",
              "accfem_solve_tip_load", "accfem_status_string", "accfem_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2503_06922_gb300 import accfem as af
    assert sorted(af.EXPORTS) == _declared()


def test_default_options_and_status_strings(lib):
    from paper_2503_06922_gb300 import accfem as af
    o = af.accfem_default_options()
    assert o.activation_gap == 1e-3 and o.step_limit == 5e-4 and o.newton_tol == 1e-11
    assert o.max_newton_iters == 200 and o.max_contacts == 256 and o.tangent_mode == 0
    assert lib.accfem_default_options(None) == af.E_INVALID_ARG
    for s in range(9):
        assert len(af.accfem_status_string(s)) > 0


def test_invalid_descriptors_are_rejected_before_any_device_work(lib):
    from paper_2503_06922_gb300 import accfem as af
    w = wl.bent_tube_workload(0)
    bad_robots = [dict(length=-1.0), dict(inner_radius=3e-3), dict(n_elements=0), dict(poisson_ratio=0.6)]
    for kw in bad_robots:
        r = wl.robot_desc(**{**dict(length=0.12, n_elements=20), **kw})
        with pytest.raises(RuntimeError, match="invalid argument"):
            af.AccFem(r, w.lumen)
    lum = wl.LumenDesc(vertices=w.lumen.vertices, triangles=w.lumen.triangles.copy(), entrance_point=w.lumen.entrance_point,
                       entrance_dir=np.zeros(3), entrance_up=w.lumen.entrance_up)
    with pytest.raises(RuntimeError, match="invalid argument"):
        af.AccFem(w.robot, lum)
    T = w.lumen.triangles.copy()
    T[5, 1] = len(w.lumen.vertices) + 3          # vertex index out of range
    lum = wl.LumenDesc(vertices=w.lumen.vertices, triangles=T, entrance_point=w.lumen.entrance_point,
                       entrance_dir=w.lumen.entrance_dir, entrance_up=w.lumen.entrance_up)
    with pytest.raises(RuntimeError, match="invalid argument"):
        af.AccFem(w.robot, lum)
    with pytest.raises(RuntimeError, match="invalid argument"):
        af.AccFem(w.robot, w.lumen, tangent_mode=1)
    H = ctypes.c_void_p()
    assert lib.accfem_create(None, None, None, ctypes.byref(H)) == af.E_INVALID_ARG


def test_setters_and_queries_reject_a_null_handle(lib):
    """Every entry point taking a handle answers E_INVALID_ARG for NULL before touching a device."""
    from paper_2503_06922_gb300 import accfem as af
    E = np.zeros(20)
    assert lib.accfem_set_precision(None, 0) == af.E_INVALID_ARG
    assert lib.accfem_set_frame_mode(None, 1) == af.E_INVALID_ARG
    assert lib.accfem_set_contact_solver(None, 0) == af.E_INVALID_ARG
    assert lib.accfem_set_element_modulus(None, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 20) == af.E_INVALID_ARG
    assert lib.accfem_set_stream(None, None) == af.E_INVALID_ARG
    assert lib.accfem_reset(None) == af.E_INVALID_ARG
    n = ctypes.c_int64()
    assert lib.accfem_device_bytes(None, ctypes.byref(n)) == af.E_INVALID_ARG
    assert lib.accfem_batch_autotune(None, 1) == af.E_INVALID_ARG
