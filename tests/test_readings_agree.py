"""The oracle and the CUDA path share no code, so the readings of the paper that both must apply
are checked to agree: the solve options that define the problem and its convergence test (the C
ABI's defaults against the oracle's), the barycentric face band of the constraint rows and the
contact compliance factor (read from the CUDA sources as text)."""
import os
import re

import pytest

from oracle import contact, solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_06922_gb300", "csrc")


@pytest.fixture(scope="module")
def af():
    from paper_2503_06922_gb300 import accfem
    if not os.path.exists(accfem.LIB_PATH):
        from paper_2503_06922_gb300 import build
        build.build()
    accfem.load()
    return accfem


def test_default_options_agree(af):
    o = af.accfem_default_options()
    d = solver.Options()
    assert o.activation_gap == d.activation_gap
    assert o.step_limit == d.step_limit
    assert o.newton_tol == d.newton_tol
    assert o.max_newton_iters == d.max_newton_iters
    assert o.tangent_mode == d.tangent_mode == 0


def test_face_band_and_compliance_agree():
    common = open(os.path.join(CSRC, "common.cuh")).read()
    band = float(re.search(r"constexpr double kFaceBand = ([0-9.eE+-]+);", common).group(1))
    assert band == contact.FACE_BAND
    src = open(os.path.join(CSRC, "contact.cu")).read()
    comp = float(re.search(r"const double eps_w = ([0-9.eE+-]+) \* wd;", src).group(1))
    assert comp == solver.CONTACT_COMPLIANCE
