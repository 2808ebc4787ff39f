"""The paper's printed material settings (Table 1; lengths from Sec. IV.B) as fixtures: a hollow
circular section with the printed area A and second moment I has r_o^2 + r_i^2 = 4 I / A and
r_o^2 - r_i^2 = A / pi.  The oracle's section constants (Sec. II.B) must give back E A and E I, and
its solve of the 470 mm tube as a cantilever must give the printed stiffness's tip deflection
P L^3 / (3 E I) (small deflection), also with the 70 mm flexible section softened."""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import workloads as wl
from oracle import beam, solver

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "table1_materials.json")))


def _robot(row, n_elements):
    A, I = row["area_m2"], row["inertia_m4"]
    s2, d2 = 4.0 * I / A, A / math.pi
    ro, ri = math.sqrt(0.5 * (s2 + d2)), math.sqrt(0.5 * (s2 - d2))
    return wl.robot_desc(GOLD["length_m"], n_elements, outer_radius=ro, inner_radius=ri,
                         youngs_modulus=row["youngs_modulus_MPa"] * 1e6)


@pytest.mark.parametrize("row", GOLD["rows"], ids=[r["experiment"] for r in GOLD["rows"]])
def test_section_constants_reproduce_table1(row):
    sec = beam.section_constants(_robot(row, 47))
    E = row["youngs_modulus_MPa"] * 1e6
    assert sec["EA"] == pytest.approx(E * row["area_m2"], rel=1e-12)
    assert sec["EI"] == pytest.approx(E * row["inertia_m4"], rel=1e-12)


@pytest.mark.parametrize("row", GOLD["rows"][:2], ids=["a", "b"])
def test_table1_cantilever(row):
    L = GOLD["length_m"]
    rob = _robot(row, 47)
    EI = row["youngs_modulus_MPa"] * 1e6 * row["inertia_m4"]
    P = 3 * EI * 1e-5 * L / L ** 3                      # tip deflection 1e-5 L
    m = solver.Model(rob, wl.free_space_lumen(), solver.Options(step_limit=1.0))
    r = m.solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK
    assert r.node_pos[-1, 1] == pytest.approx(P * L ** 3 / (3 * EI), rel=1e-8)
    # the flexible distal section (the last 70 mm, here at a tenth of the modulus): unit-load
    # integral over the two stiffnesses, EI on [0, L - s] and EI / 10 beyond
    s = GOLD["flexible_section_m"]
    soft = replace(rob, element_youngs=wl.soft_tip_moduli(rob, soft_length=s, soft_ratio=0.1))
    Es = soft.element_youngs
    assert np.count_nonzero(Es < Es.max()) == 7                  # 10 mm elements: 70 mm
    m = solver.Model(soft, wl.free_space_lumen(), solver.Options(step_limit=1.0))
    r = m.solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    v = P * (L ** 3 - s ** 3) / (3 * EI) + P * s ** 3 / (3 * EI / 10)
    assert r.status == solver.OK and r.node_pos[-1, 1] == pytest.approx(v, rel=1e-8)
