"""Pins of the oracle with a non-uniform robot (Sec. II.A: a distal section much less rigid than
the rest; each element carries its own Young's modulus).  Closed forms of Euler-Bernoulli beams
with element-wise constant stiffness: axial and torsional compliances add in series, the
small-deflection cantilever follows the unit-load integral, a pure end moment turns each element
by M l0 / EI_e and keeps every chord at l0."""
import math
from dataclasses import replace

import numpy as np
import pytest

import workloads as wl
from oracle import beam, solver
from oracle.rotation import from_quat, logm

L, M = 0.12, 20
l0 = L / M
BASE = wl.robot_desc(L, M)
RATIO = np.random.default_rng(40).uniform(0.2, 1.0, M)
ROB = replace(BASE, element_youngs=BASE.youngs_modulus * RATIO)
SECS = beam.element_sections(ROB)
EA = np.array([s["EA"] for s in SECS])
EI = np.array([s["EI"] for s in SECS])
GJ = np.array([s["GJ"] for s in SECS])


def _model(robot=ROB, lumen=None, **opt):
    return solver.Model(robot, lumen if lumen is not None else wl.free_space_lumen(), solver.Options(**opt))


def test_element_sections_follow_the_moduli():
    base = beam.section_constants(BASE)
    for e, s in enumerate(SECS):
        for k in ("EA", "EI", "GJ"):
            assert s[k] == pytest.approx(base[k] * RATIO[e], rel=1e-15)
        assert s["l0"] == base["l0"]
    assert beam.element_sections(BASE) == [base] * M


def test_soft_tip_generator():
    E = wl.soft_tip_moduli(wl.robot_desc(0.6, 300), soft_length=0.07, soft_ratio=0.1)
    # 2 mm elements: midpoints beyond 530 mm are soft -> the last 35 elements
    assert np.count_nonzero(E < 2.0e9) == 35 and np.all(E[-35:] == 2.0e8) and np.all(E[:-35] == 2.0e9)


def test_series_axial_and_torsion():
    """Tip tension P: elongation P sum(l0 / EA_e); tip torque T: twist T sum(l0 / GJ_e)."""
    P = 50.0
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((P, 0.0, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK
    assert r.node_pos[-1, 0] == pytest.approx(L + P * np.sum(l0 / EA), rel=1e-12)
    # every node: cumulative elongation
    x = np.concatenate([[0.0], np.cumsum(l0 + P * l0 / EA)])
    assert np.allclose(r.node_pos[:, 0], x, rtol=1e-12, atol=0.0)
    T = 0.5 * GJ.min() / L
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((0.0, 0.0, 0.0), (T, 0.0, 0.0), False))
    assert r.status == solver.OK
    tw = logm(from_quat(r.node_quat[-1]))
    assert tw[0] == pytest.approx(T * np.sum(l0 / GJ), rel=1e-12) and abs(tw[1]) + abs(tw[2]) <= 1e-12


def _unit_load_deflection(P, x):
    """v(x) = int_0^x P (L - s)(x - s) / EI(s) ds with EI constant on each element; the integrand's
    antiderivative is L x s - (L + x) s^2 / 2 + s^3 / 3."""
    def F(s):
        return L * x * s - (L + x) * s * s / 2.0 + s ** 3 / 3.0
    v = 0.0
    for e in range(M):
        a, b = e * l0, min((e + 1) * l0, x)
        if b <= a:
            break
        v += P * (F(b) - F(a)) / EI[e]
    return v


def test_piecewise_small_deflection_cantilever():
    """Dead transverse tip load P, delta/L ~ 1e-5: every node on the unit-load deflection."""
    P = 3 * EI.min() * 1.2e-6 / L ** 3
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK
    v = np.array([_unit_load_deflection(P, i * l0) for i in range(M + 1)])
    assert r.node_pos[-1, 1] == pytest.approx(v[-1], rel=1e-8)
    assert np.allclose(r.node_pos[:, 1], v, rtol=1e-8, atol=1e-18)
    # the uniform closed form is far off: the pin sees the per-element moduli
    uni = P * L ** 3 / (3 * beam.section_constants(BASE)["EI"])
    assert abs(v[-1] - uni) > 0.1 * uni


def test_piecewise_pure_end_moment():
    """A tip moment Mz: element e turns by phi_e = Mz l0 / EI_e, node i by the sum of the phi of
    the elements before it, and every chord keeps length l0 at the mean of its end rotations."""
    Mz = 0.4 * math.pi / np.sum(l0 / EI)
    r = _model(step_limit=5e-3).solve(delta=L, tip_load=((0.0, 0.0, 0.0), (0.0, 0.0, Mz), False))
    assert r.status == solver.OK
    phi = Mz * l0 / EI
    psi = np.concatenate([[0.0], np.cumsum(phi)])
    ang = psi[:-1] + 0.5 * phi
    chords = l0 * np.column_stack([np.cos(ang), np.sin(ang), np.zeros(M)])
    pos = np.vstack([np.zeros(3), np.cumsum(chords, axis=0)])
    assert np.abs(r.node_pos - pos).max() <= 1e-10 * L
    for i in (3, 11, M):
        assert np.allclose(logm(from_quat(r.node_quat[i])), [0, 0, psi[i]], atol=1e-10)


def test_equal_tensions_shorten_in_series():
    tau = np.array([1.5, 1.5, 1.5])
    r = _model(step_limit=1.0).solve(tensions=tau, delta=L)
    assert r.status == solver.OK
    assert r.node_pos[-1, 0] == pytest.approx(L - tau.sum() * np.sum(l0 / EA), rel=1e-12)
    assert np.abs(r.node_pos[:, 1:]).max() <= 1e-15


def test_uniform_moduli_equal_the_uniform_robot():
    """An explicit array of the robot's own modulus reproduces the uniform robot bit for bit."""
    w = wl.bent_tube_workload(0, n_steps=3)
    a = solver.Model(w.robot, w.lumen)
    b = solver.Model(replace(w.robot, element_youngs=np.full(w.robot.n_elements, w.robot.youngs_modulus)), w.lumen)
    for s in range(3):
        ra = a.solve(w.tensions[s], w.insertions[s])
        rb = b.solve(w.tensions[s], w.insertions[s])
        assert np.array_equal(ra.node_pos, rb.node_pos) and ra.newton_iters == rb.newton_iters
