"""Pins of the oracle's quasi-static solve (Eq. 1-29) against mechanics closed forms,
an independently integrated elastica, limiter/tangent independence and non-penetration."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

import workloads as wl
from oracle import beam, contact, solver
from oracle.rotation import from_quat, logm

L, M = 0.12, 20
ROB = wl.robot_desc(L, M)
SEC = beam.section_constants(ROB)
EI, EA, GJ = SEC["EI"], SEC["EA"], SEC["GJ"]


def _model(robot=ROB, lumen=None, **opt):
    return solver.Model(robot, lumen if lumen is not None else wl.free_space_lumen(), solver.Options(**opt))


def test_small_deflection_cantilever():
    """P3: tip deflection P L^3 / (3 EI) for a dead transverse tip load, delta/L ~ 1e-5."""
    P = 3 * EI * 1.2e-6 / L ** 3
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK
    assert r.node_pos[-1, 1] == pytest.approx(P * L ** 3 / (3 * EI), rel=1e-8)
    # every node: v(x) = P x^2 (3L - x) / (6 EI)
    x = np.arange(M + 1) * L / M
    assert np.allclose(r.node_pos[:, 1], P * x ** 2 * (3 * L - x) / (6 * EI), rtol=1e-8, atol=1e-18)


def test_pure_end_moment_arc():
    """P4: a tip moment M bends the chain into a polygon inscribed in a circle: every chord
    keeps l0, successive chords turn by phi = M l0 / EI, the tip turns by M L / EI."""
    Mz = 0.5 * math.pi * EI / L
    r = _model(step_limit=5e-3).solve(delta=L, tip_load=((0.0, 0.0, 0.0), (0.0, 0.0, Mz), False))
    assert r.status == solver.OK
    l0 = L / M
    phi = Mz * l0 / EI
    ang = (np.arange(M) + 0.5) * phi
    chords = l0 * np.column_stack([np.cos(ang), np.sin(ang), np.zeros(M)])
    pos = np.vstack([np.zeros(3), np.cumsum(chords, axis=0)])
    assert np.abs(r.node_pos - pos).max() <= 1e-10 * L
    for i in (5, M):
        R = from_quat(r.node_quat[i])
        assert np.allclose(logm(R), [0, 0, i * phi], atol=1e-10)
    # circle of radius l0 / (2 sin(phi/2)) through the nodes
    rad = l0 / (2 * math.sin(phi / 2))
    ctr = np.array([0.0, rad, 0.0])
    assert np.allclose(np.linalg.norm(r.node_pos - ctr, axis=1), rad, rtol=1e-10)


def test_axial_and_torsion():
    """P5: elongation P L / EA for a tip tension; twist T L / GJ for a tip torque (any angle)."""
    P = 50.0
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((P, 0.0, 0.0), (0.0, 0.0, 0.0), False))
    assert r.node_pos[-1, 0] == pytest.approx(L + P * L / EA, rel=1e-12)
    T = 1.0 * GJ / L
    r = _model(step_limit=1.0).solve(delta=L, tip_load=((0.0, 0.0, 0.0), (T, 0.0, 0.0), False))
    assert r.status == solver.OK
    tw = logm(from_quat(r.node_quat[-1]))
    assert tw[0] == pytest.approx(T * L / GJ, rel=1e-12) and abs(tw[1]) + abs(tw[2]) <= 1e-12
    assert np.abs(r.node_pos[:, 1:]).max() <= 1e-15


def test_equal_cable_tensions_compress_straight():
    """P6: equal tensions give zero tip moment (Eq. 16-18) and a pure follower compression:
    the robot stays straight and shortens by sum(tau) L / EA."""
    tau = np.array([2.0, 2.0, 2.0])
    r = _model(step_limit=1.0).solve(tensions=tau, delta=L)
    assert r.status == solver.OK
    assert r.node_pos[-1, 0] == pytest.approx(L - tau.sum() * L / EA, rel=1e-12)
    assert np.abs(r.node_pos[:, 1:]).max() <= 1e-15
    f, mo = solver.cable_load(np.eye(3), tau, ROB)
    assert np.allclose(f, [-6.0, 0, 0]) and np.abs(mo).max() <= 1e-15
    # a single cable at angle 0 bends towards +y: moment r_c tau about +z
    f, mo = solver.cable_load(np.eye(3), [1.0, 0.0, 0.0], ROB)
    assert np.allclose(mo, [0.0, 0.0, ROB.cable_radius], atol=1e-18)


def test_one_wall_tip_contact_closed_form():
    """P11: tip pressed by a dead load P onto a wall at gap g: y = P - 3 EI g / L^3
    (small-deflection superposition), and the tip rests on the wall."""
    g = 1e-6
    P = 2 * 3 * EI * g / L ** 3
    lum = wl.patch_lumen(L - 0.002, L + 0.006, ROB.outer_radius + g)
    r = _model(lumen=lum, step_limit=1.0).solve(delta=L, tip_load=((0.0, P, 0.0), (0.0, 0.0, 0.0), False))
    assert r.status == solver.OK
    assert len(r.contacts) == 1 and r.contacts[0]["node"] == M
    assert r.contacts[0]["force"] == pytest.approx(P - 3 * EI * g / L ** 3, rel=1e-6)
    assert r.node_pos[-1, 1] == pytest.approx(g, rel=1e-9)


def _elastica_tip(P, Lf):
    """Tip of an extensible elastica (Euler-Bernoulli: no shear) under a dead end load -P e_y,
    s the material arc length: EI theta' = M = -P (x_tip - x), axial strain eps = N / EA with
    N = -P sin(theta), so theta'' = P (1 + eps) cos(theta) / EI, x' = (1 + eps) cos(theta),
    y' = (1 + eps) sin(theta); theta(0) = 0, theta'(Lf) = 0; shooting on theta'(0)."""
    def run(k0):
        def f(s, u):
            eps = -P * math.sin(u[0]) / EA
            return [u[1], P / EI * (1 + eps) * math.cos(u[0]), (1 + eps) * math.cos(u[0]), (1 + eps) * math.sin(u[0])]
        return solve_ivp(f, (0, Lf), [0.0, k0, 0.0, 0.0], rtol=1e-13, atol=1e-15, method="DOP853").y[:, -1]
    k0 = brentq(lambda k: run(k)[1], -P * Lf / EI * 1.5, 0.0, xtol=1e-15)
    return run(k0)[2:]


def test_large_deflection_converges_to_elastica():
    """P8: tip position error vs the elastica decreases by ~4x per mesh halving (O(h^2))."""
    P = 2.0 * EI / L ** 2
    exact = _elastica_tip(P, L)
    errs = []
    for m in (6, 12, 24):
        rob = wl.robot_desc(L, m)
        r = _model(robot=rob, step_limit=4e-3).solve(delta=L, tip_load=((0.0, -P, 0.0), (0.0, 0.0, 0.0), False))
        assert r.status == solver.OK
        errs.append(np.linalg.norm(r.node_pos[-1, :2] - exact))
    assert exact[1] < -0.3 * L              # genuinely large deflection
    assert errs[2] < 1e-3 * L
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0


def test_limiter_and_tangent_do_not_change_the_equilibrium():
    """P7: the converged state does not depend on beta0 or on the tangent used in the QP."""
    lum = wl.patch_lumen(L - 0.03, L + 0.01, ROB.outer_radius + 2e-3, n=3)
    load = ((0.0, 3.0, 0.0), (0.0, 0.0, 0.0), False)
    ref = _model(lumen=lum, step_limit=5e-4).solve(delta=L, tip_load=load)
    assert ref.status == solver.OK and len(ref.contacts) >= 1
    for kw in ({"step_limit": 1e-4}, {"step_limit": 5e-4, "tangent_mode": 1}):
        r = _model(lumen=lum, **kw).solve(delta=L, tip_load=load)
        assert r.status == solver.OK
        assert np.abs(r.node_pos - ref.node_pos).max() <= 1e-10 * L
        assert [c["node"] for c in r.contacts] == [c["node"] for c in ref.contacts]
        assert np.allclose([c["force"] for c in r.contacts], [c["force"] for c in ref.contacts], rtol=1e-7, atol=1e-12)


def test_acceleration_changes_the_path_not_the_equilibrium(bent_sweep):
    """Anderson acceleration of the Newton iteration only changes the path: on the bent-tube sweep the
    converged states equal those of the unaccelerated iteration (1e-10 L), with the same contact rows
    and forces, in fewer iterations; with no held iterate (depth 0) the step is the plain limited one."""
    w, m, res = bent_sweep
    plain = solver.Model(w.robot, w.lumen, solver.Options(accel_depth=0))
    its_a = its_p = 0
    for s, ra in enumerate(res):
        rp = plain.solve(w.tensions[s], w.insertions[s])
        assert rp.status == solver.OK and ra.status == solver.OK
        assert np.abs(rp.node_pos - ra.node_pos).max() <= 1e-10 * w.robot.length, s
        assert [(c["node"], c["tri"]) for c in rp.contacts] == [(c["node"], c["tri"]) for c in ra.contacts], s
        assert np.allclose([c["force"] for c in rp.contacts], [c["force"] for c in ra.contacts], rtol=1e-6, atol=1e-10)
        its_a += ra.newton_iters
        its_p += rp.newton_iters
    assert its_a < 0.9 * its_p, (its_a, its_p)


def test_acceleration_removes_a_linear_tail():
    """On an affine fixed-point map (no contacts, small load: the material-tangent iteration converges
    linearly on the small-deflection cantilever), depth-3 acceleration converges in fewer iterations
    than the plain iteration, to the same state, and its steps shrink faster than linearly at the end."""
    P = 0.2
    load = ((0.0, P, 0.0), (0.0, 0.0, 0.05), True)
    a = _model(step_limit=1.0).solve(delta=L, tip_load=load)
    b = _model(step_limit=1.0, accel_depth=0).solve(delta=L, tip_load=load)
    assert a.status == b.status == solver.OK
    assert np.abs(a.node_pos - b.node_pos).max() <= 1e-10 * L
    assert a.newton_iters < b.newton_iters, (a.newton_iters, b.newton_iters)


@pytest.fixture(scope="module")
def bent_sweep():
    w = wl.bent_tube_workload(0, n_steps=10)
    m = solver.Model(w.robot, w.lumen)
    res = [m.solve(w.tensions[s], w.insertions[s]) for s in range(8)]
    return w, m, res


def test_bent_tube_sweep_converges_with_contacts(bent_sweep):
    w, m, res = bent_sweep
    assert all(r.status == solver.OK for r in res)
    assert len(res[-1].contacts) >= 2 and max(c["force"] for c in res[-1].contacts) > 0.1


def test_non_penetration_and_complementarity(bent_sweep):
    """P13: every free node keeps r_o clearance from every triangle (1e-9 m), contact forces are
    non-negative and a loaded constraint is closed (gap ~ 0)."""
    w, m, res = bent_sweep
    r = res[-1]
    V, T = w.lumen.vertices, w.lumen.triangles
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    k = solver.n_prescribed_last(w.robot.length, w.robot.n_elements, w.insertions[7])
    nf = contact.face_normals(V, T)
    for i in range(k + 1, w.robot.n_elements + 1):
        p = r.node_pos[i]
        cp, d, _, _ = contact.closest_points_all(p, A, B, C)
        t = int(np.argmin(d))
        assert d[t] >= w.robot.outer_radius - 1e-9
        assert np.dot(nf[t], cp[t] - p) > 0           # on the lumen side
    for c in r.contacts:
        assert c["force"] >= 0.0
        if c["force"] > 1e-6:
            p = r.node_pos[c["node"]]
            gap = np.dot(c["normal"], c["point"] - p) - w.robot.outer_radius
            assert abs(gap) <= 1e-9


def test_base_reaction_balances_every_external_load():
    """The reported base reaction is F(x) at the last prescribed node: the strain energy is invariant
    under rigid motions, so the internal forces of the chain sum to zero and the clamp's reaction
    balances every external load on the free nodes -- force -(sum f) and moment -(sum (x_i - x_k) x f_i
    + sum m_i) -- at any deflection, with contacts included."""
    f = np.array([0.0, 0.8, 0.3])
    mo = np.array([0.01, 0.0, 0.02])
    r = _model(step_limit=5e-3).solve(delta=L, tip_load=(tuple(f), tuple(mo), False))
    assert r.status == solver.OK
    assert np.allclose(r.base_reaction[:3], -f, atol=1e-10)
    assert np.allclose(r.base_reaction[3:], -(np.cross(r.node_pos[-1] - r.node_pos[0], f) + mo), atol=1e-10)
    # bent tube: follower cable load of Eq. 16-18 and the contact forces -y_i n_i
    w = wl.bent_tube_workload(0, n_steps=10)
    m = solver.Model(w.robot, w.lumen)
    for s in range(len(w.insertions)):
        rb = m.solve(w.tensions[s], w.insertions[s])
    assert rb.status == solver.OK and len(rb.contacts) > 0
    k = solver.n_prescribed_last(w.robot.length, w.robot.n_elements, w.insertions[-1])
    xk = rb.node_pos[k]
    fc, mc = solver.cable_load(from_quat(rb.node_quat[-1]), w.tensions[-1], w.robot)
    F = fc.copy()
    Mo = np.cross(rb.node_pos[-1] - xk, fc) + mc
    for c in rb.contacts:
        fi = -c["force"] * np.asarray(c["normal"])
        F += fi
        Mo += np.cross(rb.node_pos[c["node"]] - xk, fi)
    assert np.allclose(rb.base_reaction[:3], -F, atol=1e-6)
    assert np.allclose(rb.base_reaction[3:], -Mo, atol=1e-8)
