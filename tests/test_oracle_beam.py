"""Pins of the oracle's corotational element (Sec. II.B, Eq. 20): invariants, finite
differences of the strain energy and of the force, and the textbook linear stiffness."""
import numpy as np
import pytest

import workloads as wl
from oracle import beam
from oracle.rotation import expm, logm, tsinv, to_quat, from_quat

SEC = beam.section_constants(wl.robot_desc(0.12, 20))


def _random_element(rng, scale=0.05):
    xa = rng.normal(size=3) * 0.01
    Ta = expm(rng.normal(size=3))
    xb = xa + Ta[:, 0] * SEC["l0"] * (1 + 0.01 * rng.normal()) + rng.normal(size=3) * 1e-4
    Tb = expm(rng.normal(size=3) * scale) @ Ta
    return xa, Ta, xb, Tb


def _perturbed(k, s, xa, Ta, xb, Tb):
    e = np.zeros(3); e[k % 3] = s
    blk = k // 3
    if blk == 0:
        return xa + e, Ta, xb, Tb
    if blk == 1:
        return xa, expm(e) @ Ta, xb, Tb
    if blk == 2:
        return xa, Ta, xb + e, Tb
    return xa, Ta, xb, expm(e) @ Tb


def test_section_constants_closed_form():
    ro, ri, E, nu = 2e-3, 1e-3, 2.0e9, 0.35
    assert SEC["EA"] == pytest.approx(E * np.pi * (ro ** 2 - ri ** 2), rel=1e-15)
    assert SEC["EI"] == pytest.approx(E * np.pi * (ro ** 4 - ri ** 4) / 4, rel=1e-15)
    assert SEC["GJ"] == pytest.approx(E / (2 * (1 + nu)) * np.pi * (ro ** 4 - ri ** 4) / 2, rel=1e-15)
    assert SEC["l0"] == pytest.approx(0.006, rel=1e-15)


def test_rotation_maps_roundtrip():
    rng = np.random.default_rng(1)
    for _ in range(50):
        th = rng.normal(size=3)
        th *= rng.uniform(0, 3.0) / np.linalg.norm(th)
        R = expm(th)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-15)
        assert np.allclose(logm(R), th, atol=1e-12)
        assert np.allclose(from_quat(to_quat(R)), R, atol=1e-15)
    # Tsinv is the inverse of the spatial tangent map of exp: finite differences
    th = np.array([0.3, -0.2, 0.5]); h = 1e-6
    for k in range(3):
        e = np.zeros(3); e[k] = h
        dth = (logm(expm(e) @ expm(th)) - logm(expm(-e) @ expm(th))) / (2 * h)
        assert np.allclose(dth, tsinv(th)[:, k], atol=1e-8)


def test_rigid_motion_gives_zero_force():
    """P1: any rigid motion of an unstrained element leaves F = 0."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        Q = expm(rng.normal(size=3) * 2)
        t = rng.normal(size=3)
        xa = t; xb = t + Q[:, 0] * SEC["l0"]
        F = beam.internal_force(xa, Q, xb, Q, SEC)
        # rounding floor: EA/l0 times the spacing of doubles at |x|
        floor = SEC["EA"] / SEC["l0"] * np.finfo(float).eps * (np.abs(t).max() + SEC["l0"])
        assert np.abs(F).max() <= 20 * floor


def test_force_covariance_and_balance():
    """P1: F(Q x + t, Q T) = Q F(x, T) blockwise; forces and moments about the origin balance."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        xa, Ta, xb, Tb = _random_element(rng)
        F = beam.internal_force(xa, Ta, xb, Tb, SEC)
        assert np.abs(F[0:3] + F[6:9]).max() <= 1e-12 * np.abs(F).max()
        mom = F[3:6] + F[9:12] + np.cross(xa, F[0:3]) + np.cross(xb, F[6:9])
        assert np.abs(mom).max() <= 1e-12 * np.abs(F).max()
        Q = expm(rng.normal(size=3)); t = rng.normal(size=3)
        G = beam.internal_force(Q @ xa + t, Q @ Ta, Q @ xb + t, Q @ Tb, SEC)
        QF = np.concatenate([Q @ F[3 * i:3 * i + 3] for i in range(4)])
        assert np.allclose(G, QF, rtol=0, atol=1e-10 * np.abs(F).max())


def test_force_is_energy_gradient():
    """P2: F = dU/dd under spin variations (central differences of the strain energy)."""
    rng = np.random.default_rng(4)
    for _ in range(4):
        xa, Ta, xb, Tb = _random_element(rng)
        F = beam.internal_force(xa, Ta, xb, Tb, SEC)
        h = 1e-7
        g = np.array([(beam.strain_energy(*_perturbed(k, h, xa, Ta, xb, Tb), SEC)
                       - beam.strain_energy(*_perturbed(k, -h, xa, Ta, xb, Tb), SEC)) / (2 * h) for k in range(12)])
        assert np.abs(F - g).max() <= 1e-7 * np.abs(F).max()


def test_consistent_tangent_matches_fd_of_force():
    """P2: K_T = dF/dd (central differences, O(h^2))."""
    rng = np.random.default_rng(5)
    xa, Ta, xb, Tb = _random_element(rng)
    KT = beam.consistent_tangent(xa, Ta, xb, Tb, SEC)
    h = 1e-6
    KF = np.column_stack([(beam.internal_force(*_perturbed(k, h, xa, Ta, xb, Tb), SEC)
                           - beam.internal_force(*_perturbed(k, -h, xa, Ta, xb, Tb), SEC)) / (2 * h) for k in range(12)])
    assert np.abs(KT - KF).max() <= 1e-7 * np.abs(KT).max()


def test_material_tangent_is_textbook_at_rest_and_psd():
    """P2: K_M equals the linear 12x12 Euler-Bernoulli stiffness at the undeformed state, in any
    orientation; K_M is symmetric PSD with exactly 6 (rigid) zero eigenvalues."""
    rng = np.random.default_rng(6)
    for _ in range(5):
        Q = expm(rng.normal(size=3) * 2)
        xa = rng.normal(size=3); xb = xa + Q[:, 0] * SEC["l0"]
        K = beam.material_tangent(xa, Q, xb, Q, SEC)
        Kl = beam.linear_beam_stiffness(SEC, Q[:, 0], Q[:, 1])
        assert np.abs(K - Kl).max() <= 1e-13 * np.abs(Kl).max()
    xa, Ta, xb, Tb = _random_element(rng, 0.2)
    K = beam.material_tangent(xa, Ta, xb, Tb, SEC)
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-9 * ev.max()
    assert (np.abs(ev) <= 1e-9 * ev.max()).sum() == 6
