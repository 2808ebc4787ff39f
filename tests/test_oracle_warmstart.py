"""Pins of the warm start between insertion steps (the follow-the-path rule): material point s
takes the old pose of material point s + (delta - delta_old): linear between the old nodes for the
position, the geodesic between the old nodal rotations, and straight along the old tip's axis
beyond the old tip (along node 0's axis before the base)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import solver
from oracle.rotation import expm, logm

L, M = 0.12, 20
l0 = L / M


def _model():
    return solver.Model(wl.robot_desc(L, M), wl.free_space_lumen())


def _arc(kappa):
    """Nodes on a planar arc of curvature kappa (the polygon of chords l0 turning by kappa l0)."""
    phi = kappa * l0
    x = np.zeros((M + 1, 3))
    R = np.zeros((M + 1, 3, 3))
    for i in range(M + 1):
        R[i] = expm(np.array([0.0, 0.0, i * phi]))
        if i:
            ang = (i - 0.5) * phi
            x[i] = x[i - 1] + l0 * np.array([math.cos(ang), math.sin(ang), 0.0])
    return x, R


def test_straight_rod_moves_along_its_axis():
    m = _model()
    x0, R0 = m.straight(0.05)
    x1, R1 = m.follow_path(x0, R0, 0.05, 0.08)
    xs, Rs = m.straight(0.08)
    assert np.abs(x1 - xs).max() <= 1e-15 and np.abs(R1 - Rs).max() <= 1e-15


def test_whole_element_shift_takes_the_next_nodes_pose():
    m = _model()
    x0, R0 = _arc(5.0)
    x1, R1 = m.follow_path(x0, R0, 0.05, 0.05 + 3 * l0)
    for i in range(M - 3):
        assert np.allclose(x1[i], x0[i + 3], atol=1e-15) and np.allclose(R1[i], R0[i + 3], atol=1e-14)


def test_half_element_shift_interpolates_linearly_and_geodesically():
    m = _model()
    x0, R0 = _arc(5.0)
    x1, R1 = m.follow_path(x0, R0, 0.05, 0.05 + 0.5 * l0)
    for i in range(M - 1):
        assert np.allclose(x1[i], 0.5 * (x0[i] + x0[i + 1]), atol=1e-15)
        mid = R0[i] @ expm(0.5 * logm(R0[i].T @ R0[i + 1]))
        assert np.allclose(R1[i], mid, atol=1e-14)
        assert np.allclose(logm(R1[i]), [0.0, 0.0, (i + 0.5) * 5.0 * l0], atol=1e-13)


def test_beyond_the_tip_and_before_the_base():
    m = _model()
    x0, R0 = _arc(5.0)
    d = 2.5 * l0
    x1, R1 = m.follow_path(x0, R0, 0.05, 0.05 + d)
    for i in range(M + 1):
        s = i * l0 + d
        if s >= L:                                   # straight along the old tip axis
            assert np.allclose(x1[i], x0[M] + (s - L) * R0[M][:, 0], atol=1e-15)
            assert np.allclose(R1[i], R0[M], atol=1e-15)
    x2, R2 = m.follow_path(x0, R0, 0.05, 0.05 - d)  # retraction: before node 0, along its axis
    for i in range(3):
        s = i * l0 - d
        assert s <= 0.0
        assert np.allclose(x2[i], x0[0] + s * R0[0][:, 0], atol=1e-15) and np.allclose(R2[i], R0[0], atol=1e-15)
