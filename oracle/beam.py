"""Corotational two-node 6-DOF beam element (Sec. II.B; Eq. 20 and the corotational
reading of its tangent).  Plain FP64 numpy; every product is an explicit matrix.

Reading of the paper (it names the corotational method but prints no element):
  * nodes carry a position x and a rotation T (columns = section triad, T = E0 at rest);
  * the rigid element frame R_r = [e1 e2 e3] has e1 along the chord and e2, e3 fixed by
    the mean of the two nodal second axes q = (T_a[:,1] + T_b[:,1]) / 2;
  * the local deformations are d_l = [l - l0, theta_a(3), theta_b(3)], theta = log(R_r^T T);
  * "the local stiffness matrix is constant": linear Euler-Bernoulli energy
    U = 1/2 d_l^T K_l d_l with EA/l0, GJ/l0 and EI/l0 [[4, 2], [2, 4]] per bending plane;
  * F = dU/dd with d = (dx_a, dw_a, dx_b, dw_b) spatial spins, i.e. F = B^T K_l d_l with
    B = dd_l/dd; the material tangent is K_M = B^T K_l B (symmetric, positive semi-definite,
    which is the property the QP of Eq. 23 needs); the consistent tangent K_T = dF/dd is
    obtained by complex-step differentiation of F.
"""
import math

import numpy as np

from .rotation import expm, logm, skew, tsinv


def section_constants(robot, youngs_modulus=None):
    """Hollow circular section: A = pi (ro^2 - ri^2), I = pi (ro^4 - ri^4)/4, J = 2 I,
    G = E / (2 (1 + nu)).  Returns EA, EI, GJ and the element length l0 = L / M (Sec. II.B).
    E is the robot's modulus unless youngs_modulus is given."""
    E = robot.youngs_modulus if youngs_modulus is None else float(youngs_modulus)
    ro, ri = robot.outer_radius, robot.inner_radius
    A = math.pi * (ro ** 2 - ri ** 2)
    I = math.pi * (ro ** 4 - ri ** 4) / 4.0
    J = 2.0 * I
    G = E / (2.0 * (1.0 + robot.poisson_ratio))
    return {"EA": E * A, "EI": E * I, "GJ": G * J, "l0": robot.length / robot.n_elements}


def element_sections(robot):
    """Section constants of every element, base to tip.  The robot of Sec. II.A is not uniform: a
    distal section is much less rigid than the rest, so each element may carry its own Young's
    modulus (robot.element_youngs, one per element; None = the robot's modulus everywhere).  The
    section geometry and Poisson's ratio are the robot's."""
    Es = getattr(robot, "element_youngs", None)
    if Es is None:
        sec = section_constants(robot)
        return [sec] * robot.n_elements
    Es = np.asarray(Es, float)
    assert Es.shape == (robot.n_elements,) and np.all(Es > 0.0)
    return [section_constants(robot, E) for E in Es]


def local_stiffness(sec):
    """7x7 constant local stiffness K_l acting on d_l = [u, ta1, ta2, ta3, tb1, tb2, tb3]."""
    l0 = sec["l0"]
    K = np.zeros((7, 7))
    K[0, 0] = sec["EA"] / l0
    gj = sec["GJ"] / l0
    K[1, 1] = gj; K[4, 4] = gj; K[1, 4] = -gj; K[4, 1] = -gj
    ei = sec["EI"] / l0
    for a, b in ((2, 5), (3, 6)):
        K[a, a] = 4 * ei; K[b, b] = 4 * ei; K[a, b] = 2 * ei; K[b, a] = 2 * ei
    return K


def corotated_frame(xa, Ta, xb, Tb):
    """Chord length l and rigid frame R_r = [e1 e2 e3]."""
    d = xb - xa
    l = np.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    e1 = d / l
    q = 0.5 * (Ta[:, 1] + Tb[:, 1])
    v = np.cross(e1, q)
    e3 = v / np.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    e2 = np.cross(e3, e1)
    return l, np.column_stack([e1, e2, e3])


def local_deformation(xa, Ta, xb, Tb, l0):
    """d_l = [l - l0, log(R_r^T T_a), log(R_r^T T_b)]; l - l0 evaluated as (l^2 - l0^2)/(l + l0)."""
    l, Rr = corotated_frame(xa, Ta, xb, Tb)
    d = xb - xa
    u = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - l0 * l0) / (l + l0)
    tha = logm(Rr.T @ Ta)
    thb = logm(Rr.T @ Tb)
    return np.concatenate([[u], tha, thb]), l, Rr


def strain_energy(xa, Ta, xb, Tb, sec):
    dl, _, _ = local_deformation(xa, Ta, xb, Tb, sec["l0"])
    return 0.5 * dl @ local_stiffness(sec) @ dl


def B_local(xa, Ta, xb, Tb, sec):
    """B = dd_l/dd (7 x 12) with both d_l and the nodal variations in the element frame.

    Spin of the rigid frame, dw_r = G^T d (local components):
      dw_r1 = [ -qb1 (db3 - da3)/l + (wa1 qa2 - wa2 qa1)/2 + (wb1 qb2 - wb2 qb1)/2 ] / q2
      dw_r2 = -(db3 - da3)/l,     dw_r3 = (db2 - da2)/l
    where q, qa, qb are the local components of the mean and nodal second axes.
    dtheta_a = Tsinv(theta_a) (w_a - dw_r), dtheta_b = Tsinv(theta_b) (w_b - dw_r)."""
    dl, l, Rr = local_deformation(xa, Ta, xb, Tb, sec["l0"])
    qa = Rr.T @ Ta[:, 1]
    qb = Rr.T @ Tb[:, 1]
    q = 0.5 * (qa + qb)
    Gt = np.zeros((3, 12), dtype=np.result_type(qa, float))
    Gt[0, 2] = q[0] / (q[1] * l)
    Gt[0, 8] = -q[0] / (q[1] * l)
    Gt[0, 3] = qa[1] / (2 * q[1]); Gt[0, 4] = -qa[0] / (2 * q[1])
    Gt[0, 9] = qb[1] / (2 * q[1]); Gt[0, 10] = -qb[0] / (2 * q[1])
    Gt[1, 2] = 1.0 / l; Gt[1, 8] = -1.0 / l
    Gt[2, 1] = -1.0 / l; Gt[2, 7] = 1.0 / l
    Ea = np.zeros((3, 12)); Ea[:, 3:6] = np.eye(3)
    Eb = np.zeros((3, 12)); Eb[:, 9:12] = np.eye(3)
    B = np.zeros((7, 12), dtype=Gt.dtype)
    B[0, 0] = -1.0; B[0, 6] = 1.0
    B[1:4] = tsinv(dl[1:4]) @ (Ea - Gt)
    B[4:7] = tsinv(dl[4:7]) @ (Eb - Gt)
    return B, dl, Rr


def _to_global(Rr):
    E = np.zeros((12, 12), dtype=Rr.dtype)
    for k in range(4):
        E[3 * k:3 * k + 3, 3 * k:3 * k + 3] = Rr
    return E


def internal_force(xa, Ta, xb, Tb, sec):
    """Global element force vector [F_a, M_a, F_b, M_b] = E B^T K_l d_l (12,)."""
    B, dl, Rr = B_local(xa, Ta, xb, Tb, sec)
    return _to_global(Rr) @ (B.T @ (local_stiffness(sec) @ dl))


def material_tangent(xa, Ta, xb, Tb, sec):
    """K_M = E B^T K_l B E^T (12 x 12, symmetric PSD)."""
    B, dl, Rr = B_local(xa, Ta, xb, Tb, sec)
    E = _to_global(Rr)
    return E @ (B.T @ local_stiffness(sec) @ B) @ E.T


def consistent_tangent(xa, Ta, xb, Tb, sec, h=1e-30):
    """K_T = dF/dd by complex-step differentiation: column k = Im F(d + i h e_k) / h,
    translations perturbed additively, rotations by the spatial spin exp(i h [e_k]x) T."""
    K = np.zeros((12, 12))
    for k in range(12):
        xa_c = xa.astype(complex); xb_c = xb.astype(complex)
        Ta_c = Ta.astype(complex); Tb_c = Tb.astype(complex)
        e = np.zeros(3, dtype=complex); e[k % 3] = 1j * h
        blk = k // 3
        if blk == 0:
            xa_c = xa_c + e
        elif blk == 1:
            Ta_c = expm(e) @ Ta_c
        elif blk == 2:
            xb_c = xb_c + e
        else:
            Tb_c = expm(e) @ Tb_c
        K[:, k] = np.imag(internal_force(xa_c, Ta_c, xb_c, Tb_c, sec)) / h
    return K


def linear_beam_stiffness(sec, axis, up):
    """Textbook 12 x 12 linear Euler-Bernoulli stiffness of a straight element along unit
    ``axis`` with section axis ``up`` (used to pin K_M at the undeformed state)."""
    l0, EA, EI, GJ = sec["l0"], sec["EA"], sec["EI"], sec["GJ"]
    k = np.zeros((12, 12))
    k[0, 0] = k[6, 6] = EA / l0; k[0, 6] = k[6, 0] = -EA / l0
    k[3, 3] = k[9, 9] = GJ / l0; k[3, 9] = k[9, 3] = -GJ / l0
    # bending in the local x-y plane (v, theta_z): dofs 1, 5, 7, 11
    idx = [1, 5, 7, 11]
    kb = EI / l0 ** 3 * np.array([[12, 6 * l0, -12, 6 * l0], [6 * l0, 4 * l0 ** 2, -6 * l0, 2 * l0 ** 2],
                                  [-12, -6 * l0, 12, -6 * l0], [6 * l0, 2 * l0 ** 2, -6 * l0, 4 * l0 ** 2]])
    for i in range(4):
        for j in range(4):
            k[idx[i], idx[j]] = kb[i, j]
    # bending in the local x-z plane (w, theta_y): dofs 2, 4, 8, 10 (sign of theta_y flips)
    idx = [2, 4, 8, 10]
    s = np.array([1, -1, 1, -1])
    for i in range(4):
        for j in range(4):
            k[idx[i], idx[j]] = kb[i, j] * s[i] * s[j]
    e1 = np.asarray(axis, float) / np.linalg.norm(axis)
    e2 = np.asarray(up, float) - np.dot(up, e1) * e1
    e2 /= np.linalg.norm(e2)
    E = _to_global(np.column_stack([e1, e2, np.cross(e1, e2)]))
    return E @ k @ E.T


def spin_update(T, dtheta):
    """Multiplicative rotation update T <- exp([dtheta]x) T (spatial spin)."""
    return expm(dtheta) @ T


__all__ = ["section_constants", "element_sections", "local_stiffness", "corotated_frame", "local_deformation", "strain_energy",
           "B_local", "internal_force", "material_tangent", "consistent_tangent", "linear_beam_stiffness",
           "spin_update", "skew"]
