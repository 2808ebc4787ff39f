"""SO(3) helpers written with complex-safe operations (no abs/conj), so that the
element code built on them can be differentiated by the complex-step method.

Node rotations are 3x3 matrices whose columns are the cross-section triad in
global coordinates.  Variations are *spatial spins*: dR = [dw]x R.
"""
import numpy as np


def skew(v):
    """[v]x such that [v]x a = v x a."""
    return np.array([[0.0 * v[0], -v[2], v[1]],
                     [v[2], 0.0 * v[0], -v[0]],
                     [-v[1], v[0], 0.0 * v[0]]])


def vee(S):
    """Inverse of skew for the antisymmetric part of S."""
    return 0.5 * np.array([S[2, 1] - S[1, 2], S[0, 2] - S[2, 0], S[1, 0] - S[0, 1]])


def _sqrt_dot(v):
    return np.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])


def expm(theta):
    """Rodrigues: exp([theta]x) = I + sin t / t [theta]x + (1 - cos t)/t^2 [theta]x^2."""
    theta = np.asarray(theta)
    t = _sqrt_dot(theta)
    S = skew(theta)
    if abs(t) < 1e-4:
        t2 = t * t
        a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0
        b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0
    else:
        a = np.sin(t) / t
        b = (1.0 - np.cos(t)) / (t * t)
    return np.eye(3) + a * S + b * (S @ S)


def logm(R):
    """Rotation vector theta with exp([theta]x) = R, for rotation angles below pi.

    t = arccos((tr R - 1)/2) and theta = t / (2 sin t) * vee(R - R^T)."""
    c = 0.5 * (R[0, 0] + R[1, 1] + R[2, 2] - 1.0)
    w = vee(R - R.T)                # = 2 sin t * axis
    s2 = 0.25 * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2])   # sin^2 t
    if abs(s2) < 1e-10:
        # t small: t/(2 sin t) = 1/2 + t^2/12 + 7 t^4/720 with t^2 ~ s2 + s2^2/3
        t2 = s2 + s2 * s2 / 3.0
        f = 0.5 + t2 / 12.0 + 7.0 * t2 * t2 / 720.0
    else:
        t = np.arccos(c)
        f = t / (2.0 * np.sin(t))
    return f * w


def tsinv(theta):
    """Inverse of the spatial tangent map of exp: if R = exp([theta]x) and dR = [dw]x R then
    dtheta = Tsinv(theta) dw with Tsinv = I - [theta]x/2 + eta [theta]x^2,
    eta = (1 - (t/2) cot(t/2)) / t^2."""
    theta = np.asarray(theta)
    t2 = theta[0] * theta[0] + theta[1] * theta[1] + theta[2] * theta[2]
    if abs(t2) < 1e-6:
        eta = 1.0 / 12.0 + t2 / 720.0 + t2 * t2 / 30240.0
    else:
        t = np.sqrt(t2)
        eta = (1.0 - 0.5 * t / np.tan(0.5 * t)) / t2
    S = skew(theta)
    return np.eye(3) - 0.5 * S + eta * (S @ S)


def to_quat(R):
    """Unit quaternion (w, x, y, z), w >= 0, of a real rotation matrix (Shepperd's branch choice)."""
    R = np.asarray(R, dtype=np.float64)
    tr = np.trace(R)
    cand = [tr, R[0, 0], R[1, 1], R[2, 2]]
    k = int(np.argmax(cand))
    if k == 0:
        w = 0.5 * np.sqrt(1.0 + tr)
        q = np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])
    elif k == 1:
        x = 0.5 * np.sqrt(1.0 + 2 * R[0, 0] - tr)
        q = np.array([(R[2, 1] - R[1, 2]) / (4 * x), x, (R[0, 1] + R[1, 0]) / (4 * x), (R[0, 2] + R[2, 0]) / (4 * x)])
    elif k == 2:
        y = 0.5 * np.sqrt(1.0 + 2 * R[1, 1] - tr)
        q = np.array([(R[0, 2] - R[2, 0]) / (4 * y), (R[0, 1] + R[1, 0]) / (4 * y), y, (R[1, 2] + R[2, 1]) / (4 * y)])
    else:
        z = 0.5 * np.sqrt(1.0 + 2 * R[2, 2] - tr)
        q = np.array([(R[1, 0] - R[0, 1]) / (4 * z), (R[0, 2] + R[2, 0]) / (4 * z), (R[1, 2] + R[2, 1]) / (4 * z), z])
    if q[0] < 0:
        q = -q
    return q / np.linalg.norm(q)


def from_quat(q):
    """Rotation matrix of the unit quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
