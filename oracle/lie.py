"""Rigid-motion helpers (oracle, FP64).

Sec. 4.3 parameterises each camera transform T_i (camera -> world, R_i p + t_i)
by the matrix exponential of skew-symmetric generators: 3 rotation and 3
translation unknowns per frame.  Reading used throughout: the unknown of frame i
is a tangent 6-vector (dw, dt) at the current estimate, applied as
R <- Exp(dw) R, t <- t + dt (a rotation about world axes, left-multiplied).
"""
import numpy as np


def skew(v):
    """[v]_x such that skew(v) @ u == cross(v, u)."""
    x, y, z = v
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def exp_so3(w):
    """Exp of the skew generator of w (Rodrigues' formula), FP64."""
    w = np.asarray(w, dtype=np.float64)
    th = float(np.sqrt(w @ w))
    K = skew(w)
    if th < 1e-8:
        # series: I + K + K^2/2 (+ O(th^3)); exact to rounding for th < 1e-8
        return np.eye(3) + K + 0.5 * (K @ K)
    return np.eye(3) + (np.sin(th) / th) * K + ((1.0 - np.cos(th)) / (th * th)) * (K @ K)


def apply_update(R, t, delta):
    """Pose update of Sec. 4.4 (X^k = X^{k-1} + dX) under the left-perturbation reading."""
    return exp_so3(delta[:3]) @ R, t + delta[3:6]


def rot_angle(R):
    c = (np.trace(R) - 1.0) / 2.0
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


def pose_error(Ta, Tb):
    """(rotation angle [rad], translation distance) between two 4x4 poses."""
    return rot_angle(Ta[:3, :3].T @ Tb[:3, :3]), float(np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]))


def to44(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T
