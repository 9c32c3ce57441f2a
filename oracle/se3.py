"""Binary64 SE(3) helpers and a Gauss-Newton driver for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Convention (the reading of arXiv 2202.00242 Sec. III-A used throughout): the
factor is linearised in the right perturbation T <- T Exp(xi) with
xi = [omega; v]; Exp is the matrix exponential of the twist
[[omega]x, v; 0, 0].  The Gauss-Newton step of err(xi) ~ err + 2 b^T xi +
xi^T H xi is xi = -H^-1 b.
"""
from __future__ import annotations

import numpy as np


def hat(w):
    w = np.asarray(w, dtype=np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w):
    """Rodrigues' formula."""
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    K = hat(w)
    if th < 1e-8:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / th**2 * K @ K


def se3_exp(xi):
    """Exp of xi = [omega; v] as a 4x4 matrix (closed form of the matrix exponential)."""
    xi = np.asarray(xi, dtype=np.float64)
    w, v = xi[:3], xi[3:]
    th = float(np.linalg.norm(w))
    K = hat(w)
    if th < 1e-8:
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        V = (np.eye(3) + (1.0 - np.cos(th)) / th**2 * K
             + (th - np.sin(th)) / th**3 * K @ K)
    T = np.eye(4)
    T[:3, :3] = so3_exp(w)
    T[:3, 3] = V @ v
    return T


def so3_log(R):
    R = np.asarray(R, dtype=np.float64)
    c = np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)
    th = float(np.arccos(c))
    if th < 1e-8:
        return np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2.0
    return th / (2.0 * np.sin(th)) * np.array(
        [R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])


def inverse(T):
    T = np.asarray(T, dtype=np.float64)
    Ti = np.eye(4)
    Ti[:3, :3] = T[:3, :3].T
    Ti[:3, 3] = -T[:3, :3].T @ T[:3, 3]
    return Ti


def adjoint(T):
    """Ad_T for xi = [omega; v]:  T Exp(xi) T^-1 = Exp(Ad_T xi)."""
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[3:, 3:] = R
    A[3:, :3] = hat(t) @ R
    return A


def pose_error(T_est, T_ref):
    """(rotation angle in degrees, translation distance) of T_ref^-1 T_est."""
    E = inverse(T_ref) @ T_est
    return float(np.degrees(np.linalg.norm(so3_log(E[:3, :3])))), float(np.linalg.norm(E[:3, 3]))


def gauss_newton(linearize_fn, T0, max_iters: int = 30, tol: float = 1e-10):
    """Minimise err(T) by xi = -H^-1 b, T <- T Exp(xi) (Cholesky of the 6x6 H).

    ``linearize_fn(T) -> (H, b, err)``.  Returns (T, history) where history lists
    (err, |xi|) per iteration.
    """
    T = np.asarray(T0, dtype=np.float64).copy()
    hist = []
    for _ in range(max_iters):
        H, b, err = linearize_fn(T)
        L = np.linalg.cholesky(H)
        y = np.linalg.solve(L, -b)
        xi = np.linalg.solve(L.T, y)
        T = T @ se3_exp(xi)
        hist.append((float(err), float(np.linalg.norm(xi))))
        if np.linalg.norm(xi) < tol:
            break
    return T, hist
