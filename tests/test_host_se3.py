"""The library's host binary64 pose algebra (used by the optimizer side of the
factor: Exp of the right perturbation, its right Jacobian, the 6x6 solve)."""
import numpy as np
import pytest
import scipy.linalg


@pytest.fixture(scope="module")
def api():
    from paper_2202_00242_gb300 import api, build
    build.build()
    return api


def _twist(xi):
    X = np.zeros((4, 4))
    w, v = xi[:3], xi[3:]
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 1e-3, 0.3, 2.5])
def test_se3_exp_is_matrix_exponential(api, scale):
    rng = np.random.default_rng(int(scale * 1e6) + 1)
    xi = rng.normal(size=6) * scale
    np.testing.assert_allclose(api.se3_exp(xi), scipy.linalg.expm(_twist(xi)), rtol=1e-12,
                               atol=1e-14)


@pytest.mark.parametrize("scale", [1e-7, 1e-4, 5e-4, 2e-3, 0.2, 1.0, 3.0])
def test_right_jacobian_first_order(api, scale):
    """Exp(xi + h e_i) - Exp(xi) Exp(h J e_i) = O(h^2): with h = 1e-6 the residual
    is ~1e-12; a wrong column would leave ~h * |error| ~ 1e-7."""
    rng = np.random.default_rng(7)
    xi = rng.normal(size=6) * scale
    J = api.se3_right_jacobian(xi)
    h = 1e-6
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        lhs = api.se3_exp(xi + e)
        rhs = api.se3_exp(xi) @ api.se3_exp(J @ e)
        assert np.abs(lhs - rhs).max() < 1e-11, (i, np.abs(lhs - rhs).max())
    np.testing.assert_allclose(api.se3_right_jacobian(np.zeros(6)), np.eye(6), atol=1e-15)


def test_solve6_and_pose_mul(api):
    rng = np.random.default_rng(3)
    A = rng.normal(size=(6, 6))
    H = A @ A.T + 0.1 * np.eye(6)
    b = rng.normal(size=6)
    np.testing.assert_allclose(api.solve6(H, b), -np.linalg.solve(H, b), rtol=1e-10)
    lam = 0.5
    np.testing.assert_allclose(api.solve6(H, b, lam),
                               -np.linalg.solve(H + lam * np.diag(np.diag(H)), b), rtol=1e-10)
    from paper_2202_00242_gb300._lib import VGICPError
    with pytest.raises(VGICPError):
        api.solve6(-np.eye(6), b)
    T1 = api.se3_exp(rng.normal(size=6))
    T2 = api.se3_exp(rng.normal(size=6))
    np.testing.assert_allclose(api.pose_mul(T1, T2), T1 @ T2, atol=1e-14)


def _se3_log(T):
    """Twist [omega; v] of a 4x4 rigid transform via the matrix logarithm."""
    X = np.real(scipy.linalg.logm(T))
    return np.array([X[2, 1], X[0, 2], X[1, 0], X[0, 3], X[1, 3], X[2, 3]])


def test_binary_factor_against_finite_differences(api):
    """The 12x12 form over the world-pose perturbations: A (d xi / d [d_i; d_j]) by
    central differences of Log(T^-1 T(d)) with T(d) = (T_j Exp(d_j))^-1 T_i Exp(d_i),
    then H2 = A^T H A and b2 = A^T b."""
    rng = np.random.default_rng(3)
    Ti = api.se3_exp(rng.normal(size=6) * [0.5, 0.5, 0.5, 3, 3, 3])
    Tj = api.se3_exp(rng.normal(size=6) * [0.5, 0.5, 0.5, 3, 3, 3])
    T = np.linalg.inv(Tj) @ Ti
    M = rng.normal(size=(6, 6))
    H = M @ M.T + np.eye(6)
    b = rng.normal(size=6)
    h = 1e-6
    A = np.zeros((6, 12))
    for k in range(12):
        d = np.zeros(12)
        d[k] = h
        Tp = np.linalg.inv(Tj @ api.se3_exp(d[6:])) @ (Ti @ api.se3_exp(d[:6]))
        Tm = np.linalg.inv(Tj @ api.se3_exp(-d[6:])) @ (Ti @ api.se3_exp(-d[:6]))
        A[:, k] = (_se3_log(np.linalg.inv(T) @ Tp) - _se3_log(np.linalg.inv(T) @ Tm)) / (2 * h)
    H2, b2 = api.binary_factor(H, b, T)
    assert np.allclose(H2, A.T @ H @ A, rtol=1e-6, atol=1e-6 * np.abs(H2).max())
    assert np.allclose(b2, A.T @ b, rtol=1e-6, atol=1e-6 * np.abs(b2).max())
    assert np.allclose(H2, H2.T)
