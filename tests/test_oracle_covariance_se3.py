"""Pins of the oracle's input-side helpers: k-nearest-neighbour search, the
regularised point covariance (arXiv 2202.00242 Sec. III-A/III-C: covariance from
the neighbouring points, GICP-style eigenvalues (1, 1, eps)), the 3x3 inverse,
and the FP64 SE(3) exponential used by the Gauss-Newton driver."""
import numpy as np
import pytest
import scipy.linalg

from oracle import se3


@pytest.mark.parametrize("seed,n,k", [(0, 300, 10), (1, 500, 10), (2, 64, 5), (3, 7, 10)])
def test_knn_grid_equals_bruteforce(oracle_lib, seed, n, k):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(n, 3)).astype(np.float32) * np.array([5, 5, 0.2], np.float32)
    a = oracle_lib.knn_bruteforce(p, k)
    b = oracle_lib.knn_grid(p, k)
    np.testing.assert_array_equal(a, b)
    if n >= k:
        assert (a[:, 0] == np.arange(n)).all()  # self first (distance 0, ties by index)


def test_knn_ties_break_by_lower_index(oracle_lib):
    # duplicated points: equal distances must be ordered by index on both paths
    base = np.random.default_rng(4).normal(size=(50, 3)).astype(np.float32)
    p = np.concatenate([base, base, base])
    a = oracle_lib.knn_bruteforce(p, 10)
    b = oracle_lib.knn_grid(p, 10, cell=0.7)
    np.testing.assert_array_equal(a, b)
    # point i's three copies come first, lowest index first
    assert a[0, :3].tolist() == [0, 50, 100]
    assert a[50, :3].tolist() == [0, 50, 100]


def test_jacobi_eigen_matches_library(oracle_lib):
    rng = np.random.default_rng(5)
    for _ in range(50):
        A = rng.normal(size=(3, 3))
        A = A @ A.T
        w, V = oracle_lib.jacobi_eigen3(A)
        np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(A), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(V @ np.diag(w) @ V.T, A, atol=1e-12 * np.abs(A).max())
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-13)


def test_mat3_inverse_matches_library(oracle_lib):
    rng = np.random.default_rng(6)
    for _ in range(50):
        A = rng.normal(size=(3, 3))
        np.testing.assert_allclose(oracle_lib.mat3_inverse(A), np.linalg.inv(A), rtol=1e-10,
                                   atol=1e-12 * np.abs(np.linalg.inv(A)).max())
    with pytest.raises(ZeroDivisionError):
        oracle_lib.mat3_inverse(np.zeros((3, 3)))


def test_regularized_covariance_structure(oracle_lib):
    """Points on a tilted plane: each covariance has eigenvalues (eps, 1, 1) and its
    eps-eigenvector is the plane normal; the result does not depend on the 1/k
    normalisation or centroid, only on the eigenvectors."""
    rng = np.random.default_rng(7)
    nrm = np.array([0.3, -0.4, 0.866])
    nrm /= np.linalg.norm(nrm)
    e1 = np.cross(nrm, [1.0, 0, 0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(nrm, e1)
    uv = rng.uniform(-3, 3, size=(400, 2))
    p = (uv[:, :1] * e1 + uv[:, 1:] * e2 + rng.normal(scale=1e-4, size=(400, 1)) * nrm)
    p = p.astype(np.float32)
    C = oracle_lib.knn_covariances(p, k=10, eps=1e-3)
    for c in C:
        S = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        w, V = np.linalg.eigh(S)
        np.testing.assert_allclose(w, [1e-3, 1.0, 1.0], atol=1e-12)
        assert abs(abs(V[:, 0] @ nrm) - 1.0) < 1e-4
    # scaling the neighbourhood does not change the regularised covariance
    nbr = oracle_lib.knn_bruteforce(p, 10)
    C2 = oracle_lib.regularized_covariances((p * 3.0).astype(np.float32), nbr, 1e-3)
    np.testing.assert_allclose(C2, oracle_lib.regularized_covariances(p, nbr, 1e-3), atol=1e-6)


def test_se3_exp_is_matrix_exponential():
    rng = np.random.default_rng(8)
    for scale in (1e-9, 1e-3, 0.5, 2.0):
        xi = rng.normal(size=6) * scale
        X = np.zeros((4, 4))
        X[:3, :3] = se3.hat(xi[:3])
        X[:3, 3] = xi[3:]
        np.testing.assert_allclose(se3.se3_exp(xi), scipy.linalg.expm(X), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(se3.so3_log(se3.so3_exp(xi[:3])), xi[:3], rtol=1e-8,
                                   atol=1e-12)


def test_adjoint_identity():
    rng = np.random.default_rng(9)
    T = se3.se3_exp(rng.normal(size=6))
    xi = rng.normal(size=6) * 0.3
    np.testing.assert_allclose(T @ se3.se3_exp(xi) @ se3.inverse(T), se3.se3_exp(se3.adjoint(T) @ xi),
                               atol=1e-12)
