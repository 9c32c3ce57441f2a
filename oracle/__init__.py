"""FP64 CPU oracle for VGICP matching-cost factor linearization.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow restatement of what the
GPU library computes, written from arXiv 2202.00242 Sec. III-A (Eqs. 2-3, the
voxel map and the re-linearisation into a Hessian factor) and Sec. III-C/III-D
(k-nearest-neighbour point covariances, overlap rate).  Only ``tests/``, the
smoke check and the CPU-baseline leg of the benchmark may import it; the product
path never does, and it shares no code with the CUDA path.

Parity status of each function (what pins it lives in ``tests/test_oracle_*.py``):

* ``build_voxelmap``        pinned: brute-force grouping of tiny clouds.
* ``linearize`` (1 and 27)  pinned: brute-force lookup, closed forms (point-to-point
                            ICP normal equations, R = I block formulas), finite
                            differences of the cost, symmetry/PSD of H, exact
                            invariances, Gauss-Newton recovery of a planted pose.
* ``exact_gradient``        pinned: finite differences of the full cost.
* ``knn_*``                 pinned: brute force vs grid search.
* ``regularized_covariances`` pinned: eigen-structure (1, 1, eps), normal of planes,
                            Jacobi vs a library eigensolver.
* ``se3`` helpers           pinned: against the matrix exponential (scipy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vgicp_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle_vgicp.so")
_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the C++ oracle into ``oracle/liboracle_vgicp.so`` (g++, OpenMP).

    ``-ffp-contract=off`` keeps binary64 rounding identical on x86 and Arm.
    """
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    d = ctypes.c_double
    i32 = ctypes.c_int
    lib.oracle_voxel_keys.argtypes = [P, i64, d, P]
    lib.oracle_voxel_keys.restype = None
    lib.oracle_build_voxelmap.argtypes = [P, P, i64, d, P, P, P, P]
    lib.oracle_build_voxelmap.restype = i64
    lib.oracle_linearize.argtypes = [P, P, P, i64, d, P, P, i64, P, i32, i32, P, P, P, P, P, P,
                                     P, P]
    lib.oracle_linearize.restype = i32
    lib.oracle_cost_fixed.argtypes = [P, P, P, P, i64, P, P, P]
    lib.oracle_cost_fixed.restype = d
    lib.oracle_exact_gradient.argtypes = [P, P, P, P, i64, P, P, P]
    lib.oracle_exact_gradient.restype = None
    lib.oracle_knn_bruteforce.argtypes = [P, i64, i32, P]
    lib.oracle_knn_bruteforce.restype = None
    lib.oracle_knn_grid.argtypes = [P, i64, i32, d, i32, P]
    lib.oracle_knn_grid.restype = None
    lib.oracle_regularized_covariances.argtypes = [P, i64, i32, P, d, P]
    lib.oracle_regularized_covariances.restype = None
    lib.oracle_downsample.argtypes = [P, P, i64, d, d, P, P, P]
    lib.oracle_downsample.restype = i64
    lib.oracle_jacobi_eigen3.argtypes = [P, P, P]
    lib.oracle_jacobi_eigen3.restype = None
    lib.oracle_mat3_inverse.argtypes = [P, P]
    lib.oracle_mat3_inverse.restype = i32
    _lib = lib
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a, cols):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.reshape(-1, cols)


@dataclass
class VoxelMap:
    """Voxel map of a target cloud: voxels in order of first appearance."""
    keys: np.ndarray    # (V, 3) int64
    counts: np.ndarray  # (V,) int64
    means: np.ndarray   # (V, 3) float64
    covs: np.ndarray    # (V, 6) float64, upper triangle xx xy xz yy yz zz
    resolution: float

    @property
    def num_voxels(self) -> int:
        return int(self.keys.shape[0])


def voxel_keys(points, resolution: float) -> np.ndarray:
    """floor(x / r) per axis in binary64, for float32 points (n, 3)."""
    p = _f32(points, 3)
    out = np.empty((p.shape[0], 3), dtype=np.int64)
    _load().oracle_voxel_keys(_ptr(p), p.shape[0], float(resolution), _ptr(out))
    return out


def build_voxelmap(points, covs, resolution: float) -> VoxelMap:
    """Voxelise a target cloud (Sec. III-A): per voxel N, mean of means, mean of covs."""
    p = _f32(points, 3)
    c = _f32(covs, 6)
    n = p.shape[0]
    assert c.shape[0] == n
    keys = np.empty((max(n, 1), 3), dtype=np.int64)
    counts = np.empty(max(n, 1), dtype=np.int64)
    means = np.empty((max(n, 1), 3), dtype=np.float64)
    vcovs = np.empty((max(n, 1), 6), dtype=np.float64)
    V = _load().oracle_build_voxelmap(_ptr(p), _ptr(c), n, float(resolution), _ptr(keys),
                                      _ptr(counts), _ptr(means), _ptr(vcovs))
    return VoxelMap(keys[:V].copy(), counts[:V].copy(), means[:V].copy(), vcovs[:V].copy(),
                    float(resolution))


@dataclass
class Linearization:
    H: np.ndarray        # (6, 6)
    b: np.ndarray        # (6,)
    err: float
    inliers: int
    corr: np.ndarray | None = None   # (n,) voxel index of the point's own voxel or -1
    qkeys: np.ndarray | None = None  # (n, 3) key of T mu
    W: np.ndarray | None = None      # (n, 3, 3) 1-neighbour mode only
    d: np.ndarray | None = None      # (n, 3)


def overlap(vmap: VoxelMap, src_points, T) -> float:
    """Overlap rate (Sec. III-D): the fraction of the source points whose
    transformed position falls in an occupied voxel of the map, i.e. the inlier
    count of the 1-neighbour linearization over n (the covariances do not enter
    the lookup; identity covariances are passed)."""
    p = _f32(src_points, 3)
    if p.shape[0] == 0:
        return 0.0
    eye = np.tile(np.array([1, 0, 0, 1, 0, 1], dtype=np.float32), (p.shape[0], 1))
    return linearize(vmap, p, eye, T, nthreads=0).inliers / p.shape[0]


def linearize(vmap: VoxelMap, src_points, src_covs, T, neighbours: int = 1,
              nthreads: int = 1, debug: bool = False) -> Linearization:
    """Linearise one factor (Eqs. 2-3) at T = T_target_source (4x4, binary64)."""
    p = _f32(src_points, 3)
    c = _f32(src_covs, 6)
    n = p.shape[0]
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(4, 4)
    H = np.zeros(36)
    b = np.zeros(6)
    err = np.zeros(1)
    inl = np.zeros(1, dtype=np.int64)
    corr = qkeys = W = d = None
    if debug:
        corr = np.empty(n, dtype=np.int64)
        qkeys = np.empty((n, 3), dtype=np.int64)
        if neighbours == 1:
            W = np.empty((n, 9))
            d = np.empty((n, 3))
    keys = np.ascontiguousarray(vmap.keys, dtype=np.int64)
    means = np.ascontiguousarray(vmap.means, dtype=np.float64)
    vcovs = np.ascontiguousarray(vmap.covs, dtype=np.float64)
    rc = _load().oracle_linearize(_ptr(keys), _ptr(means), _ptr(vcovs), vmap.num_voxels,
                                  vmap.resolution, _ptr(p), _ptr(c), n, _ptr(T), int(neighbours),
                                  int(nthreads), _ptr(H), _ptr(b), _ptr(err), _ptr(inl),
                                  _ptr(corr), _ptr(qkeys), _ptr(W), _ptr(d))
    if rc != 0:
        raise ValueError("oracle_linearize: bad argument")
    return Linearization(H.reshape(6, 6), b, float(err[0]), int(inl[0]), corr, qkeys,
                         None if W is None else W.reshape(n, 3, 3), d)


def cost_fixed(vmap: VoxelMap, src_points, src_covs, T, corr, W=None) -> float:
    """Eq. 2 at T with fixed correspondences; W fixed too when given ((n,3,3))."""
    p = _f32(src_points, 3)
    c = _f32(src_covs, 6)
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(4, 4)
    corr = np.ascontiguousarray(corr, dtype=np.int64)
    Wf = None if W is None else np.ascontiguousarray(W, dtype=np.float64).reshape(-1, 9)
    return float(_load().oracle_cost_fixed(_ptr(np.ascontiguousarray(vmap.means)),
                                           _ptr(np.ascontiguousarray(vmap.covs)), _ptr(p),
                                           _ptr(c), p.shape[0], _ptr(T), _ptr(corr), _ptr(Wf)))


def exact_gradient(vmap: VoxelMap, src_points, src_covs, T, corr) -> np.ndarray:
    """d(Eq. 2)/d xi at T, correspondences fixed, W varying with the rotation."""
    p = _f32(src_points, 3)
    c = _f32(src_covs, 6)
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(4, 4)
    corr = np.ascontiguousarray(corr, dtype=np.int64)
    g = np.zeros(6)
    _load().oracle_exact_gradient(_ptr(np.ascontiguousarray(vmap.means)),
                                  _ptr(np.ascontiguousarray(vmap.covs)), _ptr(p), _ptr(c),
                                  p.shape[0], _ptr(T), _ptr(corr), _ptr(g))
    return g


def knn_bruteforce(points, k: int) -> np.ndarray:
    p = _f32(points, 3)
    out = np.empty((p.shape[0], k), dtype=np.int64)
    _load().oracle_knn_bruteforce(_ptr(p), p.shape[0], int(k), _ptr(out))
    return out


def knn_grid(points, k: int, cell: float | None = None, nthreads: int = 0) -> np.ndarray:
    p = _f32(points, 3)
    n = p.shape[0]
    if cell is None:
        # a cell holding a few k points on a surface-like cloud
        ext = np.ptp(p.astype(np.float64), axis=0) if n else np.ones(3)
        area = max(ext[0] * ext[1] + ext[1] * ext[2] + ext[0] * ext[2], 1e-12)
        cell = float(max(np.sqrt(area / max(n, 1) * 2.0 * k), 1e-3))
    out = np.empty((n, k), dtype=np.int64)
    _load().oracle_knn_grid(_ptr(p), n, int(k), float(cell), int(nthreads), _ptr(out))
    return out


def regularized_covariances(points, nbr, eps: float = 1e-3) -> np.ndarray:
    p = _f32(points, 3)
    nbr = np.ascontiguousarray(nbr, dtype=np.int64)
    n, k = nbr.shape
    out = np.empty((n, 6))
    _load().oracle_regularized_covariances(_ptr(p), n, int(k), _ptr(nbr), float(eps), _ptr(out))
    return out


def knn_covariances(points, k: int = 10, eps: float = 1e-3, nthreads: int = 0) -> np.ndarray:
    """Point covariances from the k nearest neighbours (self included), eigenvalues
    replaced by (1, 1, eps).  Returns (n, 6) binary64."""
    return regularized_covariances(points, knn_grid(points, k, nthreads=nthreads), eps)


def downsample(points, times, resolution: float, split: float = 0.0):
    """Voxel-grid downsampling with timestamp averaging (Sec. III-C): returns
    (points (V, 3) float32, times (V,) float32 or None, counts (V,) int64), the
    output voxels in order of first appearance."""
    p = _f32(points, 3)
    n = p.shape[0]
    t = None if times is None else np.ascontiguousarray(times, dtype=np.float32).reshape(n)
    op = np.empty((max(n, 1), 3), dtype=np.float32)
    ot = np.empty(max(n, 1), dtype=np.float32) if t is not None else None
    oc = np.empty(max(n, 1), dtype=np.int64)
    V = _load().oracle_downsample(_ptr(p), None if t is None else _ptr(t), n, float(resolution),
                                  float(split), _ptr(op), None if ot is None else _ptr(ot),
                                  _ptr(oc))
    return op[:V].copy(), (None if ot is None else ot[:V].copy()), oc[:V].copy()


def jacobi_eigen3(A):
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(3, 3)
    w = np.empty(3)
    V = np.empty((3, 3))
    _load().oracle_jacobi_eigen3(_ptr(A), _ptr(w), _ptr(V))
    return w, V


def mat3_inverse(A):
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(3, 3)
    out = np.empty((3, 3))
    if _load().oracle_mat3_inverse(_ptr(A), _ptr(out)) != 0:
        raise ZeroDivisionError("singular")
    return out
