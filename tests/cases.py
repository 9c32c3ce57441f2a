"""Seeded test inputs shared by the GPU parity tests: the scenes come from the
synthetic generator, the point covariances from the oracle's k-NN (k = 10,
eigenvalues (1, 1, 1e-3)) and are then rounded to float32, the precision both
paths consume."""
from __future__ import annotations

import functools

import numpy as np

import oracle
from paper_2202_00242_gb300 import synth


def knn_covs(points) -> np.ndarray:
    return oracle.knn_covariances(points, k=10, eps=1e-3).astype(np.float32)


@functools.lru_cache(maxsize=None)
def room(seed=1, n_target=8192, n_source=8192):
    w = synth.room_pair(seed=seed, n_target=n_target, n_source=n_source)
    tp, _ = w.clouds.cloud(0)
    sp, _ = w.clouds.cloud(1)
    return (np.ascontiguousarray(tp), knn_covs(tp), np.ascontiguousarray(sp), knn_covs(sp),
            w.true_poses[0], w.resolution)


@functools.lru_cache(maxsize=None)
def workload_with_knn_covs(kind: str, **kw):
    w = {"corridor": synth.config_corridor, "outdoor": synth.outdoor_submaps}[kind](**kw)
    covs = np.empty((w.clouds.points.shape[0], 6), np.float32)
    for c in range(len(w.clouds.offsets) - 1):
        a, b = w.clouds.offsets[c], w.clouds.offsets[c + 1]
        covs[a:b] = knn_covs(w.clouds.points[a:b])
    w.clouds.covs = covs
    return w


def rel_fro(a, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - ref) / max(np.linalg.norm(ref), 1e-300))


def b_rel(b, b_ref):
    """Plain relative error of b: |b - b_ref| / |b_ref|."""
    b_ref = np.asarray(b_ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(b, np.float64) - b_ref)
                 / max(np.linalg.norm(b_ref), 1e-300))


def b_error(b, b_ref, err_ref, H_ref):
    """Error of b relative to max(|b_ref|, sqrt(err |H|_F)): b vanishes at the
    optimum, and by Cauchy-Schwarz |b| <= sqrt(err * tr H) bounds its scale."""
    scale = max(np.linalg.norm(b_ref), np.sqrt(max(err_ref, 0.0) * np.linalg.norm(H_ref)), 1e-300)
    return float(np.linalg.norm(np.asarray(b) - np.asarray(b_ref)) / scale)


def near_face_count(src_points, T, r, tol=1e-5):
    q = src_points.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    f = q / r - np.floor(q / r)
    return int((np.minimum(f, 1 - f).min(axis=1) * r < tol).sum())
