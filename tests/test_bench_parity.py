"""Host logic of the benchmark's parity block: sampled factors of the timed set
against the FP64 oracle.  Fed the oracle's own results, every error is zero;
a planted error in one term of b is reported on the plain relative scale."""
import numpy as np

import oracle
from paper_2202_00242_gb300 import synth


def _oracle_results(w, neighbours=1):
    P = w.pairs.shape[0]
    out = np.zeros((P, 43))
    inl = np.zeros(P, np.int64)
    for p, (j, i) in enumerate(w.pairs):
        ref = oracle.linearize(oracle.build_voxelmap(*w.clouds.cloud(j), w.resolution),
                               *w.clouds.cloud(i), w.poses[p], neighbours=neighbours, nthreads=0)
        out[p, :36], out[p, 36:42], out[p, 42], inl[p] = ref.H.ravel(), ref.b, ref.err, ref.inliers
    return out, inl


def test_parity_block_zero_on_oracle_results_and_flags_a_planted_error():
    import bench
    w = synth.with_surface_covariances(synth.outdoor_submaps(
        seed=21, n_submaps=4, n_min=3000, n_max=4000, neighbours=2))
    out, inl = _oracle_results(w)
    res = bench.oracle_parity(w, out, inl, w.poses, n_sample=5)
    assert res["pairs_checked"] == 5 and res["inlier_mismatches"] == 0
    assert res["max_rel_fro_H"] == 0.0 and res["max_rel_b"] == 0.0 and res["max_rel_err"] == 0.0
    assert res["within_tolerance"]
    bad = out.copy()
    bad[:, 36] += 2e-4 * np.linalg.norm(out[:, 36:42], axis=1)
    res = bench.oracle_parity(w, bad, inl, w.poses, n_sample=8)
    assert 1.9e-4 < res["max_rel_b"] < 2.1e-4 and not res["within_tolerance"]
    inl2 = inl.copy()
    inl2[:] += 1
    assert bench.oracle_parity(w, out, inl2, w.poses, n_sample=8)["inlier_mismatches"] == 8


def test_parity_block_gradient_mode():
    import bench
    w = synth.with_surface_covariances(synth.outdoor_submaps(
        seed=22, n_submaps=3, n_min=3000, n_max=4000, neighbours=1))
    out, inl = _oracle_results(w)
    res = bench.oracle_parity(w, out[:, 42], inl, w.poses, n_sample=3, grad=2 * out[:, 36:42])
    assert res["max_rel_grad_vs_2b"] == 0.0 and res["within_tolerance"]
    assert "max_rel_fro_H" not in res


def test_near_face_points():
    import bench
    r = 0.5
    pts = np.array([[0.5 + 1e-7, 0.2, 0.2], [0.25, 0.25, 0.25], [0.2, 1.0 - 5e-6, 0.3]],
                   np.float32)
    assert bench.near_face_points(pts, np.eye(4), r) == 2
