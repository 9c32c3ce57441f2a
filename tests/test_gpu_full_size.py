"""Parity at full workload sizes, on sampled factors the oracle computes one by
one, plus properties checked on every factor.

  * global map: 500 submaps (30k-80k points), 5,000 pairs, res 1.0 m, in the
    launch configuration the benchmark times (voxel maps as sources, autotuned
    plan replayed as a CUDA graph);
  * large map: 2,000 submaps x 100k points, 40,000 pairs, res 0.5 m,
    27-neighbour correspondences, admitted in batches under a 24 GB budget.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2202_00242_gb300 import api, synth

from test_gpu_parity import check_factor, cu, dev  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _sampled(n, k, seed):
    return np.random.default_rng(seed).choice(n, k, replace=False)


def test_global_map_full_size_plan(dev):  # noqa: F811
    import bench
    w = bench.make_workload(bench.parse_args([]), 0)
    off = w.clouds.offsets
    assert len(off) == 501 and w.pairs.shape[0] == 5000
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, off, w.resolution)
    maps[0].status()
    plan = api.Plan(maps, maps, w.pairs)
    plan.autotune(w.poses)
    res = plan.execute(w.poses)
    torch.cuda.synchronize()
    out, inl = res.out.cpu().numpy(), res.inliers.cpu().numpy()
    H = out[:, :36].reshape(-1, 6, 6)
    assert np.isfinite(out).all() and (inl > 0).all()
    assert np.array_equal(H, H.transpose(0, 2, 1))
    assert (np.linalg.eigvalsh(H).min(axis=1) >= -1e-6 * np.abs(H).max(axis=(1, 2))).all()
    for p in _sampled(len(w.pairs), 6, 1):
        j, i = w.pairs[p]
        tp, tc = w.clouds.cloud(j)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(oracle.build_voxelmap(tp, tc, w.resolution), sp, sc, w.poses[p],
                               nthreads=0)
        check_factor(res.out[p], inl[p], ref, f"pair {p}")
    plan.close()


def test_large_map_full_size_admission(dev):  # noqa: F811
    t0 = time.time()
    w = synth.with_surface_covariances(synth.config_large_map())
    off = w.clouds.offsets
    assert len(off) == 2001 and w.pairs.shape[0] == 40000
    assert (np.diff(off) == 100000).all()
    gen_s = time.time() - t0
    out, inl, nb = api.linearize_admitted(w.clouds.points, w.clouds.covs, off, w.pairs, w.poses,
                                          w.resolution, budget=24 << 30, neighbours=27)
    print(f"large map: generated in {gen_s:.0f} s, {nb} admission batches, "
          f"{time.time() - t0 - gen_s:.1f} s on the device path")
    assert nb >= 2
    H = out[:, :36].reshape(-1, 6, 6)
    assert np.isfinite(out).all() and (inl > 0).all()
    assert np.array_equal(H, H.transpose(0, 2, 1))
    for p in _sampled(len(w.pairs), 6, 2):
        j, i = w.pairs[p]
        tp, tc = w.clouds.cloud(j)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(oracle.build_voxelmap(tp, tc, w.resolution), sp, sc, w.poses[p],
                               neighbours=27, nthreads=0)
        check_factor(torch.from_numpy(out[p]), inl[p], ref, f"pair {p}")
