"""Large-map stress workload, scaled in the number of submaps: 100k-point
submaps, res 0.5 m, 27-neighbour correspondences (each transformed source
point against the 3x3x3 voxel block around it), batched by device-memory
admission.

The factor set is linearized twice, once under a budget that forces several
admission batches and once in a single batch; the two must agree bit for bit
(each pair's result depends only on its own map and source).  Sampled pairs
are checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_00242_gb300 import api, synth

from test_gpu_parity import check_factor, dev  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

N_SUBMAPS = 48


@pytest.fixture(scope="module")
def large():
    w = synth.with_surface_covariances(synth.config_large_map(seed=11, n_submaps=N_SUBMAPS,
                                                              neighbours=8))
    pts = np.ascontiguousarray(w.clouds.points, dtype=np.float32)
    covs = np.ascontiguousarray(w.clouds.covs, dtype=np.float32)
    return w, pts, covs


def test_admission_batches_match_single_batch_and_oracle(dev, large):  # noqa: F811
    w, pts, covs = large
    off = np.asarray(w.clouds.offsets, np.int64)
    per_map = api.voxelmap_bytes(100000) + 36 * 100000
    out_b, inl_b, nb = api.linearize_admitted(pts, covs, off, w.pairs, w.poses, w.resolution,
                                              budget=12 * per_map, neighbours=27)
    assert nb >= 3
    out_1, inl_1, n1 = api.linearize_admitted(pts, covs, off, w.pairs, w.poses, w.resolution,
                                              budget=1 << 40, neighbours=27)
    assert n1 == 1
    assert np.array_equal(out_b, out_1) and np.array_equal(inl_b, inl_1)
    assert (inl_1 > 0).all()
    rng = np.random.default_rng(0)
    for p in rng.choice(len(w.pairs), 4, replace=False):
        j, i = w.pairs[p]
        ref = oracle.linearize(oracle.build_voxelmap(pts[off[j]:off[j + 1]],
                                                     covs[off[j]:off[j + 1]], w.resolution),
                               pts[off[i]:off[i + 1]], covs[off[i]:off[i + 1]], w.poses[p],
                               neighbours=27, nthreads=0)
        check_factor(torch.from_numpy(out_1[p]), inl_1[p], ref, f"pair {p}")


def test_admission_rejects_budget_below_one_pair(dev, large):  # noqa: F811
    from paper_2202_00242_gb300._lib import VGICPError
    w, pts, covs = large
    with pytest.raises(VGICPError):
        api.linearize_admitted(pts, covs, w.clouds.offsets, w.pairs[:2], w.poses[:2],
                               w.resolution, budget=1000, neighbours=27)
