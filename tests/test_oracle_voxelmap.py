"""Pins of the oracle's voxel key and voxel map (arXiv 2202.00242 Sec. III-A: the
target cloud is discretised into voxels, each holding the aggregate of its points'
means and covariances).  Brute force on tiny clouds, hand-checked key values."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def test_voxel_key_floor_semantics(oracle_lib):
    r = 0.5
    xs = np.array([[0.0, 0.49999997, 0.5],
                   [-1e-7, -0.5, -0.50000006],
                   [1.0, 3.25, -3.25]], dtype=np.float32)
    k = oracle_lib.voxel_keys(xs, r)
    # floor, not truncation: negative coordinates go down; a point on a face goes
    # to the voxel above it.
    assert k.tolist() == [[0, 0, 1], [-1, -1, -2], [2, 6, -7]]


def test_voxel_key_matches_python_floor(oracle_lib):
    rng = np.random.default_rng(0)
    for r in (0.25, 0.5, 1.0, 0.3):
        p = (rng.normal(size=(500, 3)) * 20).astype(np.float32)
        k = oracle_lib.voxel_keys(p, r)
        ref = [[math.floor(float(v) / r) for v in row] for row in p]
        assert k.tolist() == ref


def _clustered(rng, n, r):
    """points clustered so that most voxels receive several points"""
    centers = rng.uniform(-3, 3, size=(12, 3))
    idx = rng.integers(0, 12, size=n)
    return (centers[idx] + rng.normal(scale=0.3 * r, size=(n, 3))).astype(np.float32)


@pytest.mark.parametrize("seed,n,r", [(1, 200, 0.5), (2, 150, 1.0), (3, 60, 0.25), (4, 1, 0.5)])
def test_build_matches_bruteforce_grouping(oracle_lib, seed, n, r):
    rng = np.random.default_rng(seed)
    p = _clustered(rng, n, r)
    c = rng.normal(size=(n, 6)).astype(np.float32)
    vm = oracle_lib.build_voxelmap(p, c, r)
    # brute force: scan points in order; a voxel is created at its first point
    order, groups = [], {}
    for i in range(n):
        key = tuple(math.floor(float(v) / r) for v in p[i])
        if key not in groups:
            groups[key] = []
            order.append(key)
        groups[key].append(i)
    assert vm.num_voxels == len(order)
    assert [tuple(k) for k in vm.keys.tolist()] == order
    for v, key in enumerate(order):
        idx = groups[key]
        assert vm.counts[v] == len(idx)
        mu = np.mean(p[idx].astype(np.float64), axis=0)
        cv = np.mean(c[idx].astype(np.float64), axis=0)
        np.testing.assert_allclose(vm.means[v], mu, rtol=1e-15, atol=1e-15)
        np.testing.assert_allclose(vm.covs[v], cv, rtol=1e-14, atol=1e-15)


def test_build_counts_sum_and_empty(oracle_lib):
    rng = np.random.default_rng(5)
    p = _clustered(rng, 300, 0.5)
    c = np.ones((300, 6), dtype=np.float32)
    vm = oracle_lib.build_voxelmap(p, c, 0.5)
    assert vm.counts.sum() == 300
    assert len({tuple(k) for k in vm.keys.tolist()}) == vm.num_voxels
    empty = oracle_lib.build_voxelmap(np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32), 0.5)
    assert empty.num_voxels == 0


def test_downsample_pins(oracle_lib):
    """Voxel-grid downsampling (Sec. III-C): without a time split it is the voxel
    map's means and counts; with it, brute-force grouping by (voxel, |t - t_first|
    > split) in first-appearance order, binary64 means rounded to float32."""
    import oracle
    rng = np.random.default_rng(4)
    pts = (rng.random((400, 3)) * 3.0 - 1.5).astype(np.float32)
    t = rng.random(400).astype(np.float32) * 0.1
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (400, 1))
    dp, dt, dc = oracle.downsample(pts, None, 0.5)
    vm = oracle.build_voxelmap(pts, covs, 0.5)
    assert dt is None
    assert np.array_equal(dc, vm.counts)
    assert np.array_equal(dp, vm.means.astype(np.float32))
    split = 0.01
    dp, dt, dc = oracle.downsample(pts, t, 0.5, split)
    groups, order = {}, []
    first_t = {}
    for i in range(400):
        k = tuple(int(v) for v in np.floor(pts[i].astype(np.float64) / 0.5))
        first_t.setdefault(k, float(t[i]))
        g = (k, abs(float(t[i]) - first_t[k]) > split)
        if g not in groups:
            groups[g] = []
            order.append(g)
        groups[g].append(i)
    assert len(order) == len(dc) > vm.num_voxels
    for v, g in enumerate(order):
        idx = groups[g]
        assert dc[v] == len(idx)
        s = np.zeros(4)
        for i in idx:  # binary64 sums in index order
            s[:3] += pts[i].astype(np.float64)
            s[3] += float(t[i])
        assert np.array_equal(dp[v], (s[:3] / len(idx)).astype(np.float32))
        assert dt[v] == np.float32(s[3] / len(idx))
