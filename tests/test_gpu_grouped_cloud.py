"""The voxel-grouped cloud and dense voxels against the FP64 oracle (Sec. III-A
voxel map; the grouped cloud is what a map-as-source factor reads, Sec. III-F).

  * voxel keys, counts, means and covariances (first-appearance order) are
    bit-exact with the oracle's, also for voxels holding thousands of points
    (lists longer than the build's shared-memory stage are sorted in place);
  * the grouped cloud is a permutation of the input rows, each voxel's points
    one contiguous run, in ascending input index;
  * factors match the oracle to the parity bar, also across rebuilds that
    alternate dense and plain clouds.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_00242_gb300 import api

import cases

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_00242_gb300 import build
    build.build()
    return torch.device("cuda:0")


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def iso_covs(n, s=0.02):
    return np.tile(np.array([s, 0, 0, s, 0, s], np.float32), (n, 1))


def check_export(vm, pts, covs, r):
    ex = vm.export()
    ref = oracle.build_voxelmap(pts, covs, r)
    assert np.array_equal(ex["keys"], ref.keys)
    assert np.array_equal(ex["counts"], ref.counts)
    assert np.array_equal(ex["means"], ref.means.astype(np.float32))
    assert np.array_equal(ex["covs"], ref.covs.astype(np.float32))
    return ref


def check_grouped(vm, pts, covs, r):
    """The grouped cloud holds every input row once; each voxel's rows are one
    contiguous run, in ascending input index."""
    g, gc = vm.grouped_cloud()
    rows = np.concatenate([g.cpu().numpy(), gc.cpu().numpy()], 1)
    inp = np.concatenate([pts, covs], 1)
    where = {inp[i].tobytes(): i for i in range(inp.shape[0])}
    assert len(where) == inp.shape[0], "test clouds must have distinct rows"
    idx = np.array([where[row.tobytes()] for row in rows])
    assert np.array_equal(np.sort(idx), np.arange(inp.shape[0]))
    keys = np.floor(g.cpu().numpy().astype(np.float64) / r).astype(np.int64)
    change = np.any(keys[1:] != keys[:-1], axis=1)
    starts = np.concatenate([[0], np.nonzero(change)[0] + 1])
    run_keys = keys[starts]
    assert np.unique(run_keys, axis=0).shape[0] == run_keys.shape[0], "a voxel split in two runs"
    same = ~change
    assert np.all(idx[1:][same] > idx[:-1][same]), "a voxel's points out of index order"


def check_factor(vm, ref_map, src, scov, T, what):
    lin = api.linearize(vm, cu(src), cu(scov), T)
    ref = oracle.linearize(ref_map, src, scov, T)
    H, b, err = (x.numpy() for x in api.unpack(lin.out.cpu().double()))
    assert int(lin.inliers) == ref.inliers, what
    assert cases.rel_fro(H, ref.H) <= TOL, what
    assert cases.b_rel(b, ref.b) <= TOL, what
    assert abs(float(err) - ref.err) <= TOL * abs(ref.err), what


def off_pose(T):
    """The planted pose moved by a few centimetres (b is not near zero there)."""
    T = np.array(T, np.float64, copy=True)
    T[:3, 3] += [0.05, -0.03, 0.02]
    return T


def dense_blob(rng, n, lo=0.1, hi=0.4):
    """n points inside one voxel at r = 0.5."""
    return (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)


@pytest.mark.parametrize("r", [0.5, 0.25])
def test_room_grouped_cloud(dev, r):
    tp, tc, sp, sc, T, _ = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    vm.status()
    ref = check_export(vm, tp, tc, r)
    check_grouped(vm, tp, tc, r)
    check_factor(vm, ref, sp, sc, off_pose(T), f"room r={r}")


@pytest.mark.parametrize("n_dense", [1200, 4000])
def test_dense_voxel(dev, n_dense):
    """n_dense points in one voxel among a room's: one long list (4,000 exceeds the
    3,072 indices the build stages in shared memory)."""
    rng = np.random.default_rng(n_dense)
    tp, tc, sp, sc, T, _ = cases.room(n_target=3000, n_source=2000)
    pts = np.concatenate([tp[:1500], dense_blob(rng, n_dense), tp[1500:]])
    covs = np.concatenate([tc[:1500], iso_covs(n_dense), tc[1500:]])
    r = 0.5
    vm = api.VoxelMap.build(cu(pts), cu(covs), r)
    vm.status()
    ref = check_export(vm, pts, covs, r)
    check_grouped(vm, pts, covs, r)
    check_factor(vm, ref, sp, sc, off_pose(T), f"dense voxel {n_dense}")


def test_rebuilds_dense_and_plain(dev):
    """A batch of three maps rebuilt alternately with and without a dense voxel in
    its middle map: every rebuild gives the oracle's maps, grouped clouds and
    factors."""
    rng = np.random.default_rng(5)
    r = 0.5
    tp, tc, sp, sc, T, _ = cases.room(n_target=6000, n_source=3000)
    n = 6000
    plain = [tp[:n], (tp[:n] + np.float32(0.37)), (tp[:n] - np.float32(0.21))]
    dense_mid = np.concatenate([dense_blob(rng, 2600), tp[: n - 2600]])
    covs = np.concatenate([tc[:n]] * 3)
    off = np.array([0, n, 2 * n, 3 * n], np.int64)
    clouds = {
        "plain": np.concatenate(plain),
        "dense": np.concatenate([plain[0], dense_mid, plain[2]]),
    }
    maps = api.build_voxelmaps(cu(clouds["plain"]), cu(covs), off, r)
    maps[0].status()
    for kind in ("dense", "plain", "dense", "plain"):
        pts = clouds[kind]
        api.rebuild_voxelmaps(maps, cu(pts), cu(covs))
        maps[0].status()
        for m in range(3):
            a, b = off[m], off[m + 1]
            ref = check_export(maps[m], pts[a:b], covs[a:b], r)
            check_factor(maps[m], ref, sp, sc, off_pose(T), f"{kind} map {m}")
        check_grouped(maps[1], pts[off[1]:off[2]], covs[off[1]:off[2]], r)
