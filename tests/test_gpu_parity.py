"""GPU parity: the CUDA library against the FP64 oracle on the same seeded inputs.

Bars (arXiv 2202.00242 Sec. III-A quantities):
  * voxel keys, per-voxel counts and voxel order: bit-exact; voxel means and
    covariances: bit-exact with the binary64 definition rounded to float32;
  * per-point correspondences (voxel index) and keys of T mu: bit-exact; the
    number of points within 1e-5 m of a voxel face is reported;
  * H: relative Frobenius error <= 1e-4; err: relative error <= 1e-4; inliers
    exact; b: plain relative error |b - b_ref| / |b_ref| <= 1e-4 at every pose
    away from the scene's planted pose.  At the planted pose b nearly vanishes
    (it is the gradient at the optimum), so there b is held to 1e-4 relative to
    max(|b|, sqrt(err |H|_F)), the scale Cauchy-Schwarz bounds |b| by.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_00242_gb300 import api, synth
from paper_2202_00242_gb300._lib import VGICPError

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


def check_factor(out, inl, ref, what="", planted=False):
    """H, b, err and the inlier count of one factor against the oracle's.
    ``planted``: the pose is the scene's planted (ground-truth) pose, where b is
    held to the Cauchy-Schwarz scale only; elsewhere also to plain 1e-4."""
    H, b, err = api.unpack(out.cpu().double())
    H, b, err = H.numpy(), b.numpy(), float(err)
    assert int(inl) == ref.inliers, what
    eH = cases.rel_fro(H, ref.H)
    eb = cases.b_error(b, ref.b, ref.err, ref.H)
    ebp = cases.b_rel(b, ref.b)
    ee = abs(err - ref.err) / max(abs(ref.err), 1e-300)
    assert eH <= TOL and eb <= TOL and ee <= TOL, (what, eH, eb, ee)
    if not planted:
        assert ebp <= TOL, (what, "plain relative b", ebp)
    assert np.array_equal(H, H.T)
    return eH, eb, ee


@pytest.mark.parametrize("r", [0.5, 0.25, 1.0, 0.3])
def test_voxelmap_bit_exact(dev, r):
    tp, tc, _, _, _, _ = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    vm.status()
    ex = vm.export()
    ref = oracle.build_voxelmap(tp, tc, r)
    assert np.array_equal(ex["keys"], ref.keys)
    assert np.array_equal(ex["counts"], ref.counts)
    assert np.array_equal(ex["means"], ref.means.astype(np.float32))
    assert np.array_equal(ex["covs"], ref.covs.astype(np.float32))


def test_voxelmap_points_on_faces(dev):
    # coordinates on exact multiples of r and just below: floor semantics at faces
    r = 0.5
    g = np.arange(-8, 8, dtype=np.float64) * r
    pts = np.stack(np.meshgrid(g, g, g[:4]), -1).reshape(-1, 3)
    pts = np.concatenate([pts, np.nextafter(pts.astype(np.float32), -np.inf)]).astype(np.float32)
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (pts.shape[0], 1))
    vm = api.VoxelMap.build(cu(pts), cu(covs), r)
    vm.status()
    ex = vm.export()
    ref = oracle.build_voxelmap(pts, covs, r)
    assert np.array_equal(ex["keys"], ref.keys)
    assert np.array_equal(ex["counts"], ref.counts)
    assert np.array_equal(ex["means"], ref.means.astype(np.float32))


@pytest.mark.parametrize("which", ["planted", "identity", "perturbed"])
def test_linearize_room_matches_oracle(dev, which):
    tp, tc, sp, sc, T_true, r = cases.room()
    T = {"planted": T_true, "identity": np.eye(4),
         "perturbed": synth.perturb_pose(np.random.default_rng(3), T_true, 0.05, 1.0)}[which]
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    lin = api.linearize(vm, cu(sp), cu(sc), T, corr=True, qkeys=True)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T, debug=True)
    assert np.array_equal(lin.qkeys.cpu().numpy().astype(np.int64), ref.qkeys)
    assert np.array_equal(lin.corr.cpu().numpy().astype(np.int64), ref.corr)
    check_factor(lin.out, lin.inliers, ref, which, planted=which == "planted")
    print(f"near-face points (<1e-5 m): {cases.near_face_count(sp, T, r)} of {sp.shape[0]}")


@pytest.mark.parametrize("n", [1, 31, 255, 256, 257, 1000, 8191])
@pytest.mark.parametrize("tile", [256, 1024, 0])
def test_ragged_sizes_and_tiles(dev, n, tile):
    tp, tc, sp, sc, T_true, r = cases.room()
    T = synth.perturb_pose(np.random.default_rng(3), T_true, 0.05, 1.0)
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    lin = api.linearize(vm, cu(sp[:n]), cu(sc[:n]), T, tile=tile)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp[:n], sc[:n], T)
    if ref.inliers == 0:
        assert int(lin.inliers) == 0
        return
    check_factor(lin.out, lin.inliers, ref, f"n={n} tile={tile}")


def test_empty_inputs(dev):
    tp, tc, sp, sc, T, r = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    e = api.linearize(vm, cu(sp[:0]), cu(sc[:0]), T)
    assert int(e.inliers) == 0 and not e.out.any()
    empty = api.VoxelMap.build(cu(tp[:0]), cu(tc[:0]), r)
    empty.status()
    assert empty.info()[0] == 0
    m = api.linearize(empty, cu(sp), cu(sc), T)
    assert int(m.inliers) == 0 and not m.out.any()
    far = T.copy()
    far[:3, 3] += 5000.0
    f = api.linearize(vm, cu(sp), cu(sc), far)
    assert int(f.inliers) == 0 and not f.out.any()


def test_batched_equals_single_bitwise(dev):
    tp, tc, sp, sc, T, r = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    poses = [T, np.eye(4), synth.perturb_pose(np.random.default_rng(1), T, 0.1, 2.0)]
    srcs = [(cu(sp), cu(sc)), (cu(sp[:5000]), cu(sc[:5000]))]
    pairs = np.array([[0, 0], [0, 1], [0, 0]])
    bat = api.linearize_batched([vm], srcs, pairs, np.stack(poses), tile=1024)
    for p in range(3):
        s = srcs[pairs[p, 1]]
        one = api.linearize(vm, s[0], s[1], poses[p], tile=1024)
        assert torch.equal(bat.out[p], one.out), p
        assert int(bat.inliers[p]) == int(one.inliers)


@pytest.mark.parametrize("r", [0.25, 1.0])
def test_corridor_window_batched(dev, r):
    w = cases.workload_with_knn_covs("corridor", resolution=r, perturb=(0.05, 1.0))
    K = len(w.clouds.offsets) - 2
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts[: w.clouds.offsets[K]], covs[: w.clouds.offsets[K]],
                               w.clouds.offsets[: K + 1], r)
    maps[0].status()
    sp, sc = w.clouds.cloud(K)
    src = [(cu(sp), cu(sc))]
    pairs = np.stack([np.arange(K), np.zeros(K, np.int64)], 1)
    bat = api.linearize_batched(maps, src, pairs, w.poses)
    for k in range(K):
        tp, tc = w.clouds.cloud(k)
        ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, w.poses[k], nthreads=0)
        check_factor(bat.out[k], bat.inliers[k], ref, f"keyframe {k}")


def test_outdoor_submaps_batched(dev):
    w = cases.workload_with_knn_covs("outdoor", seed=33, n_submaps=10, neighbours=3)
    C = len(w.clouds.offsets) - 1
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    srcs = [(pts[w.clouds.offsets[c]:w.clouds.offsets[c + 1]],
             covs[w.clouds.offsets[c]:w.clouds.offsets[c + 1]]) for c in range(C)]
    bat = api.linearize_batched(maps, srcs, w.pairs, w.poses, tile=4096)
    omaps = {}
    for p, (j, i) in enumerate(w.pairs):
        if j not in omaps:
            tp, tc = w.clouds.cloud(j)
            omaps[j] = oracle.build_voxelmap(tp, tc, w.resolution)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(omaps[j], sp, sc, w.poses[p], nthreads=0)
        check_factor(bat.out[p], bat.inliers[p], ref, f"pair {p}")


@pytest.mark.parametrize("pose", ["planted", "perturbed"])
@pytest.mark.parametrize("mode", ["single", "batched"])
def test_27_neighbours_match_oracle(dev, mode, pose):
    tp, tc, sp, sc, T, r = cases.room(seed=4, n_target=4096, n_source=3000)
    if pose == "perturbed":
        T = synth.perturb_pose(np.random.default_rng(4), T, 0.05, 1.0)
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T, neighbours=27,
                           debug=True)
    if mode == "single":
        lin = api.linearize(vm, cu(sp), cu(sc), T, neighbours=27, corr=True)
        assert np.array_equal(lin.corr.cpu().numpy().astype(np.int64), ref.corr)
        out, inl = lin.out, lin.inliers
    else:
        bat = api.linearize_batched([vm], [(cu(sp), cu(sc))], [[0, 0]], T[None], neighbours=27,
                                    tile=512)
        out, inl = bat.out[0], bat.inliers[0]
    check_factor(out, inl, ref, mode, planted=pose == "planted")


def test_repeated_linearizations_identical(dev):
    w = cases.workload_with_knn_covs("corridor", resolution=0.25, perturb=(0.05, 1.0))
    K = len(w.clouds.offsets) - 2
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts[: w.clouds.offsets[K]], covs[: w.clouds.offsets[K]],
                               w.clouds.offsets[: K + 1], 0.25)
    sp, sc = w.clouds.cloud(K)
    src = [(cu(sp), cu(sc))]
    pairs = np.stack([np.arange(K), np.zeros(K, np.int64)], 1)
    first = api.linearize_batched(maps, src, pairs, w.poses).out.clone()
    for _ in range(100):
        again = api.linearize_batched(maps, src, pairs, w.poses).out
        assert torch.equal(first, again)


def test_rebuild_matches_fresh_build(dev):
    w = cases.workload_with_knn_covs("corridor", resolution=0.25, perturb=(0.05, 1.0))
    K = len(w.clouds.offsets) - 2
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    off = w.clouds.offsets[: K + 1]
    maps = api.build_voxelmaps(pts[: off[-1]], covs[: off[-1]], off, 0.25)
    # rebuild from shuffled-within-cloud data, then back to the original
    perm = np.concatenate([np.random.default_rng(0).permutation(np.arange(off[c], off[c + 1]))
                           for c in range(K)])
    api.rebuild_voxelmaps(maps, pts[perm].contiguous(), covs[perm].contiguous())
    maps[0].status()
    api.rebuild_voxelmaps(maps, pts[: off[-1]], covs[: off[-1]])
    fresh = api.build_voxelmaps(pts[: off[-1]], covs[: off[-1]], off, 0.25)
    for a, b in zip(maps, fresh):
        ea, eb = a.export(), b.export()
        for k in ea:
            assert np.array_equal(ea[k], eb[k])


def test_build_error_paths_leave_context_usable(dev):
    rng = np.random.default_rng(0)
    pts = rng.uniform(-100, 100, size=(4096, 3)).astype(np.float32)
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (4096, 1))
    full = api.VoxelMap.build(cu(pts), cu(covs), 0.01, max_probe=1, capacity_factor=1)
    with pytest.raises(VGICPError) as e:
        full.status()
    assert e.value.code == -3
    far = pts.copy()
    far[7] = [3.0e7, 0.0, 0.0]
    bad = api.VoxelMap.build(cu(far), cu(covs), 0.5)
    with pytest.raises(VGICPError) as e:
        bad.status()
    assert e.value.code == -4
    nan = pts.copy()
    nan[3, 1] = np.nan
    badn = api.VoxelMap.build(cu(nan), cu(covs), 0.5)
    with pytest.raises(VGICPError) as e:
        badn.status()
    assert e.value.code == -4
    # the context still works
    tp, tc, sp, sc, T, r = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    vm.status()
    lin = api.linearize(vm, cu(sp), cu(sc), T)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T)
    check_factor(lin.out, lin.inliers, ref, planted=True)


def test_pose_validation(dev):
    tp, tc, sp, sc, T, r = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    bad = T.copy()
    bad[0, 3] = np.nan
    with pytest.raises(VGICPError) as e:
        api.linearize(vm, cu(sp), cu(sc), bad)
    assert e.value.code == -1
    scaled = T.copy()
    scaled[:3, :3] *= 1.1
    with pytest.raises(VGICPError):
        api.linearize(vm, cu(sp), cu(sc), scaled)
    with pytest.raises(VGICPError):
        api.linearize_batched([vm], [(cu(sp), cu(sc))], [[0, 1]], T[None])


@pytest.mark.parametrize("pose", ["planted", "perturbed"])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_kernel_variants_match_oracle(dev, variant, pose):
    tp, tc, sp, sc, T, r = cases.room()
    if pose == "perturbed":
        T = synth.perturb_pose(np.random.default_rng(6), T, 0.05, 1.0)
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    lin = api.linearize(vm, cu(sp), cu(sc), T, corr=True, variant=variant)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T, debug=True)
    assert np.array_equal(lin.corr.cpu().numpy().astype(np.int64), ref.corr)
    planted = pose == "planted"
    check_factor(lin.out, lin.inliers, ref, f"variant {variant}", planted=planted)
    bat = api.linearize_batched([vm], [(cu(sp), cu(sc))], [[0, 0]], T[None], variant=variant,
                                tile=1000)
    check_factor(bat.out[0], bat.inliers[0], ref, f"batched variant {variant}", planted=planted)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_map_as_source(dev, variant):
    """A map's own (voxel-grouped) cloud as the source gives the same factor as the
    original cloud, within tolerance, and matches the oracle."""
    w = cases.workload_with_knn_covs("outdoor", seed=33, n_submaps=10, neighbours=3)
    C = len(w.clouds.offsets) - 1
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    srcs = [(pts[w.clouds.offsets[c]:w.clouds.offsets[c + 1]],
             covs[w.clouds.offsets[c]:w.clouds.offsets[c + 1]]) for c in range(C)]
    a = api.linearize_batched(maps, srcs, w.pairs, w.poses, variant=variant)
    b = api.linearize_batched(maps, maps, w.pairs, w.poses, variant=variant)
    assert torch.equal(a.inliers, b.inliers)
    omaps = {}
    for p, (j, i) in enumerate(w.pairs[:8]):
        if j not in omaps:
            tp, tc = w.clouds.cloud(j)
            omaps[j] = oracle.build_voxelmap(tp, tc, w.resolution)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(omaps[j], sp, sc, w.poses[p], nthreads=0)
        check_factor(b.out[p], b.inliers[p], ref, f"pair {p}")


def test_plan_graph_autotune_matches_oracle_and_batched(dev):
    """The plan (work list built once, autotuned launch shape, CUDA graph replay)
    gives the oracle's factors; replays with the same poses are bitwise identical
    and a replay with other poses equals a fresh batched call of that shape."""
    w = cases.workload_with_knn_covs("outdoor", seed=33, n_submaps=10, neighbours=3)
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    plan = api.Plan(maps, maps, w.pairs)
    info = plan.autotune(w.poses)
    assert info["variant"] in (1, 2, 3) and info["item_points"] in (4096, 8192, 16384, 32768)
    a = plan.execute(w.poses).out.clone()
    b = plan.execute(w.poses).out.clone()
    assert torch.equal(a, b)
    poses2 = np.stack([synth.perturb_pose(np.random.default_rng(k), T, 0.02, 0.5)
                       for k, T in enumerate(w.poses)])
    c = plan.execute(poses2)
    d = api.linearize_batched(maps, maps, w.pairs, poses2, tile=info["item_points"],
                              variant=info["variant"])
    assert torch.equal(c.out, d.out) and torch.equal(c.inliers, d.inliers)
    omaps = {}
    for p, (j, i) in enumerate(w.pairs[:6]):
        if j not in omaps:
            tp, tc = w.clouds.cloud(j)
            omaps[j] = oracle.build_voxelmap(tp, tc, w.resolution)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(omaps[j], sp, sc, poses2[p], nthreads=0)
        check_factor(c.out[p], c.inliers[p], ref, f"plan pair {p}")
    plan.close()


def test_overlap_rate_matches_oracle_and_linearize(dev):
    """Overlap rate (Sec. III-D) of every factor equals the oracle's and the
    linearization's inlier count over n, exactly."""
    w = cases.workload_with_knn_covs("outdoor", seed=33, n_submaps=10, neighbours=3)
    C = len(w.clouds.offsets) - 1
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    srcs = [(pts[w.clouds.offsets[c]:w.clouds.offsets[c + 1]],
             covs[w.clouds.offsets[c]:w.clouds.offsets[c + 1]]) for c in range(C)]
    rate, inl = api.overlap_batched(maps, srcs, w.pairs, w.poses, tile=4096)
    lin = api.linearize_batched(maps, srcs, w.pairs, w.poses, tile=4096)
    assert torch.equal(inl, lin.inliers)
    rate_m, inl_m = api.overlap_batched(maps, maps, w.pairs, w.poses)
    assert torch.equal(inl_m, inl)  # the grouped copy holds the same points
    for p, (j, i) in enumerate(w.pairs):
        tp, tc = w.clouds.cloud(j)
        sp, _ = w.clouds.cloud(i)
        assert float(rate[p]) == oracle.overlap(oracle.build_voxelmap(tp, tc, w.resolution), sp,
                                                w.poses[p])


def test_factor_candidates_threshold(dev):
    """Global-map factor creation (Sec. III-F): all ordered pairs whose overlap at
    the relative world pose reaches the threshold, and no others."""
    w = cases.workload_with_knn_covs("outdoor", seed=34, n_submaps=8, neighbours=2)
    C = len(w.clouds.offsets) - 1
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    pairs, rates = api.factor_candidates(maps, maps, w.world_poses, threshold=0.05)
    got = {(int(j), int(i)) for j, i in pairs}
    assert (rates >= 0.05).all() and len(got) > 0
    omaps = [oracle.build_voxelmap(*w.clouds.cloud(j), w.resolution) for j in range(C)]
    for j in range(C):
        for i in range(C):
            if i == j:
                continue
            T = api.relative_poses(w.world_poses, [[j, i]])[0]
            o = oracle.overlap(omaps[j], w.clouds.cloud(i)[0], T)
            assert ((j, i) in got) == (o >= 0.05), (j, i, o)


def test_plan_27_neighbours_matches_oracle(dev):
    """A 27-neighbour factor set as a plan (CUDA graph, autotuned item size)."""
    w = cases.workload_with_knn_covs("outdoor", seed=35, n_submaps=6, neighbours=2)
    w_r = 0.5
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w_r)
    maps[0].status()
    plan = api.Plan(maps, maps, w.pairs, neighbours=27)
    plan.autotune(w.poses)
    res = plan.execute(w.poses)
    for p, (j, i) in enumerate(w.pairs[:4]):
        ref = oracle.linearize(oracle.build_voxelmap(*w.clouds.cloud(j), w_r),
                               *w.clouds.cloud(i), w.poses[p], neighbours=27, nthreads=0)
        check_factor(res.out[p], res.inliers[p], ref, f"27-neighbour plan pair {p}")
    plan.close()


def test_rebuild_with_more_voxels_keeps_parity(dev):
    """A rebuild keeps the lookup-table region of the first build (sized from its
    voxel count, and at least 2 n slots); clouds of the same size with many more
    voxels still give the oracle's map and factors."""
    rng = np.random.default_rng(12)
    n = 6000
    dense = (rng.normal(size=(n, 3)) * 0.6).astype(np.float32)   # few voxels
    sparse = (rng.random((n, 3)) * 12.0 - 6.0).astype(np.float32)  # many more
    covs = np.tile(np.array([0.02, 0, 0, 0.02, 0, 0.02], np.float32), (n, 1))
    r = 0.5
    vm = api.VoxelMap.build(cu(dense), cu(covs), r)
    vm.status()
    v_first = vm.info()[0]
    api.rebuild_voxelmaps([vm], cu(sparse), cu(covs))
    vm.status()
    ex = vm.export()
    ref = oracle.build_voxelmap(sparse, covs, r)
    assert ref.num_voxels > 4 * v_first
    assert np.array_equal(ex["keys"], ref.keys) and np.array_equal(ex["counts"], ref.counts)
    src = sparse[::3] + np.float32(0.05)
    T = np.eye(4)
    lin = api.linearize(vm, cu(src), cu(covs[::3]), T)
    refl = oracle.linearize(ref, src, covs[::3], T)
    check_factor(lin.out, lin.inliers, refl, "after rebuild")


@pytest.mark.gpu
def test_rebuilds_leave_no_stale_table_entries(dev):
    """A rebuild empties only the table slots of the previous build's voxels.
    Alternating clouds with many and few voxels must give, after every rebuild,
    exactly the maps and factors of a fresh build: a slot left behind would add
    hits (inliers) for voxels the new cloud does not have."""
    rng = np.random.default_rng(31)
    n, K, r = 5000, 3, 0.5
    sparse = (rng.random((K * n, 3)) * 14.0 - 7.0).astype(np.float32)
    dense = (rng.normal(size=(K * n, 3)) * 0.7).astype(np.float32)
    covs = np.tile(np.array([0.02, 0, 0, 0.02, 0, 0.02], np.float32), (K * n, 1))
    off = np.arange(K + 1, dtype=np.int64) * n
    probe = (rng.random((4000, 3)) * 14.0 - 7.0).astype(np.float32)
    pcov = np.tile(np.array([0.02, 0, 0, 0.02, 0, 0.02], np.float32), (4000, 1))
    pairs = np.array([[m, 0] for m in range(K)], np.int32)
    poses = np.stack([np.eye(4)] * K)
    srcs = [(cu(probe), cu(pcov))]
    maps = api.build_voxelmaps(cu(sparse), cu(covs), off, r)
    for cloud in (dense, sparse, dense, sparse):
        api.rebuild_voxelmaps(maps, cu(cloud), cu(covs))
        fresh = api.build_voxelmaps(cu(cloud), cu(covs), off, r)
        for a, b in zip(maps, fresh):
            a.status()
            ea, eb = a.export(), b.export()
            for k in ea:
                assert np.array_equal(ea[k], eb[k]), k
        got = api.linearize_batched(maps, srcs, pairs, poses)
        ref = api.linearize_batched(fresh, srcs, pairs, poses)
        assert torch.equal(got.out, ref.out) and torch.equal(got.inliers, ref.inliers)
        ring = [[m, (m + 1) % K] for m in range(K)]  # the maps' grouped clouds as sources
        got = api.linearize_batched(maps, maps, ring, poses)
        ref = api.linearize_batched(fresh, fresh, ring, poses)
        assert torch.equal(got.out, ref.out) and torch.equal(got.inliers, ref.inliers)
        for b in fresh:
            b.close()
