"""Differentiable factors and the optimizer loop on the GPU (arXiv 2202.00242
Sec. III-A: the factor is re-linearized at every iteration).

  * cost / Gauss-Newton gradient / exact gradient kernels vs the oracle's err,
    2 b and exact gradient;
  * the autograd Function's backward vs binary64 central differences (h = 1e-6)
    of the oracle's cost, and vs 2 b;
  * gradient-descent refinement from a 0.3 m / 5 deg perturbation;
  * Gauss-Newton with the library's host solve and exp map vs the oracle's
    Gauss-Newton trajectory, and recovery of the planted pose.
"""
import numpy as np
import pytest
import torch

import cases
import oracle
from oracle import se3
from paper_2202_00242_gb300 import api, autograd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_00242_gb300 import build
    build.build()
    return torch.device("cuda:0")


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def small_set(dev):
    """8 factors among 6 outdoor submaps (k-NN covariances), perturbed 0.3 m / 5 deg."""
    w = cases.workload_with_knn_covs("outdoor", seed=44, n_submaps=6, neighbours=2,
                                     n_min=20000, n_max=50000, size_dist="uniform",
                                     perturb=(0.3, 5.0))
    pts, covs = cu(w.clouds.points), cu(w.clouds.covs)
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    srcs = [(pts[w.clouds.offsets[c]:w.clouds.offsets[c + 1]],
             covs[w.clouds.offsets[c]:w.clouds.offsets[c + 1]])
            for c in range(len(w.clouds.offsets) - 1)]
    omaps = {}
    for j in set(int(j) for j in w.pairs[:, 0]):
        tp, tc = w.clouds.cloud(j)
        omaps[j] = oracle.build_voxelmap(tp, tc, w.resolution)
    return w, maps, srcs, omaps


def _ref(w, omaps, p, T):
    j, i = (int(x) for x in w.pairs[p])
    sp, sc = w.clouds.cloud(i)
    return oracle.linearize(omaps[j], sp, sc, T, debug=True, nthreads=0), sp, sc


def test_evaluate_modes_match_oracle(small_set):
    w, maps, srcs, omaps = small_set
    g2, err, inl = api.evaluate_batched(maps, srcs, w.pairs, w.poses, mode=api.GRADIENT)
    g3, err3, _ = api.evaluate_batched(maps, srcs, w.pairs, w.poses, mode=api.EXACT_GRADIENT)
    _, err1, _ = api.evaluate_batched(maps, srcs, w.pairs, w.poses, mode=api.COST)
    g2, g3 = g2.cpu().numpy(), g3.cpu().numpy()
    for p in range(w.pairs.shape[0]):
        ref, sp, sc = _ref(w, omaps, p, w.poses[p])
        j = int(w.pairs[p, 0])
        gex = oracle.exact_gradient(omaps[j], sp, sc, w.poses[p], ref.corr)
        assert int(inl[p]) == ref.inliers
        scale = max(np.linalg.norm(2 * ref.b), 2 * np.sqrt(ref.err * np.linalg.norm(ref.H)))
        assert np.linalg.norm(g2[p] - 2 * ref.b) <= 1e-4 * scale
        assert np.linalg.norm(g2[p] - 2 * ref.b) <= 1e-4 * np.linalg.norm(2 * ref.b)
        assert np.linalg.norm(g3[p] - gex) <= 1e-4 * max(scale, np.linalg.norm(gex))
        for e in (err, err3, err1):
            assert abs(float(e[p]) - ref.err) <= 1e-4 * ref.err


def test_backward_batched_is_the_gradient_mode(small_set):
    """vgicp_backward_batched gives the gradient modes of vgicp_evaluate_batched,
    bit for bit, and rejects an exact flag other than 0 or 1."""
    import ctypes
    from paper_2202_00242_gb300 import _lib
    w, maps, srcs, omaps = small_set
    for exact, mode in ((False, api.GRADIENT), (True, api.EXACT_GRADIENT)):
        g, e, i = api.backward_batched(maps, srcs, w.pairs, w.poses, exact=exact)
        g2, e2, i2 = api.evaluate_batched(maps, srcs, w.pairs, w.poses, mode=mode)
        assert torch.equal(g, g2) and torch.equal(e, e2) and torch.equal(i, i2)
    lib = _lib.load()
    clouds = api.make_clouds(srcs)
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    pairs = np.ascontiguousarray(w.pairs, dtype=np.int32)
    poses = np.ascontiguousarray(w.poses, dtype=np.float64)
    out = torch.empty((len(pairs), 7), dtype=torch.float64, device="cuda")
    inl = torch.empty(len(pairs), dtype=torch.int64, device="cuda")
    rc = lib.vgicp_backward_batched(arr, len(maps), clouds, len(srcs),
                                    pairs.ctypes.data_as(ctypes.c_void_p), len(pairs),
                                    poses.ctypes.data_as(ctypes.c_void_p), 2,
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(inl.data_ptr()), None,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1


def test_autograd_backward_vs_finite_differences(small_set):
    """d err / d xi at a nonzero xi: the backward kernel (exact mode) composed with
    the SE(3) right Jacobian vs binary64 central differences of the oracle's cost
    with the correspondences of the evaluation point held."""
    w, maps, srcs, omaps = small_set
    fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses, exact=True)
    rng = np.random.default_rng(5)
    x0 = rng.normal(size=(w.pairs.shape[0], 6)) * np.array([0.01, 0.01, 0.01, 0.05, 0.05, 0.05])
    xi = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    err = fs.cost(xi)
    err.sum().backward()
    err = err.detach()
    g = xi.grad.numpy()
    h = 1e-6
    for p in range(w.pairs.shape[0]):
        T = w.poses[p] @ se3.se3_exp(x0[p])
        ref, sp, sc = _ref(w, omaps, p, T)
        j = int(w.pairs[p, 0])
        assert abs(float(err[p]) - ref.err) <= 1e-4 * ref.err
        gfd = np.zeros(6)
        for i in range(6):
            e = np.zeros(6)
            e[i] = h
            fp = oracle.cost_fixed(omaps[j], sp, sc, w.poses[p] @ se3.se3_exp(x0[p] + e), ref.corr)
            fm = oracle.cost_fixed(omaps[j], sp, sc, w.poses[p] @ se3.se3_exp(x0[p] - e), ref.corr)
            gfd[i] = (fp - fm) / (2 * h)
        assert np.linalg.norm(g[p] - gfd) <= 2e-4 * np.linalg.norm(gfd), (p, g[p], gfd)


def test_autograd_gauss_newton_gradient_is_2b(small_set):
    w, maps, srcs, omaps = small_set
    fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses, exact=False)
    xi = torch.zeros((w.pairs.shape[0], 6), dtype=torch.float64, requires_grad=True)
    fs.cost(xi).sum().backward()
    for p in range(w.pairs.shape[0]):
        ref, _, _ = _ref(w, omaps, p, w.poses[p])
        scale = max(np.linalg.norm(2 * ref.b), 2 * np.sqrt(ref.err * np.linalg.norm(ref.H)))
        assert np.linalg.norm(xi.grad[p].numpy() - 2 * ref.b) <= 1e-4 * scale
        assert np.linalg.norm(xi.grad[p].numpy() - 2 * ref.b) <= 1e-4 * np.linalg.norm(2 * ref.b)


def test_gradient_descent_refinement_reduces_cost(small_set):
    """Pose refinement by gradient steps preconditioned with H (the backward
    kernel's gradient, re-evaluated each step) from 0.3 m / 5 deg."""
    w, maps, srcs, omaps = small_set
    poses = w.poses.copy()
    _, err0, _ = api.evaluate_batched(maps, srcs, w.pairs, poses, mode=api.COST)
    for _ in range(15):
        lin = api.linearize_batched(maps, srcs, w.pairs, poses)
        H, _, _ = api.unpack(lin.out.cpu())
        fs = autograd.FactorSet(maps, srcs, w.pairs, poses, exact=False)
        xi = torch.zeros((w.pairs.shape[0], 6), dtype=torch.float64, requires_grad=True)
        fs.cost(xi).sum().backward()
        for p in range(w.pairs.shape[0]):
            step = -0.5 * np.linalg.solve(H[p].numpy(), xi.grad[p].numpy())
            poses[p] = poses[p] @ api.se3_exp(step)
    _, err1, _ = api.evaluate_batched(maps, srcs, w.pairs, poses, mode=api.COST)
    assert (err1 < err0).all()
    rot, tr = zip(*[se3.pose_error(poses[p], w.true_poses[p]) for p in range(w.pairs.shape[0])])
    rot0, tr0 = zip(*[se3.pose_error(w.poses[p], w.true_poses[p]) for p in range(w.pairs.shape[0])])
    assert np.median(tr) < 0.5 * np.median(tr0) and np.median(rot) < 0.5 * np.median(rot0)


def test_gauss_newton_matches_oracle_trajectory(dev):
    tp, tc, sp, sc, T_true, r = cases.room()
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    T_gpu, hist = api.gauss_newton(vm, cu(sp), cu(sc), np.eye(4), max_iters=8, tol=0)
    ovm = oracle.build_voxelmap(tp, tc, r)

    def lin(T):
        x = oracle.linearize(ovm, sp, sc, T)
        return x.H, x.b, x.err

    T_ref, hist_ref = se3.gauss_newton(lin, np.eye(4), max_iters=8, tol=0)
    for (e, s), (er, sr) in zip(hist, hist_ref):
        assert abs(e - er) <= 1e-4 * er
    rot, tr = se3.pose_error(T_gpu, T_ref)
    assert rot < 1e-3 and tr < 1e-4
    T_conv, _ = api.gauss_newton(vm, cu(sp), cu(sc), np.eye(4), max_iters=40, tol=1e-9)
    rot, tr = se3.pose_error(T_conv, T_true)
    assert rot < 0.1 and tr < 0.01, (rot, tr)


def test_pose_graph_gauss_newton_converges(dev):  # noqa: F811
    """Global-map optimization over submap world poses (Sec. III-F, matching-cost
    factors only): the first iteration's normal equations match those built from
    the oracle's linearizations, and the perturbed poses converge to the true
    ones within the bias of the voxelized cost."""
    from paper_2202_00242_gb300 import api, synth
    w = synth.with_surface_covariances(synth.outdoor_submaps(
        seed=41, n_submaps=8, n_min=20000, n_max=30000, neighbours=3, size_dist="uniform"))
    C = len(w.clouds.offsets) - 1
    pts = torch.from_numpy(w.clouds.points).cuda()
    covs = torch.from_numpy(w.clouds.covs).cuda()
    maps = api.build_voxelmaps(pts, covs, w.clouds.offsets, w.resolution)
    maps[0].status()
    srcs = [(pts[w.clouds.offsets[c]:w.clouds.offsets[c + 1]],
             covs[w.clouds.offsets[c]:w.clouds.offsets[c + 1]]) for c in range(C)]
    rng = np.random.default_rng(5)
    W0 = np.array(w.world_poses)
    for c in range(1, C):
        W0[c] = W0[c] @ api.se3_exp(np.r_[rng.normal(0, np.radians(1.0), 3), rng.normal(0, 0.1, 3)])
    # first-iteration normal equations against the oracle's factors
    poses = api.relative_poses(W0, w.pairs)
    lin = api.linearize_batched(maps, srcs, w.pairs, poses).out.cpu().numpy()
    Hg = np.zeros((6 * C, 6 * C))
    Ho = np.zeros((6 * C, 6 * C))
    for p, (j, i) in enumerate(w.pairs):
        ref = oracle.linearize(oracle.build_voxelmap(*w.clouds.cloud(j), w.resolution),
                               *w.clouds.cloud(i), poses[p], nthreads=0)
        idx = np.r_[6 * i:6 * i + 6, 6 * j:6 * j + 6]
        Hg[np.ix_(idx, idx)] += api.binary_factor(lin[p, :36], lin[p, 36:42], poses[p])[0]
        Ho[np.ix_(idx, idx)] += api.binary_factor(ref.H, ref.b, poses[p])[0]
    assert np.linalg.norm(Hg - Ho) <= 1e-4 * np.linalg.norm(Ho)

    def errors(W):  # (max translation error [m], max rotation error [deg])
        e = [se3.pose_error(np.linalg.inv(W[0]) @ W[c],
                            np.linalg.inv(w.world_poses[0]) @ w.world_poses[c])
             for c in range(1, C)]
        return max(t for _, t in e), max(r for r, _ in e)

    t0, r0 = errors(W0)
    W, hist = api.optimize_pose_graph(maps, srcs, w.pairs, W0, fixed=0, iters=8)
    t1, r1 = errors(W)
    assert hist[-1] < hist[0]
    assert t1 < 0.3 * t0 and t1 < 0.05, (t0, t1)
    assert r1 < 0.3 * r0, (r0, r1)
