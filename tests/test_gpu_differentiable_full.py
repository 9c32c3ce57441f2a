"""Differentiable factors at the full size of the differentiable workload:
256 factor pairs among 64 submaps of 20k-50k points, poses perturbed by 0.3 m /
5 deg, res 1.0 m (arXiv 2202.00242 Sec. III-A: the cost is re-evaluated and
differentiated at every optimizer iteration).

  * forward err and backward gradient (W held: 2 J^T W d) of every factor vs the
    oracle's err and 2 b; the exact gradient vs the oracle's exact gradient;
  * the backward pass at a nonzero increment xi vs binary64 central differences
    (h = 1e-6) of the oracle's cost, correspondences held, on sampled factors;
  * gradient-descent refinement of all 256 poses from the perturbed start.
The poses T0 Exp(xi) and the right Jacobians are composed on the device.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import se3
from paper_2202_00242_gb300 import api, autograd, synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def full_set():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_00242_gb300 import build
    build.build()
    w = synth.with_surface_covariances(synth.config_differentiable())
    assert w.pairs.shape[0] == 256
    sizes = np.diff(w.clouds.offsets)
    assert sizes.min() >= 20000 and sizes.max() <= 50000
    pts = torch.from_numpy(w.clouds.points).cuda()
    covs = torch.from_numpy(w.clouds.covs).cuda()
    off = w.clouds.offsets
    maps = api.build_voxelmaps(pts, covs, off, w.resolution)
    maps[0].status()
    srcs = [(pts[off[c]:off[c + 1]], covs[off[c]:off[c + 1]]) for c in range(len(off) - 1)]
    omaps = {j: oracle.build_voxelmap(*w.clouds.cloud(j), w.resolution)
             for j in sorted(set(int(j) for j in w.pairs[:, 0]))}
    refs = []
    for p, (j, i) in enumerate(w.pairs):
        refs.append(oracle.linearize(omaps[int(j)], *w.clouds.cloud(int(i)), w.poses[p],
                                     debug=True, nthreads=0))
    return w, maps, srcs, omaps, refs


def _grad(fs, xi):
    xi = xi.clone().requires_grad_(True)
    err = fs.cost(xi)
    err.sum().backward()
    return err.detach(), xi.grad.detach()


def test_forward_and_backward_match_oracle_on_all_factors(full_set):
    w, maps, srcs, omaps, refs = full_set
    P = w.pairs.shape[0]
    xi = torch.zeros((P, 6), dtype=torch.float64, device="cuda")
    fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses)
    err, g = _grad(fs, xi)
    err, g = err.cpu().numpy(), g.cpu().numpy()
    fx = autograd.FactorSet(maps, srcs, w.pairs, w.poses, exact=True)
    _, gx = _grad(fx, xi)
    gx = gx.cpu().numpy()
    worst = [0.0, 0.0, 0.0]
    for p, ref in enumerate(refs):
        j, i = (int(x) for x in w.pairs[p])
        e_err = abs(err[p] - ref.err) / ref.err
        e_g = np.linalg.norm(g[p] - 2 * ref.b) / np.linalg.norm(2 * ref.b)
        gex = oracle.exact_gradient(omaps[j], *w.clouds.cloud(i), w.poses[p], ref.corr)
        e_x = np.linalg.norm(gx[p] - gex) / np.linalg.norm(gex)
        assert e_err <= TOL and e_g <= TOL and e_x <= TOL, (p, e_err, e_g, e_x)
        worst = [max(a, b) for a, b in zip(worst, (e_err, e_g, e_x))]
    print(f"256 factors: max rel err {worst[0]:.2e}, grad vs 2b {worst[1]:.2e}, "
          f"exact grad {worst[2]:.2e}")


def test_backward_vs_finite_differences(full_set):
    w, maps, srcs, omaps, refs = full_set
    P = w.pairs.shape[0]
    rng = np.random.default_rng(8)
    x0 = rng.normal(size=(P, 6)) * np.array([0.01, 0.01, 0.01, 0.05, 0.05, 0.05])
    fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses, exact=True)
    err, g = _grad(fs, torch.tensor(x0, device="cuda"))
    err, g = err.cpu().numpy(), g.cpu().numpy()
    h = 1e-6
    for p in rng.choice(P, 6, replace=False):
        j, i = (int(x) for x in w.pairs[p])
        sp, sc = w.clouds.cloud(i)
        T = w.poses[p] @ se3.se3_exp(x0[p])
        ref = oracle.linearize(omaps[j], sp, sc, T, debug=True, nthreads=0)
        assert abs(err[p] - ref.err) <= TOL * ref.err
        gfd = np.zeros(6)
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            fp = oracle.cost_fixed(omaps[j], sp, sc, w.poses[p] @ se3.se3_exp(x0[p] + e), ref.corr)
            fm = oracle.cost_fixed(omaps[j], sp, sc, w.poses[p] @ se3.se3_exp(x0[p] - e), ref.corr)
            gfd[k] = (fp - fm) / (2 * h)
        assert np.linalg.norm(g[p] - gfd) <= 2e-4 * np.linalg.norm(gfd), (p, g[p], gfd)


def test_gradient_descent_refinement_from_perturbed_poses(full_set):
    """Gradient steps preconditioned by H (the backward kernel's gradient and a
    batched linearization at the current poses, re-evaluated every step) from
    the 0.3 m / 5 deg perturbations.  The raw cost is a sum over the points that
    currently have a voxel, so it may grow as a pose improves and more points
    find one; convergence is judged by the error per inlier and by the pose
    error against the ground truth."""
    w, maps, srcs, omaps, refs = full_set
    P = w.pairs.shape[0]
    zero = torch.zeros((P, 6), dtype=torch.float64, device="cuda")
    fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses)
    poses = w.poses.copy()

    def per_inlier(poses_now):
        fs.rebase(poses_now)
        out, inl = fs.plan.evaluate(fs.base, zero, mode=api.COST)
        return out[:, 6].cpu().numpy() / np.maximum(inl.cpu().numpy(), 1)

    e0 = per_inlier(poses)
    for _ in range(12):
        fs.rebase(poses)
        lin = api.linearize_batched(maps, srcs, w.pairs, poses)
        H = lin.out[:, :36].reshape(P, 6, 6).cpu().numpy()
        _, g = _grad(fs, zero)
        g = g.cpu().numpy()
        for p in range(P):
            poses[p] = poses[p] @ api.se3_exp(-0.5 * np.linalg.solve(H[p], g[p]))
    e1 = per_inlier(poses)
    rot, tr = map(np.array, zip(*[se3.pose_error(poses[p], w.true_poses[p]) for p in range(P)]))
    rot0, tr0 = map(np.array, zip(*[se3.pose_error(w.poses[p], w.true_poses[p])
                                    for p in range(P)]))
    print(f"median error per inlier {np.median(e0):.3f} -> {np.median(e1):.3f}; median pose "
          f"error {np.median(tr0):.3f} m / {np.median(rot0):.2f} deg -> {np.median(tr):.4f} m / "
          f"{np.median(rot):.3f} deg; improved {np.mean(tr < tr0):.3f} / {np.mean(rot < rot0):.3f}")
    assert np.median(e1) < 0.5 * np.median(e0)
    assert np.median(tr) < 0.3 * np.median(tr0) and np.median(rot) < 0.3 * np.median(rot0)
    assert np.mean(tr < tr0) >= 0.8 and np.mean(rot < rot0) >= 0.8
