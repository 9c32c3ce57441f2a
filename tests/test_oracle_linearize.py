"""Pins of the oracle's factor linearisation (arXiv 2202.00242 Sec. III-A, Eqs. 2-3
and the Hessian factor obtained from their derivatives).

Each pin is independent of the oracle's own formula: brute-force lookups,
hand-expanded closed forms (point-to-point ICP normal equations), finite
differences, exact invariances of the cost, and Gauss-Newton recovery of a
planted pose.  Together they fail on a dropped term, a flipped sign, a wrong
index or a transposed operand anywhere in the oracle."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import se3
from paper_2202_00242_gb300 import synth


def _room_case(n_t=1500, n_s=1500, seed=11, r=0.5, dyadic=False):
    import oracle
    w = synth.room_pair(seed=seed, n_target=n_t, n_source=n_s)
    tp, _ = w.clouds.cloud(0)
    sp, _ = w.clouds.cloud(1)
    if dyadic:  # values exactly representable after 90-degree rotations / shifts
        # odd multiples of 2^-13: exact in float32, never on a voxel face
        tp = (np.floor(tp * 4096) + 0.5) / 4096
        sp = (np.floor(sp * 4096) + 0.5) / 4096
    tc = oracle.knn_covariances(tp).astype(np.float32)
    sc = oracle.knn_covariances(sp).astype(np.float32)
    if dyadic:
        tc = (np.round(tc * 2**20) / 2**20).astype(np.float32)
        sc = (np.round(sc * 2**20) / 2**20).astype(np.float32)
    return tp.astype(np.float32), tc, sp.astype(np.float32), sc, w.true_poses[0], r


def _perturbed(T, seed=0, rot_deg=2.0, trans=0.05):
    rng = np.random.default_rng(seed)
    return synth.perturb_pose(rng, T, trans, rot_deg)


def _min_face_distance(q, r):
    f = q / r - np.floor(q / r)
    return float(np.min(np.minimum(f, 1 - f)) * r)


def test_lookup_matches_bruteforce(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case(400, 300)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    keys = [tuple(k) for k in vm.keys.tolist()]
    for i in range(sp.shape[0]):
        mu = sp[i].astype(np.float64)
        q = [((T[a, 0] * mu[0] + T[a, 1] * mu[1]) + T[a, 2] * mu[2]) + T[a, 3] for a in range(3)]
        key = tuple(math.floor(v / r) for v in q)
        assert tuple(lin.qkeys[i]) == key
        found = -1
        for v, kk in enumerate(keys):  # linear scan
            if kk == key:
                found = v
        assert lin.corr[i] == found
    assert lin.inliers == int((lin.corr >= 0).sum())


def test_point_to_point_closed_form(oracle_lib):
    """C_k = C'_v = I/2 makes W = I: e = sum |d|^2 and H, b are the point-to-point
    ICP normal equations under the right perturbation:
      H = sum [[ |mu|^2 I - mu mu^T, [mu]x ], [ -[mu]x, I ]],
      b = sum [ (R^T d) x mu ; -R^T d ]."""
    rng = np.random.default_rng(3)
    r = 1.0
    # one target point per voxel, at voxel centres; sources near them
    keys = rng.choice(np.arange(-4, 4), size=(40, 3))
    keys = np.unique(keys, axis=0)
    tp = (keys + 0.5).astype(np.float32)
    half = np.array([0.5, 0, 0, 0.5, 0, 0.5], dtype=np.float32)
    tc = np.tile(half, (tp.shape[0], 1))
    T = synth.make_pose(synth.axis_angle_matrix([1, 2, 3], 0.3), [0.1, -0.2, 0.05])
    Ti = synth.pose_inverse(T)
    # sources: target points pulled back through T, plus a small offset
    sp = ((tp.astype(np.float64) + rng.uniform(-0.2, 0.2, tp.shape)) @ Ti[:3, :3].T + Ti[:3, 3])
    sp = sp.astype(np.float32)
    sc = np.tile(half, (sp.shape[0], 1))
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    assert lin.inliers == sp.shape[0]
    R, t = T[:3, :3], T[:3, 3]
    H = np.zeros((6, 6))
    b = np.zeros(6)
    e = 0.0
    for i in range(sp.shape[0]):
        mu = sp[i].astype(np.float64)
        v = lin.corr[i]
        d = vm.means[v] - (R @ mu + t)
        e += d @ d
        mx = np.array([[0, -mu[2], mu[1]], [mu[2], 0, -mu[0]], [-mu[1], mu[0], 0]])
        H[:3, :3] += (mu @ mu) * np.eye(3) - np.outer(mu, mu)
        H[:3, 3:] += mx
        H[3:, :3] += -mx
        H[3:, 3:] += np.eye(3)
        dl = R.T @ d
        b[:3] += np.cross(dl, mu)
        b[3:] += -dl
    np.testing.assert_allclose(lin.err, e, rtol=1e-12)
    np.testing.assert_allclose(lin.H, H, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(lin.b, b, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(lin.W, np.tile(np.eye(3), (sp.shape[0], 1, 1)), atol=1e-12)


def test_identity_rotation_block_formulas(oracle_lib):
    """With R = I, J = [[mu]x, -I]: H_vv = sum W, H_wv = -sum [mu]x^T W,
    H_ww = sum [mu]x^T W [mu]x, b_v = -sum W d, b_w = sum (W d) x mu, and W is
    the inverse of C'_v + C_k."""
    tp, tc, sp, sc, T, r = _room_case(800, 600)
    T = T.copy()
    T[:3, :3] = np.eye(3)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    Hvv = np.zeros((3, 3))
    Hwv = np.zeros((3, 3))
    Hww = np.zeros((3, 3))
    bv = np.zeros(3)
    bw = np.zeros(3)
    e = 0.0
    for i in np.nonzero(lin.corr >= 0)[0]:
        v = lin.corr[i]
        Cv = _sym(vm.covs[v])
        Ck = _sym(sc[i].astype(np.float64))
        W = np.linalg.inv(Cv + Ck)
        np.testing.assert_allclose(lin.W[i], W, rtol=1e-9, atol=1e-9 * np.abs(W).max())
        mu = sp[i].astype(np.float64)
        d = vm.means[v] - (mu + T[:3, 3])
        np.testing.assert_allclose(lin.d[i], d, rtol=1e-13, atol=1e-14)
        mx = np.array([[0, -mu[2], mu[1]], [mu[2], 0, -mu[0]], [-mu[1], mu[0], 0]])
        Hvv += W
        Hwv += -mx.T @ W
        Hww += mx.T @ W @ mx
        bv += -W @ d
        bw += np.cross(W @ d, mu)
        e += d @ W @ d
    scale = np.abs(lin.H).max()
    np.testing.assert_allclose(lin.H[3:, 3:], Hvv, atol=1e-9 * scale)
    np.testing.assert_allclose(lin.H[:3, 3:], Hwv, atol=1e-9 * scale)
    np.testing.assert_allclose(lin.H[3:, :3], Hwv.T, atol=1e-9 * scale)
    np.testing.assert_allclose(lin.H[:3, :3], Hww, atol=1e-9 * scale)
    np.testing.assert_allclose(lin.b[3:], bv, rtol=1e-9, atol=1e-9 * np.abs(lin.b).max())
    np.testing.assert_allclose(lin.b[:3], bw, rtol=1e-9, atol=1e-9 * np.abs(lin.b).max())
    np.testing.assert_allclose(lin.err, e, rtol=1e-10)


def _sym(c):
    return np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])


def test_b_matches_finite_differences_with_frozen_weights(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case()
    T = _perturbed(T)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    h = 1e-6
    g = np.zeros(6)
    for i in range(6):
        xi = np.zeros(6)
        xi[i] = h
        fp = oracle_lib.cost_fixed(vm, sp, sc, T @ se3.se3_exp(xi), lin.corr, lin.W)
        fm = oracle_lib.cost_fixed(vm, sp, sc, T @ se3.se3_exp(-xi), lin.corr, lin.W)
        g[i] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(oracle_lib.cost_fixed(vm, sp, sc, T, lin.corr, lin.W), lin.err,
                               rtol=1e-12)
    np.testing.assert_allclose(g, 2 * lin.b, rtol=0, atol=1e-7 * np.linalg.norm(2 * lin.b) + 1e-6)


def test_H_is_half_hessian_of_residual_change(oracle_lib):
    """f(xi) = sum (d(xi) - d(0))^T W (d(xi) - d(0)) has Hessian exactly 2 J^T W J
    at 0; d(xi) = mu' - R Exp(xi) mu - t is evaluated with the matrix exponential."""
    tp, tc, sp, sc, T, r = _room_case(600, 400)
    T = _perturbed(T, seed=4)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    m = lin.corr >= 0
    mu = sp[m].astype(np.float64)
    mup = vm.means[lin.corr[m]]
    W = lin.W[m]

    def resid(xi):
        Tx = T @ scipy.linalg.expm(_twist(xi))
        return mup - (mu @ Tx[:3, :3].T + Tx[:3, 3])

    d0 = resid(np.zeros(6))

    def f(xi):
        dd = resid(xi) - d0
        return float(np.einsum("ni,nij,nj->", dd, W, dd))

    h = 1e-4
    Hfd = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            ei = np.zeros(6); ei[i] = h
            ej = np.zeros(6); ej[j] = h
            Hfd[i, j] = (f(ei + ej) - f(ei - ej) - f(-ei + ej) + f(-ei - ej)) / (4 * h * h)
    np.testing.assert_allclose(Hfd / 2, lin.H, rtol=0, atol=1e-5 * np.abs(lin.H).max())


def _twist(xi):
    w, v = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


def test_H_symmetric_psd(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case()
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    for Tx in (T, _perturbed(T, 1), np.eye(4)):
        lin = oracle_lib.linearize(vm, sp, sc, Tx)
        nrm = np.linalg.norm(lin.H)
        assert np.abs(lin.H - lin.H.T).max() <= 1e-12 * nrm
        assert np.linalg.eigvalsh(lin.H).min() >= -1e-12 * nrm
        assert lin.err >= 0


def test_exact_gradient_matches_finite_differences(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case(800, 600)
    T = _perturbed(T, 2)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    g = oracle_lib.exact_gradient(vm, sp, sc, T, lin.corr)
    h = 1e-6
    gfd = np.zeros(6)
    for i in range(6):
        xi = np.zeros(6)
        xi[i] = h
        gfd[i] = (oracle_lib.cost_fixed(vm, sp, sc, T @ se3.se3_exp(xi), lin.corr)
                  - oracle_lib.cost_fixed(vm, sp, sc, T @ se3.se3_exp(-xi), lin.corr)) / (2 * h)
    np.testing.assert_allclose(g, gfd, rtol=0, atol=1e-6 * np.linalg.norm(g) + 1e-6)
    # the translational part has no W term; the rotational part differs from 2b
    np.testing.assert_allclose(g[3:], 2 * lin.b[3:], rtol=1e-10, atol=1e-9)
    assert np.linalg.norm(g[:3] - 2 * lin.b[:3]) > 1e-6 * np.linalg.norm(g)


def test_invariance_reframing_source(oracle_lib):
    """Source re-expressed by a rigid G (mu -> G mu, C -> R_G C R_G^T, T -> T G^-1):
    xi' = Ad_G xi, so H' = Ad_G^-T H Ad_G^-1, b' = Ad_G^-T b, err and the
    correspondences unchanged.  G is a 90-degree rotation with a dyadic translation
    so that float32 inputs transform exactly."""
    tp, tc, sp, sc, T, r = _room_case(1000, 800, dyadic=True)
    T = _perturbed(T, 3)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    G = np.eye(4)
    G[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    G[:3, 3] = [0.75, -1.25, 0.5]
    sp2 = (sp.astype(np.float64) @ G[:3, :3].T + G[:3, 3]).astype(np.float32)
    assert np.array_equal(sp2.astype(np.float64), sp.astype(np.float64) @ G[:3, :3].T + G[:3, 3])
    R = G[:3, :3]
    sc2 = np.array([_upper(R @ _sym(c) @ R.T) for c in sc.astype(np.float64)], dtype=np.float32)
    T2 = T @ se3.inverse(G)
    a = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    bb = oracle_lib.linearize(vm, sp2, sc2, T2, debug=True)
    assert np.array_equal(a.corr, bb.corr)
    np.testing.assert_allclose(bb.err, a.err, rtol=1e-12)
    Ai = np.linalg.inv(se3.adjoint(G))
    np.testing.assert_allclose(bb.H, Ai.T @ a.H @ Ai, rtol=0, atol=1e-10 * np.abs(a.H).max())
    np.testing.assert_allclose(bb.b, Ai.T @ a.b, rtol=0, atol=1e-10 * np.abs(a.H).max())


def test_invariance_reframing_source_general_rotation(oracle_lib):
    """Same relation for a general rotation; float32 rounding of G mu limits it to
    ~1e-6 relative."""
    tp, tc, sp, sc, T, r = _room_case(1000, 800)
    T = _perturbed(T, 5)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    G = synth.make_pose(synth.axis_angle_matrix([0.3, -0.5, 0.8], 0.7), [1.0, -2.0, 0.3])
    sp2 = (sp.astype(np.float64) @ G[:3, :3].T + G[:3, 3]).astype(np.float32)
    R = G[:3, :3]
    sc2 = np.array([_upper(R @ _sym(c) @ R.T) for c in sc.astype(np.float64)], dtype=np.float32)
    a = oracle_lib.linearize(vm, sp, sc, T, debug=True)
    bb = oracle_lib.linearize(vm, sp2, sc2, T @ se3.inverse(G), debug=True)
    same = a.corr == bb.corr
    assert same.mean() > 0.999
    Ai = np.linalg.inv(se3.adjoint(G))
    np.testing.assert_allclose(bb.H, Ai.T @ a.H @ Ai, rtol=0, atol=2e-5 * np.abs(a.H).max())
    np.testing.assert_allclose(bb.err, a.err, rtol=1e-3)


def _upper(S):
    return [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]


def test_invariance_grid_translation(oracle_lib):
    """Shifting the target and the pose translation by r * Z^3 shifts every key by
    the same integer vector and leaves err, H and b unchanged."""
    tp, tc, sp, sc, T, r = _room_case(1000, 800, dyadic=True)
    T = _perturbed(T, 6)
    s = np.array([3.0, -2.0, 5.0]) * r
    tp2 = (tp.astype(np.float64) + s).astype(np.float32)
    assert np.array_equal(tp2.astype(np.float64), tp.astype(np.float64) + s)
    T2 = T.copy()
    T2[:3, 3] += s
    a = oracle_lib.linearize(oracle_lib.build_voxelmap(tp, tc, r), sp, sc, T, debug=True)
    q = sp.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    assert _min_face_distance(q, r) > 1e-9
    bb = oracle_lib.linearize(oracle_lib.build_voxelmap(tp2, tc, r), sp, sc, T2, debug=True)
    np.testing.assert_array_equal(bb.qkeys, a.qkeys + (s / r).astype(np.int64))
    np.testing.assert_array_equal(bb.corr, a.corr)
    np.testing.assert_allclose(bb.err, a.err, rtol=1e-12)
    np.testing.assert_allclose(bb.H, a.H, rtol=0, atol=1e-12 * np.abs(a.H).max())
    np.testing.assert_allclose(bb.b, a.b, rtol=0, atol=1e-12 * np.abs(a.H).max())


@pytest.mark.parametrize("Q", [
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
    [[1, 0, 0], [0, 0, -1], [0, 1, 0]],
    [[-1, 0, 0], [0, -1, 0], [0, 0, 1]],
])
def test_invariance_grid_rotation(oracle_lib, Q):
    """A 90-degree rotation Q of the target maps the voxel grid onto itself; with
    the pose conjugated to Q T the source-side perturbation sees identical terms:
    err, H and b unchanged and the inlier set the same."""
    Q = np.array(Q, dtype=np.float64)
    tp, tc, sp, sc, T, r = _room_case(1000, 800, dyadic=True)
    T = _perturbed(T, 7)
    tp2 = (tp.astype(np.float64) @ Q.T).astype(np.float32)
    tc2 = np.array([_upper(Q @ _sym(c) @ Q.T) for c in tc.astype(np.float64)], dtype=np.float32)
    Q4 = np.eye(4)
    Q4[:3, :3] = Q
    q = sp.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    assert _min_face_distance(q, r) > 1e-9
    assert _min_face_distance(tp.astype(np.float64), r) > 1e-9
    a = oracle_lib.linearize(oracle_lib.build_voxelmap(tp, tc, r), sp, sc, T, debug=True)
    bb = oracle_lib.linearize(oracle_lib.build_voxelmap(tp2, tc2, r), sp, sc, Q4 @ T, debug=True)
    np.testing.assert_array_equal(bb.corr >= 0, a.corr >= 0)
    np.testing.assert_allclose(bb.err, a.err, rtol=1e-12)
    np.testing.assert_allclose(bb.H, a.H, rtol=0, atol=1e-12 * np.abs(a.H).max())
    np.testing.assert_allclose(bb.b, a.b, rtol=0, atol=1e-12 * np.abs(a.H).max())


def test_gauss_newton_recovers_planted_pose(oracle_lib):
    """Room scene, planted 5 deg / 0.2 m, start at identity (Sec. III-A factor,
    relinearised every iteration)."""
    tp, tc, sp, sc, T_true, r = _room_case(4096, 4096, seed=1)
    vm = oracle_lib.build_voxelmap(tp, tc, r)

    def lin(T):
        x = oracle_lib.linearize(vm, sp, sc, T)
        return x.H, x.b, x.err

    T, hist = se3.gauss_newton(lin, np.eye(4), max_iters=40, tol=1e-9)
    rot_err, trans_err = se3.pose_error(T, T_true)
    assert rot_err < 0.1 and trans_err < 0.01, (rot_err, trans_err, hist[-3:])
    assert hist[-1][0] < hist[0][0]


def test_27_neighbour_matches_bruteforce(oracle_lib):
    """27-neighbour mode = sum of independent single-voxel terms over every
    occupied voxel whose key differs by at most 1 per axis (linear scan)."""
    rng = np.random.default_rng(8)
    r = 0.5
    centers = rng.uniform(-1.5, 1.5, size=(6, 3))
    tp = (centers[rng.integers(0, 6, 160)] + rng.normal(scale=0.4, size=(160, 3))).astype(np.float32)
    tc = oracle_lib.knn_covariances(tp).astype(np.float32)
    sp = (tp[rng.integers(0, 160, 40)] + rng.normal(scale=0.2, size=(40, 3))).astype(np.float32)
    sc = oracle_lib.knn_covariances(sp).astype(np.float32)
    T = synth.make_pose(synth.axis_angle_matrix([0, 0, 1], 0.05), [0.03, 0.02, -0.01])
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    lin27 = oracle_lib.linearize(vm, sp, sc, T, neighbours=27, debug=True)
    H = np.zeros((6, 6)); b = np.zeros(6); e = 0.0; cnt = 0
    for i in range(sp.shape[0]):
        qk = lin27.qkeys[i]
        for v in range(vm.num_voxels):
            if np.abs(vm.keys[v] - qk).max() <= 1:
                one = oracle_lib.VoxelMap(qk[None].copy(), vm.counts[v:v + 1], vm.means[v:v + 1],
                                          vm.covs[v:v + 1], r)
                # place the single voxel at the point's own key so the 1-mode lookup hits
                x = oracle_lib.linearize(one, sp[i:i + 1], sc[i:i + 1], T)
                assert x.inliers == 1
                H += x.H; b += x.b; e += x.err; cnt += 1
    assert lin27.inliers == cnt and cnt > sp.shape[0]
    np.testing.assert_allclose(lin27.H, H, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    np.testing.assert_allclose(lin27.b, b, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    np.testing.assert_allclose(lin27.err, e, rtol=1e-12)


def test_nthreads_do_not_change_result(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case(3000, 9000)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    a = oracle_lib.linearize(vm, sp, sc, T, nthreads=1)
    b = oracle_lib.linearize(vm, sp, sc, T, nthreads=4)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.b, b.b) and a.err == b.err


def test_empty_and_all_miss(oracle_lib):
    tp, tc, sp, sc, T, r = _room_case(300, 300)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    e = oracle_lib.linearize(vm, sp[:0], sc[:0], T)
    assert e.inliers == 0 and e.err == 0 and not e.H.any() and not e.b.any()
    far = T.copy()
    far[:3, 3] += 1000.0
    m = oracle_lib.linearize(vm, sp, sc, far)
    assert m.inliers == 0 and m.err == 0 and not m.H.any()


def test_overlap_rate_pins(oracle_lib):
    """Overlap rate (Sec. III-D): a cloud against its own map at the identity is
    1 (every point lies in its own voxel); far away it is 0; in general it is the
    brute-force fraction of transformed points whose key is a map key."""
    import oracle
    rng = np.random.default_rng(8)
    pts = (rng.random((500, 3)) * 4.0 - 2.0).astype(np.float32)
    covs = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (500, 1))
    vm = oracle.build_voxelmap(pts, covs, 0.5)
    assert oracle.overlap(vm, pts, np.eye(4)) == 1.0
    far = np.eye(4)
    far[:3, 3] = 100.0
    assert oracle.overlap(vm, pts, far) == 0.0
    src = (rng.random((300, 3)) * 6.0 - 3.0).astype(np.float32)
    T = np.eye(4)
    T[:3, 3] = [0.3, -0.2, 0.1]
    q = src.astype(np.float64) + T[:3, 3]
    keys = {tuple(k) for k in np.floor(q / 0.5).astype(np.int64)}
    mk = {tuple(k) for k in vm.keys}
    hits = sum(tuple(k) in mk for k in np.floor(q / 0.5).astype(np.int64))
    assert len(keys) > 1
    assert oracle.overlap(vm, src, T) == hits / 300


def test_27_neighbour_reduces_to_one_voxel_when_voxels_are_isolated(oracle_lib):
    """With occupied voxels at least two keys apart on some axis, the 3 x 3 x 3
    block of a point in an occupied voxel holds that voxel alone: the
    27-neighbour factor is the 1-neighbour factor."""
    rng = np.random.default_rng(21)
    r = 0.5
    lattice = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(2), indexing="ij"),
                       -1).reshape(-1, 3) * 3  # voxel keys three apart
    keys = lattice[rng.integers(0, len(lattice), 400)]
    tp = ((keys + rng.uniform(0.1, 0.9, size=(400, 3))) * r).astype(np.float32)
    tc = oracle_lib.knn_covariances(tp).astype(np.float32)
    src_keys = lattice[rng.integers(0, len(lattice), 150)]
    sp = ((src_keys + rng.uniform(0.2, 0.8, size=(150, 3))) * r).astype(np.float32)
    sc = oracle_lib.knn_covariances(sp).astype(np.float32)
    T = synth.make_pose(synth.axis_angle_matrix([0, 1, 0], 0.01), [0.01, -0.01, 0.005])
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    one = oracle_lib.linearize(vm, sp, sc, T, neighbours=1)
    many = oracle_lib.linearize(vm, sp, sc, T, neighbours=27)
    assert one.inliers == many.inliers == sp.shape[0]
    np.testing.assert_allclose(many.H, one.H, rtol=1e-14, atol=1e-14 * np.abs(one.H).max())
    np.testing.assert_allclose(many.b, one.b, rtol=1e-14, atol=1e-14 * np.abs(one.H).max())
    np.testing.assert_allclose(many.err, one.err, rtol=1e-14)


def test_factor_is_a_sum_over_source_points(oracle_lib):
    """Eq. 2 sums per-point terms: the factor of a source cloud is the sum of the
    factors of any split of it (a dropped or doubled point fails this)."""
    tp, tc, sp, sc, T, r = _room_case(2000, 3000, seed=5)
    vm = oracle_lib.build_voxelmap(tp, tc, r)
    Tp = _perturbed(T, seed=3)
    whole = oracle_lib.linearize(vm, sp, sc, Tp)
    mask = np.random.default_rng(4).random(sp.shape[0]) < 0.4
    a = oracle_lib.linearize(vm, sp[mask], sc[mask], Tp)
    b = oracle_lib.linearize(vm, sp[~mask], sc[~mask], Tp)
    assert whole.inliers == a.inliers + b.inliers and 0 < a.inliers < whole.inliers
    scale = np.abs(whole.H).max()
    np.testing.assert_allclose(whole.H, a.H + b.H, rtol=1e-12, atol=1e-12 * scale)
    np.testing.assert_allclose(whole.b, a.b + b.b, rtol=1e-12, atol=1e-12 * scale)
    np.testing.assert_allclose(whole.err, a.err + b.err, rtol=1e-12)
