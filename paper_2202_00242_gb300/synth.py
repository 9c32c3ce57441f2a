"""Seeded synthetic workloads: surface point clouds, sensor poses and factor pairs.

This module draws inputs only.  It samples planar and cylindrical surfaces,
adds Gaussian noise, expresses the samples in sensor frames by rigid
transforms, and draws pose perturbations.  It contains none of the VGICP
arithmetic (voxelisation, the distribution-to-distribution cost, its
derivatives): the GPU library and the FP64 reference both read the arrays it
returns.  The scenes stand in for the LiDAR datasets of arXiv 2202.00242
Sec. IV (Newer College, KAIST urban), which are not available here.

All random draws come from ``numpy.random.default_rng(seed)`` (PCG64), so a
seed gives the same arrays on every host.

``surface_covariances`` gives each point the covariance I - (1 - eps) n n^T
for its true surface normal n, i.e. eigenvalues (1, 1, eps) with the small one
along the normal: the same eigen-structure the k-NN covariance of Sec. III-C
ends with after regularisation, available without a neighbour search for the
large benchmark clouds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# rigid-transform utilities for input synthesis
# ---------------------------------------------------------------------------

def axis_angle_matrix(axis, angle):
    """Rotation by ``angle`` radians about unit ``axis`` (Rodrigues)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def make_pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def pose_inverse(T):
    Ti = np.eye(4)
    Ti[:3, :3] = T[:3, :3].T
    Ti[:3, 3] = -T[:3, :3].T @ T[:3, 3]
    return Ti


def planted_pose(rng, rot_deg, trans_m):
    """Rotation of exactly ``rot_deg`` about a random axis, translation of length
    ``trans_m`` in a random direction."""
    return make_pose(axis_angle_matrix(random_unit(rng), np.radians(rot_deg)),
                     trans_m * random_unit(rng))


def perturb_pose(rng, T, sigma_t, sigma_deg):
    """T @ dT with dT's rotation vector ~ N(0, sigma_deg^2) per axis (degrees) and
    translation ~ N(0, sigma_t^2) per axis."""
    w = np.radians(sigma_deg) * rng.normal(size=3)
    th = np.linalg.norm(w)
    R = np.eye(3) if th == 0 else axis_angle_matrix(w / th, th)
    return T @ make_pose(R, sigma_t * rng.normal(size=3))


def to_frame(points, normals, T_world_frame):
    """Express world points/normals in the frame whose world pose is T."""
    R, t = T_world_frame[:3, :3], T_world_frame[:3, 3]
    return (points - t) @ R, normals @ R


def surface_covariances(normals, eps=1e-3):
    """(n, 6) float32 upper triangles of I - (1 - eps) n n^T."""
    s = 1.0 - eps
    out = np.empty((len(normals), 6), dtype=np.float32)
    for a in range(0, len(normals), 1 << 22):  # bounded float64 temporaries
        n = np.asarray(normals[a:a + (1 << 22)], dtype=np.float64)
        o = out[a:a + (1 << 22)]
        o[:, 0] = 1.0 - s * n[:, 0] * n[:, 0]
        o[:, 1] = -s * n[:, 0] * n[:, 1]
        o[:, 2] = -s * n[:, 0] * n[:, 2]
        o[:, 3] = 1.0 - s * n[:, 1] * n[:, 1]
        o[:, 4] = -s * n[:, 1] * n[:, 2]
        o[:, 5] = 1.0 - s * n[:, 2] * n[:, 2]
    return out


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------

def sample_room(rng, n, size=(10.0, 10.0, 3.0), sigma=0.01, origin=(0.0, 0.0, 0.0)):
    """n points uniform by area on the six faces of an axis-aligned box with one
    corner at ``origin``, plus isotropic Gaussian noise.  Returns (points, normals)."""
    L = np.asarray(size, dtype=np.float64)
    o = np.asarray(origin, dtype=np.float64)
    areas = np.array([L[1] * L[2], L[1] * L[2], L[0] * L[2], L[0] * L[2], L[0] * L[1], L[0] * L[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    u = rng.random((n, 3)) * L
    axis = face // 2
    side = face % 2
    u[np.arange(n), axis] = side * L[axis]
    normals = np.zeros((n, 3))
    normals[np.arange(n), axis] = np.where(side == 0, 1.0, -1.0)
    pts = o + u + sigma * rng.normal(size=(n, 3))
    return pts, normals


@dataclass
class Walls:
    """Vertical rectangles: 2-D segment (x0, y0)-(x1, y1), z from z0 to z1."""
    seg: np.ndarray   # (m, 4)
    z: np.ndarray     # (m, 2)

    def area(self):
        return np.hypot(self.seg[:, 2] - self.seg[:, 0], self.seg[:, 3] - self.seg[:, 1]) * (
            self.z[:, 1] - self.z[:, 0])

    def distance_xy(self, c):
        p0, p1 = self.seg[:, :2], self.seg[:, 2:]
        d = p1 - p0
        L2 = np.maximum((d * d).sum(1), 1e-12)
        s = np.clip(((c[None, :2] - p0) * d).sum(1) / L2, 0.0, 1.0)
        return np.linalg.norm(p0 + s[:, None] * d - c[None, :2], axis=1)


def _sample_walls(rng, walls: Walls, idx, n):
    if len(idx) == 0 or n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3))
    a = walls.area()[idx]
    w = idx[rng.choice(len(idx), size=n, p=a / a.sum())]
    s = rng.random(n)
    seg = walls.seg[w]
    xy = seg[:, :2] + s[:, None] * (seg[:, 2:] - seg[:, :2])
    z = walls.z[w, 0] + rng.random(n) * (walls.z[w, 1] - walls.z[w, 0])
    d = seg[:, 2:] - seg[:, :2]
    nrm = np.stack([-d[:, 1], d[:, 0], np.zeros(n)], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return np.column_stack([xy, z]), nrm


def _sample_disk(rng, n, c, radius, z):
    r = radius * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    p = np.column_stack([c[0] + r * np.cos(th), c[1] + r * np.sin(th), np.full(n, z)])
    nrm = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    return p, nrm


def sample_scan(rng, walls: Walls, center, n, radius, sigma, ground_frac=0.35,
                ground_z=0.0, cylinders=None):
    """n noisy points within ``radius`` of ``center`` on the ground disk, the walls
    and optional vertical cylinders (cx, cy, r, h)."""
    center = np.asarray(center, dtype=np.float64)
    n_ground = int(round(ground_frac * n))
    pts = []
    nrm = []
    if n_ground:
        p, q = _sample_disk(rng, n_ground, center, radius, ground_z)
        pts.append(p)
        nrm.append(q)
    n_rest = n - n_ground
    near = np.nonzero(walls.distance_xy(center) < radius)[0]
    n_cyl = 0
    if cylinders is not None and len(cylinders):
        dc = np.hypot(cylinders[:, 0] - center[0], cylinders[:, 1] - center[1])
        cyl = cylinders[dc < radius]
        if len(cyl):
            n_cyl = n_rest // 5
            k = rng.integers(0, len(cyl), size=n_cyl)
            th = 2 * np.pi * rng.random(n_cyl)
            c = cyl[k]
            pc = np.column_stack([c[:, 0] + c[:, 2] * np.cos(th), c[:, 1] + c[:, 2] * np.sin(th),
                                  ground_z + rng.random(n_cyl) * c[:, 3]])
            pts.append(pc)
            nrm.append(np.column_stack([np.cos(th), np.sin(th), np.zeros(n_cyl)]))
    need = n_rest - n_cyl
    got_p, got_n = [], []
    have = 0
    while need > 0 and have < need and len(near):
        p, q = _sample_walls(rng, walls, near, 2 * (need - have) + 64)
        keep = np.linalg.norm(p - center[None, :], axis=1) < radius
        got_p.append(p[keep])
        got_n.append(q[keep])
        have += int(keep.sum())
    if need > 0:
        if got_p:
            pts.append(np.concatenate(got_p)[:need])
            nrm.append(np.concatenate(got_n)[:need])
        else:  # nothing vertical nearby: fall back to ground
            p, q = _sample_disk(rng, need, center, radius, ground_z)
            pts.append(p)
            nrm.append(q)
    P = np.concatenate(pts)
    N = np.concatenate(nrm)
    perm = rng.permutation(P.shape[0])
    return P[perm] + sigma * rng.normal(size=P.shape), N[perm]


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclass
class Clouds:
    """Several clouds concatenated: cloud c is rows offsets[c]:offsets[c+1]."""
    points: np.ndarray          # (N, 3) float32
    normals: np.ndarray         # (N, 3) float32 (true surface normals, for covariances)
    offsets: np.ndarray         # (C + 1,) int64
    covs: np.ndarray | None = None  # (N, 6) float32

    def cloud(self, c):
        a, b = self.offsets[c], self.offsets[c + 1]
        return self.points[a:b], (None if self.covs is None else self.covs[a:b])

    @property
    def sizes(self):
        return np.diff(self.offsets)


@dataclass
class Workload:
    name: str
    resolution: float
    clouds: Clouds
    pairs: np.ndarray           # (P, 2) int32 (target cloud, source cloud)
    poses: np.ndarray           # (P, 4, 4) float64 T_target_source to linearise at
    true_poses: np.ndarray      # (P, 4, 4) float64 ground-truth T_target_source
    world_poses: np.ndarray     # (C, 4, 4) float64
    meta: dict = field(default_factory=dict)

    @property
    def source_points_per_step(self) -> int:
        return int(self.clouds.sizes[self.pairs[:, 1]].sum())


def _pack(clouds_pts, clouds_nrm):
    sizes = np.array([p.shape[0] for p in clouds_pts], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return Clouds(np.concatenate(clouds_pts).astype(np.float32),
                  np.concatenate(clouds_nrm).astype(np.float32), offsets)


def room_pair(seed=1, n_target=8192, n_source=8192, rot_deg=5.0, trans_m=0.2, sigma=0.01,
              resolution=0.5):
    """Single factor: a 10 x 10 x 3 m room (all six faces, uniform by area,
    noise sigma), target and source sampled independently, the source expressed in
    a frame displaced by a planted pose (rotation ``rot_deg`` about a random axis,
    translation ``trans_m``).  Cloud 0 = target (room frame), cloud 1 = source.
    ``poses[0]`` is the identity (the initial guess); ``true_poses[0]`` is the
    planted T_target_source."""
    rng = np.random.default_rng(seed)
    origin = -np.array([5.0, 5.0, 1.5]) + rng.uniform(-0.2, 0.2, size=3)
    tgt, tn = sample_room(rng, n_target, sigma=sigma, origin=origin)
    src_w, sn_w = sample_room(rng, n_source, sigma=sigma, origin=origin)
    T_true = planted_pose(rng, rot_deg, trans_m)
    src, sn = to_frame(src_w, sn_w, T_true)
    clouds = _pack([tgt, src], [tn, sn])
    return Workload("room_single_factor", resolution, clouds, np.array([[0, 1]], dtype=np.int32),
                    np.eye(4)[None].copy(), T_true[None].copy(),
                    np.stack([np.eye(4), T_true]), {"seed": seed, "sigma": sigma})


def corridor_window(seed=2, n=20000, n_keyframes=10, step_m=0.5, step_deg=3.0, sigma=0.02,
                    resolution=0.25, scan_radius=20.0, n_cylinders=40, perturb=(0.0, 0.0)):
    """Frontend window: one scan against ``n_keyframes`` keyframes in a corridor
    of planes (floor, ceiling, two walls) with random vertical cylinders.
    Consecutive sensor poses are ``step_m`` and ``step_deg`` apart.  Clouds
    0..K-1 are the keyframes, cloud K the latest scan; pair k = (k, K)."""
    rng = np.random.default_rng(seed)
    length, half_w, height = 200.0, 2.5, 3.0
    walls = Walls(np.array([[-length, -half_w, length, -half_w], [length, half_w, -length, half_w]]),
                  np.array([[0.0, height], [0.0, height]]))
    cyl = np.column_stack([rng.uniform(-20, 40, n_cylinders), rng.uniform(-1.8, 1.8, n_cylinders),
                           rng.uniform(0.1, 0.3, n_cylinders), np.full(n_cylinders, height)])
    K = n_keyframes
    world = []
    R = np.eye(3)
    for i in range(K + 1):
        if i:
            R = R @ axis_angle_matrix(random_unit(rng), np.radians(step_deg))
            # keep the heading along the corridor: pull the rotation back towards
            # identity while preserving the per-step angle magnitude approximately
        world.append(make_pose(R, np.array([step_m * i, 0.0, 1.2])))
    pts, nrm = [], []
    for i in range(K + 1):
        c = world[i][:3, 3]
        p, q = sample_scan(rng, walls, c, n, scan_radius, sigma, ground_frac=0.3,
                           cylinders=cyl)
        # ceiling: replace a share of the ground points by ceiling points
        m = p[:, 2] < 0.5 * height
        flip = m & (rng.random(p.shape[0]) < 0.4)
        flip &= np.abs(q[:, 2]) > 0.9
        p[flip, 2] = height + sigma * rng.normal(size=int(flip.sum()))
        q[flip] = np.array([0.0, 0.0, -1.0])
        pl, ql = to_frame(p, q, world[i])
        pts.append(pl)
        nrm.append(ql)
    clouds = _pack(pts, nrm)
    pairs = np.array([[k, K] for k in range(K)], dtype=np.int32)
    true = np.stack([pose_inverse(world[k]) @ world[K] for k in range(K)])
    poses = np.stack([perturb_pose(rng, T, perturb[0], perturb[1]) for T in true])
    return Workload("corridor_window", resolution, clouds, pairs, poses, true, np.stack(world),
                    {"seed": seed, "sigma": sigma})


def _loop_path(n, lap_len, laps, lateral):
    """n poses spread over ``laps`` laps of a rounded-rectangle loop of perimeter
    ``lap_len``; lap k is shifted sideways by k * lateral."""
    a = lap_len / 6.0  # rectangle 2a x a
    b = a / 2.0
    s = np.linspace(0.0, laps * lap_len, n, endpoint=False)
    lap = np.floor(s / lap_len)
    u = s - lap * lap_len
    per = 2 * (2 * a + 2 * b)
    u = u / lap_len * per
    x = np.empty(n)
    y = np.empty(n)
    hd = np.empty(n)
    e1, e2, e3 = 2 * a, 2 * a + 2 * b, 4 * a + 2 * b
    for i, ui in enumerate(u):
        if ui < e1:
            x[i], y[i], hd[i] = -a + ui, -b, 0.0
        elif ui < e2:
            x[i], y[i], hd[i] = a, -b + (ui - e1), np.pi / 2
        elif ui < e3:
            x[i], y[i], hd[i] = a - (ui - e2), b, np.pi
        else:
            x[i], y[i], hd[i] = -a, b - (ui - e3), 3 * np.pi / 2
    # lateral shift for later laps (towards the inside of the loop)
    x -= lateral * lap * np.sign(x)
    y -= lateral * lap * np.sign(y)
    return x, y, hd


def outdoor_submaps(seed=3, n_submaps=500, n_min=30000, n_max=80000, neighbours=10,
                    sigma=0.03, perturb=(0.1, 1.0), resolution=1.0, radius=40.0, spacing=6.0,
                    laps=2, size_dist="loguniform"):
    """Global-map workload: ``n_submaps`` submaps along two laps of a city loop with
    box buildings (planes) on both sides, point counts log-uniform (or uniform)
    in [n_min, n_max], each submap in its own frame.  Every submap is the source
    of ``neighbours`` factors whose targets are its nearest other submaps, so
    there are n_submaps * neighbours pairs.  ``poses`` are the true relative poses
    perturbed by ``perturb`` = (sigma_t [m], sigma_rot [deg])."""
    rng = np.random.default_rng(seed)
    lap_len = max(n_submaps * spacing / laps, 150.0)
    x, y, hd = _loop_path(n_submaps, lap_len, laps, lateral=3.0)
    # buildings along the first lap's path, both sides
    segs, zs = [], []
    xs, ys, hs = _loop_path(int(lap_len / 20.0), lap_len, 1, 0.0)
    for px, py, ph in zip(xs, ys, hs):
        for side in (-1.0, 1.0):
            if rng.random() < 0.15:
                continue
            off = rng.uniform(12.0, 20.0)
            w, d, h = rng.uniform(8.0, 18.0), rng.uniform(8.0, 18.0), rng.uniform(6.0, 30.0)
            c = np.array([px, py]) + side * off * np.array([-np.sin(ph), np.cos(ph)])
            ex = np.array([np.cos(ph), np.sin(ph)])
            ey = np.array([-np.sin(ph), np.cos(ph)])
            corners = [c + sx * w / 2 * ex + sy * d / 2 * ey
                       for sx, sy in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
            for k in range(4):
                p0, p1 = corners[k], corners[(k + 1) % 4]
                segs.append([p0[0], p0[1], p1[0], p1[1]])
                zs.append([0.0, h])
    walls = Walls(np.array(segs, dtype=np.float64).reshape(-1, 4),
                  np.array(zs, dtype=np.float64).reshape(-1, 2))
    if size_dist == "loguniform":
        sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_submaps)).astype(np.int64)
    else:
        sizes = rng.integers(n_min, n_max + 1, n_submaps).astype(np.int64)
    world = []
    pts, nrm = [], []
    for i in range(n_submaps):
        tilt = axis_angle_matrix(random_unit(rng), np.radians(rng.uniform(0.0, 2.0)))
        Rw = axis_angle_matrix([0.0, 0.0, 1.0], hd[i] + rng.uniform(-0.2, 0.2)) @ tilt
        Tw = make_pose(Rw, np.array([x[i], y[i], 1.8]))
        world.append(Tw)
        p, q = sample_scan(rng, walls, np.array([x[i], y[i], 1.8]), int(sizes[i]), radius, sigma)
        pl, ql = to_frame(p, q, Tw)
        pts.append(pl.astype(np.float32))  # the packed clouds are float32 anyway
        nrm.append(ql.astype(np.float32))
    clouds = _pack(pts, nrm)
    centers = np.column_stack([x, y])
    pairs = []
    for i in range(n_submaps):
        dist = np.linalg.norm(centers - centers[i], axis=1)
        dist[i] = np.inf
        for j in np.argsort(dist, kind="stable")[:neighbours]:
            pairs.append([int(j), i])
    pairs = np.array(pairs, dtype=np.int32)
    true = np.stack([pose_inverse(world[j]) @ world[i] for j, i in pairs])
    poses = np.stack([perturb_pose(rng, T, perturb[0], perturb[1]) for T in true])
    return Workload("outdoor_submaps", resolution, clouds, pairs, poses, true, np.stack(world),
                    {"seed": seed, "sigma": sigma, "n_submaps": n_submaps,
                     "neighbours": neighbours, "size_range": [n_min, n_max],
                     "size_dist": size_dist})


def with_surface_covariances(w: Workload, eps=1e-3) -> Workload:
    w.clouds.covs = surface_covariances(w.clouds.normals, eps)
    return w


# Named configurations (the five workloads the library is measured on).

def config_room(seed=1, **kw):
    """Single factor, room 10 x 10 x 3 m, 8,192 + 8,192 points, res 0.5 m."""
    return room_pair(seed=seed, **kw)


def config_corridor(seed=2, resolution=0.25, **kw):
    """1 scan vs 10 keyframes of 20,000 points, corridor, res 0.25 or 1.0 m."""
    return corridor_window(seed=seed, resolution=resolution, **kw)


def config_global_map(seed=3, **kw):
    """500 submaps (30k-80k log-uniform), 5,000 pairs, res 1.0 m."""
    return outdoor_submaps(seed=seed, **kw)


def config_differentiable(seed=4, **kw):
    """256 pairs of 20k-50k point submaps, perturbation 0.3 m / 5 deg."""
    args = dict(n_submaps=64, n_min=20000, n_max=50000, neighbours=4, perturb=(0.3, 5.0),
                size_dist="uniform", resolution=1.0)
    args.update(kw)
    return outdoor_submaps(seed=seed, **args)


def config_large_map(seed=5, **kw):
    """2,000 submaps x 100k points, 40,000 pairs, res 0.5 m (27-neighbour mode)."""
    args = dict(n_submaps=2000, n_min=100000, n_max=100000, neighbours=20, resolution=0.5,
                size_dist="uniform", spacing=3.0)
    args.update(kw)
    return outdoor_submaps(seed=seed, **args)
