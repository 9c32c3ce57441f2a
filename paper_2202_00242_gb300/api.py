"""Python API over the C ABI (include/vgicp.h).  PyTorch provides device memory
and streams; every step of the computation runs in the library's CUDA kernels.

Layouts: clouds are float32 CUDA tensors, points (n, 3) and covariances (n, 6)
upper triangles (xx, xy, xz, yy, yz, zz); poses are float64 host arrays (4, 4)
T_target_source.  A factor result is 43 float64 values: H (36), b (6), err (1),
see ``unpack``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import Cloud, LinOpts, MapOpts, check

RESULT_SIZE = 43


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_cloud(points: torch.Tensor, covs: torch.Tensor, what="cloud"):
    if not (points.is_cuda and covs.is_cuda):
        raise ValueError(f"{what}: tensors must be on a CUDA device")
    if points.dtype != torch.float32 or covs.dtype != torch.float32:
        raise ValueError(f"{what}: tensors must be float32")
    if points.dim() != 2 or points.shape[1] != 3 or covs.dim() != 2 or covs.shape[1] != 6:
        raise ValueError(f"{what}: expected points (n, 3) and covs (n, 6)")
    if points.shape[0] != covs.shape[0]:
        raise ValueError(f"{what}: points and covs differ in length")
    if not (points.is_contiguous() and covs.is_contiguous()):
        raise ValueError(f"{what}: tensors must be contiguous")


def _pose_array(T, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64))
    if n is None:
        if a.shape != (4, 4):
            raise ValueError("pose must be (4, 4)")
    elif a.shape != (n, 4, 4):
        raise ValueError(f"poses must be ({n}, 4, 4)")
    return a


def _map_opts(max_probe, capacity_factor):
    return MapOpts(int(max_probe), int(capacity_factor))


class VoxelMap:
    """Voxel map of a target cloud on the GPU (Sec. III-A of arXiv 2202.00242)."""

    def __init__(self, handle, resolution, n, refs):
        self._h = ctypes.c_void_p(handle)
        self.resolution = float(resolution)
        self.n = int(n)
        self._refs = refs  # inputs read by queued build kernels

    @property
    def handle(self):
        return self._h

    @staticmethod
    def build(points: torch.Tensor, covs: torch.Tensor, resolution: float, max_probe=0,
              capacity_factor=0, stream=None) -> "VoxelMap":
        _check_cloud(points, covs, "target")
        lib = _lib.load()
        h = ctypes.c_void_p()
        opts = _map_opts(max_probe, capacity_factor)
        check(lib.vgicp_build_voxelmap(ctypes.c_void_p(points.data_ptr()),
                                       ctypes.c_void_p(covs.data_ptr()), points.shape[0],
                                       float(resolution), ctypes.byref(opts), _stream_ptr(stream),
                                       ctypes.byref(h)))
        return VoxelMap(h.value, resolution, points.shape[0], [points, covs])

    def status(self, stream=None) -> int:
        """Synchronizes; raises VGICPError on a device-side build error."""
        return check(_lib.load().vgicp_voxelmap_status(self._h, _stream_ptr(stream)))

    def info(self, stream=None):
        V = ctypes.c_int64()
        cap = ctypes.c_int64()
        check(_lib.load().vgicp_voxelmap_info(self._h, _stream_ptr(stream), ctypes.byref(V),
                                              ctypes.byref(cap)))
        return int(V.value), int(cap.value)

    @property
    def num_voxels(self) -> int:
        return self.info()[0]

    def export(self, stream=None) -> dict:
        V, _ = self.info(stream)
        keys = np.zeros((max(V, 1), 3), np.int64)
        counts = np.zeros(max(V, 1), np.int32)
        means = np.zeros((max(V, 1), 3), np.float32)
        covs = np.zeros((max(V, 1), 6), np.float32)
        check(_lib.load().vgicp_voxelmap_export(
            self._h, _stream_ptr(stream), max(V, 1), keys.ctypes.data_as(ctypes.c_void_p),
            counts.ctypes.data_as(ctypes.c_void_p), means.ctypes.data_as(ctypes.c_void_p),
            covs.ctypes.data_as(ctypes.c_void_p)))
        return {"keys": keys[:V], "counts": counts[:V], "means": means[:V], "covs": covs[:V]}

    def grouped_cloud(self, stream=None):
        """The map's voxel-grouped cloud (points n x 3, covs n x 6, on the device)."""
        pts = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
        cov = torch.empty((self.n, 6), dtype=torch.float32, device="cuda")
        check(_lib.load().vgicp_voxelmap_grouped_cloud(
            self._h, _stream_ptr(stream), ctypes.c_void_p(pts.data_ptr()),
            ctypes.c_void_p(cov.data_ptr())))
        return pts, cov

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().vgicp_destroy_voxelmap(self._h)
        self._h = None
        self._refs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_voxelmaps(points: torch.Tensor, covs: torch.Tensor, offsets, resolution: float,
                    max_probe=0, capacity_factor=0, stream=None) -> list[VoxelMap]:
    """Build one map per cloud of a concatenation (rows offsets[m]:offsets[m+1])."""
    _check_cloud(points, covs, "targets")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_maps = off.shape[0] - 1
    if n_maps < 1 or off[0] != 0 or off[-1] != points.shape[0]:
        raise ValueError("offsets must start at 0 and end at the number of points")
    handles = (ctypes.c_void_p * n_maps)()
    opts = _map_opts(max_probe, capacity_factor)
    check(_lib.load().vgicp_build_voxelmaps(ctypes.c_void_p(points.data_ptr()),
                                            ctypes.c_void_p(covs.data_ptr()),
                                            off.ctypes.data_as(ctypes.c_void_p), n_maps,
                                            float(resolution), ctypes.byref(opts),
                                            _stream_ptr(stream), handles))
    refs = [points, covs]
    return [VoxelMap(handles[m], resolution, off[m + 1] - off[m], refs) for m in range(n_maps)]


def rebuild_voxelmaps(maps: list[VoxelMap], points: torch.Tensor, covs: torch.Tensor,
                      stream=None):
    """Refill a batch of maps (all handles of one build, in order) from new clouds of
    the same sizes; allocates nothing."""
    _check_cloud(points, covs, "targets")
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    check(_lib.load().vgicp_rebuild_voxelmaps(arr, len(maps), ctypes.c_void_p(points.data_ptr()),
                                              ctypes.c_void_p(covs.data_ptr()),
                                              _stream_ptr(stream)))
    for m in maps:
        m._refs = [points, covs]


@dataclass
class Linearization:
    out: torch.Tensor       # (43,) or (P, 43) float64, device
    inliers: torch.Tensor   # () or (P,) int64, device
    corr: torch.Tensor | None = None
    qkeys: torch.Tensor | None = None

    def unpack(self):
        return unpack(self.out)


def unpack(out):
    """Split (..., 43) results into H (..., 6, 6), b (..., 6), err (...)."""
    H = out[..., :36].reshape(*out.shape[:-1], 6, 6)
    return H, out[..., 36:42], out[..., 42]


def linearize(vmap: VoxelMap, points: torch.Tensor, covs: torch.Tensor, T, neighbours=1, tile=0,
              grid=0, corr=False, qkeys=False, out=None, inliers=None, variant=0,
              stream=None) -> Linearization:
    """Linearize one factor at T = T_target_source (Eqs. 2-3 of arXiv 2202.00242)."""
    _check_cloud(points, covs, "source")
    dev = points.device
    T = _pose_array(T)
    n = points.shape[0]
    if out is None:
        out = torch.empty(RESULT_SIZE, dtype=torch.float64, device=dev)
    if inliers is None:
        inliers = torch.empty((), dtype=torch.int64, device=dev)
    c = torch.empty(n, dtype=torch.int32, device=dev) if corr else None
    q = torch.empty((n, 3), dtype=torch.int32, device=dev) if qkeys else None
    opts = LinOpts(int(neighbours), int(tile), int(grid), int(variant),
                   ctypes.c_void_p(c.data_ptr()) if c is not None else None,
                   ctypes.c_void_p(q.data_ptr()) if q is not None else None, None, None)
    check(_lib.load().vgicp_linearize(vmap.handle, ctypes.c_void_p(points.data_ptr()),
                                      ctypes.c_void_p(covs.data_ptr()), n,
                                      T.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(inliers.data_ptr()), ctypes.byref(opts),
                                      _stream_ptr(stream)))
    return Linearization(out, inliers, c, q)


def make_clouds(sources) -> tuple:
    """ctypes array of vgicp_cloud from a list whose entries are (points, covs)
    tensors or VoxelMap objects (the map's own cloud, in voxel-grouped order)."""
    arr = (Cloud * len(sources))()
    for i, src in enumerate(sources):
        if isinstance(src, VoxelMap):
            arr[i] = Cloud(None, None, 0, src.handle.value)
        else:
            p, c = src
            _check_cloud(p, c, f"source {i}")
            arr[i] = Cloud(p.data_ptr(), c.data_ptr(), p.shape[0], None)
    return arr


def linearize_batched(maps: list[VoxelMap], sources, pairs, poses, neighbours=1, tile=0, grid=0,
                      out=None, inliers=None, variant=0, events=None,
                      stream=None) -> Linearization:
    """Linearize many factors in one persistent launch.  sources: list of (points,
    covs) or VoxelMap (its own cloud); pairs: (P, 2) int (map index, source
    index); poses: (P, 4, 4).  events: optional (start, stop) torch.cuda.Event
    recorded around the linearize kernel."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0]
    poses = _pose_array(poses, P)
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty((P, RESULT_SIZE), dtype=torch.float64, device=dev)
    if inliers is None:
        inliers = torch.empty(P, dtype=torch.int64, device=dev)
    clouds = make_clouds(sources)
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    ev0 = ctypes.c_void_p(events[0].cuda_event) if events is not None else None
    ev1 = ctypes.c_void_p(events[1].cuda_event) if events is not None else None
    opts = LinOpts(int(neighbours), int(tile), int(grid), int(variant), None, None, ev0, ev1)
    check(_lib.load().vgicp_linearize_batched(arr, len(maps), clouds, len(sources),
                                              pairs.ctypes.data_as(ctypes.c_void_p), P,
                                              poses.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(inliers.data_ptr()),
                                              ctypes.byref(opts), _stream_ptr(stream)))
    return Linearization(out, inliers)


class Plan:
    """A fixed factor set linearized repeatedly (one CUDA graph per iteration).

    maps, sources and pairs as in ``linearize_batched``; ``tile`` = points per
    work item (0: default), ``variant`` = 1-neighbour kernel (0: default).
    ``autotune(poses)`` times the kernel variants and item sizes and keeps the
    fastest; ``execute(poses)`` linearizes all factors.
    """

    def __init__(self, maps, sources, pairs, neighbours=1, tile=0, variant=0, grid=0,
                 stream=None):
        self._lib = _lib.load()
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.n_pairs = self.pairs.shape[0]
        self._refs = (list(maps), list(sources))
        clouds = make_clouds(sources)
        arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
        opts = LinOpts(int(neighbours), int(tile), int(grid), int(variant), None, None, None,
                       None)
        h = ctypes.c_void_p()
        check(self._lib.vgicp_plan_create(arr, len(maps), clouds, len(sources),
                                          self.pairs.ctypes.data_as(ctypes.c_void_p),
                                          self.n_pairs, ctypes.byref(opts), _stream_ptr(stream),
                                          ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    def autotune(self, poses, stream=None):
        poses = _pose_array(poses, self.n_pairs)
        check(self._lib.vgicp_plan_autotune(self._h, poses.ctypes.data_as(ctypes.c_void_p),
                                            _stream_ptr(stream)))
        return self.info()

    def execute(self, poses, out=None, inliers=None, events=None, stream=None) -> Linearization:
        poses = _pose_array(poses, self.n_pairs)
        if out is None:
            out = torch.empty((self.n_pairs, RESULT_SIZE), dtype=torch.float64, device=self.device)
        if inliers is None:
            inliers = torch.empty(self.n_pairs, dtype=torch.int64, device=self.device)
        ev0 = ctypes.c_void_p(events[0].cuda_event) if events is not None else None
        ev1 = ctypes.c_void_p(events[1].cuda_event) if events is not None else None
        check(self._lib.vgicp_plan_execute(self._h, poses.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(inliers.data_ptr()), ev0, ev1,
                                           _stream_ptr(stream)))
        return Linearization(out, inliers)

    def evaluate(self, base_poses: torch.Tensor, xi: torch.Tensor | None = None, mode=2,
                 grad_scale: torch.Tensor | None = None, out=None, inliers=None, stream=None):
        """Cost (mode 1) or gradient (2: W held, 3: exact) of every factor at
        T_p = base_p Exp(xi_p), composed on the device.  base_poses: CUDA float64
        (P, 4, 4); xi: CUDA float64 (P, 6) or None; grad_scale: CUDA float64 (P,)
        or None.  Returns (out (P, 7): gradient w.r.t. xi (6) and err, inliers)."""
        P = self.n_pairs
        for name, t, shape in (("base_poses", base_poses, (P, 4, 4)), ("xi", xi, (P, 6)),
                               ("grad_scale", grad_scale, (P,))):
            if t is None:
                continue
            if not t.is_cuda or t.dtype != torch.float64 or tuple(t.shape) != shape \
                    or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor {shape}")
        if out is None:
            out = torch.empty((P, 7), dtype=torch.float64, device=self.device)
        if inliers is None:
            inliers = torch.empty(P, dtype=torch.int64, device=self.device)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        check(self._lib.vgicp_plan_evaluate(self._h, ptr(base_poses), ptr(xi), int(mode),
                                            ptr(grad_scale), ptr(out), ptr(inliers),
                                            _stream_ptr(stream)))
        return out, inliers

    def info(self) -> dict:
        v, it, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        n = ctypes.c_int64()
        check(self._lib.vgicp_plan_info(self._h, ctypes.byref(v), ctypes.byref(it), ctypes.byref(g),
                                        ctypes.byref(n)))
        return {"variant": v.value, "item_points": it.value, "grid": g.value, "items": n.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vgicp_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# host binary64 pose algebra (library calls)
# ---------------------------------------------------------------------------

def se3_exp(xi) -> np.ndarray:
    """Exp(xi) for xi = [omega; v] (4x4, binary64)."""
    x = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(6))
    T = np.empty((4, 4))
    check(_lib.load().vgicp_se3_exp(x.ctypes.data_as(ctypes.c_void_p),
                                    T.ctypes.data_as(ctypes.c_void_p)))
    return T


def se3_right_jacobian(xi) -> np.ndarray:
    """J with Exp(xi + d) = Exp(xi) Exp(J d) + O(|d|^2) (6x6)."""
    x = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(6))
    J = np.empty((6, 6))
    check(_lib.load().vgicp_se3_right_jacobian(x.ctypes.data_as(ctypes.c_void_p),
                                               J.ctypes.data_as(ctypes.c_void_p)))
    return J


def pose_mul(A, B) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(4, 4))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(4, 4))
    C = np.empty((4, 4))
    check(_lib.load().vgicp_pose_mul(A.ctypes.data_as(ctypes.c_void_p),
                                     B.ctypes.data_as(ctypes.c_void_p),
                                     C.ctypes.data_as(ctypes.c_void_p)))
    return C


def solve6(H, b, damping: float = 0.0) -> np.ndarray:
    """-(H + damping diag(H))^-1 b by Cholesky (binary64)."""
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(6, 6))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(6))
    x = np.empty(6)
    check(_lib.load().vgicp_solve6(H.ctypes.data_as(ctypes.c_void_p),
                                   b.ctypes.data_as(ctypes.c_void_p), float(damping),
                                   x.ctypes.data_as(ctypes.c_void_p)))
    return x


def binary_factor(H, b, T):
    """12x12 H2 and 12 b2 of a factor over [delta_i; delta_j], the right
    perturbations of the source and target world poses (binary64, host)."""
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(6, 6))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(6))
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))
    H2 = np.empty((12, 12))
    b2 = np.empty(12)
    check(_lib.load().vgicp_binary_factor(H.ctypes.data_as(ctypes.c_void_p),
                                          b.ctypes.data_as(ctypes.c_void_p),
                                          T.ctypes.data_as(ctypes.c_void_p),
                                          H2.ctypes.data_as(ctypes.c_void_p),
                                          b2.ctypes.data_as(ctypes.c_void_p)))
    return H2, b2


def optimize_pose_graph(maps, sources, pairs, world_poses, fixed=0, iters=10, damping=1e-6,
                        tile=0, stream=None):
    """Gauss-Newton over the world poses of submaps joined by matching-cost
    factors (the global-mapping graph of Sec. III-F without IMU factors): every
    iteration re-linearizes all factors in one batched launch (Sec. III-A),
    expands each to its two poses, and solves the normal equations on the host
    in binary64 with pose ``fixed`` held as the gauge.  Returns (poses (C, 4, 4),
    total cost per iteration)."""
    W = np.array(world_poses, dtype=np.float64).reshape(-1, 4, 4)
    C = W.shape[0]
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    hist = []
    for _ in range(int(iters)):
        poses = relative_poses(W, pairs)
        out = linearize_batched(maps, sources, pairs, poses, tile=tile,
                                stream=stream).out.cpu().numpy()
        Hg = np.zeros((6 * C, 6 * C))
        bg = np.zeros(6 * C)
        hist.append(float(out[:, 42].sum()))
        for p, (j, i) in enumerate(pairs):
            H2, b2 = binary_factor(out[p, :36], out[p, 36:42], poses[p])
            idx = np.r_[6 * i:6 * i + 6, 6 * j:6 * j + 6]
            Hg[np.ix_(idx, idx)] += H2
            bg[idx] += b2
        keep = np.ones(6 * C, dtype=bool)
        keep[6 * fixed:6 * fixed + 6] = False
        A = Hg[np.ix_(keep, keep)]
        A = A + damping * np.diag(np.diag(A))
        d = np.zeros(6 * C)
        d[keep] = -np.linalg.solve(A, bg[keep])
        for c in range(C):
            if c != fixed:
                W[c] = W[c] @ se3_exp(d[6 * c:6 * c + 6])
    return W, hist


COST, GRADIENT, EXACT_GRADIENT = 1, 2, 3


def evaluate_batched(maps, sources, pairs, poses, mode=GRADIENT, neighbours=1, tile=0,
                     stream=None):
    """Cost (mode 1), Gauss-Newton gradient 2 J^T W d (mode 2) or exact gradient
    (mode 3) of each factor.  Returns (grad (P, 6), err (P,), inliers (P,)), device."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0]
    poses = _pose_array(poses, P)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((P, 7), dtype=torch.float64, device=dev)
    inl = torch.empty(P, dtype=torch.int64, device=dev)
    clouds = make_clouds(sources)
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    opts = LinOpts(int(neighbours), int(tile), 0, 0, None, None, None, None)
    check(_lib.load().vgicp_evaluate_batched(arr, len(maps), clouds, len(sources),
                                             pairs.ctypes.data_as(ctypes.c_void_p), P,
                                             poses.ctypes.data_as(ctypes.c_void_p), int(mode),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(inl.data_ptr()), ctypes.byref(opts),
                                             _stream_ptr(stream)))
    return out[:, :6], out[:, 6], inl


def backward_batched(maps, sources, pairs, poses, exact=False, neighbours=1, tile=0,
                     stream=None):
    """Gradient of each factor's err with respect to its pose increment: 2 J^T W d
    with W held (``exact=False``) or the exact gradient.  Returns (grad (P, 6),
    err (P,), inliers (P,)), device."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0]
    poses = _pose_array(poses, P)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((P, 7), dtype=torch.float64, device=dev)
    inl = torch.empty(P, dtype=torch.int64, device=dev)
    clouds = make_clouds(sources)
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    opts = LinOpts(int(neighbours), int(tile), 0, 0, None, None, None, None)
    check(_lib.load().vgicp_backward_batched(arr, len(maps), clouds, len(sources),
                                             pairs.ctypes.data_as(ctypes.c_void_p), P,
                                             poses.ctypes.data_as(ctypes.c_void_p),
                                             1 if exact else 0, ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(inl.data_ptr()), ctypes.byref(opts),
                                             _stream_ptr(stream)))
    return out[:, :6], out[:, 6], inl


def downsample(points: torch.Tensor, resolution: float, times: torch.Tensor | None = None,
               split: float = 0.0, offsets=None, stream=None):
    """Voxel-grid downsampling with timestamp averaging (Sec. III-C).  Returns
    (points (V, 3), times (V,) or None, counts (V,) int32, out_offsets (C + 1,)
    int64 host), the output voxels in order of first appearance per cloud."""
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be (n, 3) float32")
    points = points.contiguous()
    n = points.shape[0]
    off = np.ascontiguousarray(np.asarray([0, n] if offsets is None else offsets, dtype=np.int64))
    if times is not None:
        times = times.to(torch.float32).contiguous()
    op = torch.empty((max(n, 1), 3), dtype=torch.float32, device=points.device)
    ot = torch.empty(max(n, 1), dtype=torch.float32, device=points.device) if times is not None else None
    oc = torch.empty(max(n, 1), dtype=torch.int32, device=points.device)
    oo = np.zeros(len(off), dtype=np.int64)
    check(_lib.load().vgicp_downsample(
        ctypes.c_void_p(points.data_ptr()), ctypes.c_void_p(times.data_ptr()) if times is not None else None,
        off.ctypes.data_as(ctypes.c_void_p), len(off) - 1, float(resolution), float(split),
        ctypes.c_void_p(op.data_ptr()), ctypes.c_void_p(ot.data_ptr()) if ot is not None else None,
        ctypes.c_void_p(oc.data_ptr()), oo.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    V = int(oo[-1])
    return op[:V], (ot[:V] if ot is not None else None), oc[:V], oo


def estimate_covariances(points: torch.Tensor, offsets=None, k: int = 10, eps: float = 1e-3,
                         cell: float = 0.0, neighbours: bool = False, stream=None):
    """Regularised k-nearest-neighbour covariances (Sec. III-C) of each point of
    the clouds concatenated in ``points`` (device (n, 3) float32; ``offsets``
    host, default one cloud).  Returns covs (n, 6) float32 device, and with
    ``neighbours`` also the (n, k) int32 cloud-local neighbour indices."""
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be (n, 3) float32")
    points = points.contiguous()
    n = points.shape[0]
    off = np.ascontiguousarray(np.asarray([0, n] if offsets is None else offsets, dtype=np.int64))
    covs = torch.empty((n, 6), dtype=torch.float32, device=points.device)
    nbr = torch.empty((n, k), dtype=torch.int32, device=points.device) if neighbours else None
    check(_lib.load().vgicp_estimate_covariances(
        ctypes.c_void_p(points.data_ptr()), off.ctypes.data_as(ctypes.c_void_p), len(off) - 1,
        int(k), float(eps), float(cell), ctypes.c_void_p(nbr.data_ptr()) if nbr is not None else None,
        ctypes.c_void_p(covs.data_ptr()), _stream_ptr(stream)))
    return (covs, nbr) if neighbours else covs


def overlap_batched(maps, sources, pairs, poses, tile=0, stream=None):
    """Overlap rate of each factor (Sec. III-D): the fraction of the source
    points that fall in an occupied voxel of the target map at the pose.
    Returns (rate (P,) float64, inliers (P,) int64), device."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0]
    poses = _pose_array(poses, P)
    dev = torch.device("cuda", torch.cuda.current_device())
    inl = torch.empty(P, dtype=torch.int64, device=dev)
    clouds = make_clouds(sources)
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    opts = LinOpts(1, int(tile), 0, 0, None, None, None, None)
    check(_lib.load().vgicp_overlap_batched(arr, len(maps), clouds, len(sources),
                                            pairs.ctypes.data_as(ctypes.c_void_p), P,
                                            poses.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.c_void_p(inl.data_ptr()), ctypes.byref(opts),
                                            _stream_ptr(stream)))
    sizes = [s.n if isinstance(s, VoxelMap) else int(s[0].shape[0]) for s in sources]
    n = torch.tensor([sizes[int(c)] for c in pairs[:, 1]], dtype=torch.float64, device=dev)
    return inl.double() / n.clamp(min=1.0), inl


def relative_poses(world_poses, pairs) -> np.ndarray:
    """T_target_source = T_j^-1 T_i for each pair (j, i) of world poses (binary64)."""
    W = np.asarray(world_poses, dtype=np.float64).reshape(-1, 4, 4)
    pairs = np.asarray(pairs).reshape(-1, 2)
    inv = np.linalg.inv(W)
    return np.stack([inv[j] @ W[i] for j, i in pairs]) if len(pairs) else np.zeros((0, 4, 4))


def factor_candidates(maps, sources, world_poses, threshold=0.05, tile=0, stream=None):
    """Global-mapping factor creation (Sec. III-F): every ordered pair (target j,
    source i), i != j, whose overlap rate at T_j^-1 T_i reaches ``threshold``.
    ``sources[i]`` is submap i's cloud (or its map), ``world_poses[i]`` its pose.
    Returns (pairs (K, 2) int32 host, rates (K,) float64 host)."""
    W = np.asarray(world_poses, dtype=np.float64).reshape(-1, 4, 4)
    C = len(maps)
    jj, ii = np.meshgrid(np.arange(C), np.arange(C), indexing="ij")
    sel = jj != ii
    pairs = np.stack([jj[sel], ii[sel]], 1).astype(np.int32)
    poses = relative_poses(W, pairs)
    rate, _ = overlap_batched(maps, sources, pairs, poses, tile=tile, stream=stream)
    rate = rate.cpu().numpy()
    keep = rate >= threshold
    return pairs[keep], rate[keep]


def gauss_newton(vmap: VoxelMap, points: torch.Tensor, covs: torch.Tensor, T0, max_iters=30,
                 tol=1e-9, damping=0.0, neighbours=1):
    """Minimise one factor's cost over T = T_target_source: linearize on the GPU
    (H, b, err at T), solve the 6x6 system on the host in binary64 (Cholesky),
    update T <- T Exp(xi) in binary64.  Returns (T, history) with history the
    list of (err, |xi|) per iteration."""
    T = np.ascontiguousarray(np.asarray(T0, dtype=np.float64).reshape(4, 4)).copy()
    hist = []
    out = torch.empty(RESULT_SIZE, dtype=torch.float64, device=points.device)
    inl = torch.empty((), dtype=torch.int64, device=points.device)
    for _ in range(max_iters):
        linearize(vmap, points, covs, T, neighbours=neighbours, out=out, inliers=inl)
        o = out.cpu().numpy()
        xi = solve6(o[:36], o[36:42], damping)
        T = pose_mul(T, se3_exp(xi))
        hist.append((float(o[42]), float(np.linalg.norm(xi))))
        if np.linalg.norm(xi) < tol:
            break
    return T, hist


# ---------------------------------------------------------------------------
# admission: factor sets whose maps and clouds exceed device memory
# ---------------------------------------------------------------------------

def voxelmap_bytes(n_points: int, max_probe=0, capacity_factor=0) -> int:
    opts = _map_opts(max_probe, capacity_factor)
    return int(_lib.load().vgicp_voxelmap_bytes(int(n_points), ctypes.byref(opts)))


def admission_schedule(map_bytes, pairs, budget, src_bytes=None):
    """Batch index of every pair so that each batch's maps and sources fit in
    ``budget`` bytes (sources are the maps themselves when src_bytes is None)."""
    mb = np.ascontiguousarray(np.asarray(map_bytes, dtype=np.int64))
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    sb = None if src_bytes is None else np.ascontiguousarray(np.asarray(src_bytes, np.int64))
    out = np.empty(pairs.shape[0], dtype=np.int32)
    nb = ctypes.c_int32()
    check(_lib.load().vgicp_admission_schedule(
        mb.ctypes.data_as(ctypes.c_void_p), mb.shape[0],
        None if sb is None else sb.ctypes.data_as(ctypes.c_void_p),
        0 if sb is None else sb.shape[0], pairs.ctypes.data_as(ctypes.c_void_p), pairs.shape[0],
        int(budget), 1 if sb is None else 0, out.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(nb)))
    return out, nb.value


def _host_rows(x, a, b):
    return x[a:b] if isinstance(x, torch.Tensor) else torch.from_numpy(x[a:b])


def linearize_admitted(points_host, covs_host, offsets, pairs, poses, resolution, budget,
                       neighbours=27, tile=0, stream=None, kernel_events=None, variant=0):
    """Linearize factors among submaps that live in host memory, batch by batch:
    each batch's submaps are uploaded, built into voxel maps (which also serve
    as the sources) and linearized in one batched launch.  Consecutive batches
    whose submaps have the same sizes reuse one set of device buffers and maps
    (rebuilt in place); the last set is released at the end.
    ``points_host`` / ``covs_host``: numpy arrays or CPU tensors (pinned tensors
    upload at full speed).  Returns (out (P, 43) float64 host, inliers (P,) host,
    n_batches).  ``kernel_events``: optional list; each batch appends the
    (start, stop) torch.cuda.Event pair recorded around its linearize kernel."""
    off = np.asarray(offsets, dtype=np.int64)
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0]
    sizes = np.diff(off)
    mbytes = np.array([voxelmap_bytes(n) + 36 * n for n in sizes], dtype=np.int64)
    batch, nb = admission_schedule(mbytes, pairs, budget)
    out = np.zeros((P, RESULT_SIZE))
    inl = np.zeros(P, dtype=np.int64)
    dev = torch.device("cuda", torch.cuda.current_device())
    # the device buffers and voxel maps of the last batch: a batch whose submaps
    # have the same sizes, in order, refills them (a rebuild allocates nothing)
    # instead of allocating and freeing its own; one batch is resident at a time
    held = None  # (sizes, pts, cvs, maps)
    try:
        for b in range(nb):
            sel = np.nonzero(batch == b)[0]
            used = np.unique(pairs[sel].ravel())
            local = {int(m): k for k, m in enumerate(used)}
            bsizes = tuple(int(x) for x in sizes[used])
            boff = np.concatenate([[0], np.cumsum(sizes[used])]).astype(np.int64)
            reuse = held is not None and held[0] == bsizes
            if not reuse:
                if held is not None:
                    for m in held[3]:
                        m.close()
                    held = None
                pts = torch.empty((int(boff[-1]), 3), dtype=torch.float32, device=dev)
                cvs = torch.empty((int(boff[-1]), 6), dtype=torch.float32, device=dev)
            else:
                _, pts, cvs, maps = held
            for k, m in enumerate(used):
                pts[boff[k]:boff[k + 1]].copy_(_host_rows(points_host, off[m], off[m + 1]),
                                               non_blocking=True)
                cvs[boff[k]:boff[k + 1]].copy_(_host_rows(covs_host, off[m], off[m + 1]),
                                               non_blocking=True)
            if reuse:
                rebuild_voxelmaps(maps, pts, cvs, stream=stream)
            else:
                maps = build_voxelmaps(pts, cvs, boff, resolution, stream=stream)
                held = (bsizes, pts, cvs, maps)
            lp = np.array([[local[int(j)], local[int(i)]] for j, i in pairs[sel]], dtype=np.int32)
            ev = None
            if kernel_events is not None:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for e in ev:  # creates the CUDA event the library then records
                    e.record()
                kernel_events.append(ev)
            res = linearize_batched(maps, maps, lp, poses[sel], neighbours=neighbours, tile=tile,
                                    variant=variant, events=ev, stream=stream)
            out[sel] = res.out.cpu().numpy()
            inl[sel] = res.inliers.cpu().numpy()
            maps[0].status()  # a device-side build error of this batch raises here
    finally:
        if held is not None:
            for m in held[3]:
                m.close()
    return out, inl, nb
