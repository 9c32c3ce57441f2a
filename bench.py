#!/usr/bin/env python3
"""Throughput of VGICP factor linearization on one GB300 per rank.

Workload (default): the global-map factor set of arXiv 2202.00242 Sec. III-F
(a matching-cost factor for every overlapping submap pair) on a seeded
synthetic city loop: 500 submaps with log-uniform 30k-80k points each, 5,000
factor pairs (each submap is the source of factors to its 10 nearest submaps),
pose perturbation 0.1 m / 1 deg, voxel resolution 1.0 m.

One step = one pass of the whole hot path: (re)build the 500 target voxel maps
(Sec. III-A voxelization) and linearize all 5,000 factors (Eqs. 2-3 -> H, b, err)
in one batched launch.  Metric: source points per second (sum over the
factors of their source cloud sizes / step time).  Inputs (0.9 GB of points and
covariances) are larger than the 129 MB L2, so no explicit flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VGICP linearize: source pts/s and % HBM peak; batched vs per-factor"
BYTES_PER_POINT = 36  # xyz (12 B) + 6-float covariance (24 B) per source point per factor
# FP32 operations of the linearization, counted from the kernel's formula (an FMA
# counts 2, the reciprocal 1, comparisons and integer key arithmetic 0): per
# point-voxel term, the residual rotated into the source frame (15),
# R^T C' R + C_k from the Cholesky factor (63), the adjugate inverse (30),
# u = W' d' (15), err (6), b (15), H_vv (6), [mu]x W' and its accumulation (36),
# H_ww (24) and the term count (1); per source point, T mu (18) and the float32
# part of the exact key test (11).
FLOPS_PER_TERM = 211
FLOPS_PER_POINT_27 = 29


def fp32_peak_tflops(peaks) -> float:
    """Dense FP32 peak of the GPU: SMs x 128 FP32 lanes x 2 flops (FMA) x the
    maximum SM clock (152 SMs and 2.07 GHz on GB300)."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--submaps", type=int, default=500)
    ap.add_argument("--neighbours-per-submap", type=int, default=10)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0,
                    help="1-neighbour kernel: 0 auto, 1 per-point, 2 shared-memory staged, "
                         "3 hit-compacting (27 neighbours always use 1)")
    ap.add_argument("--sources", choices=["maps", "clouds"], default="maps",
                    help="maps: each submap's own (voxel-grouped) cloud is the source of its "
                         "factors; clouds: the caller's arrays as given")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--parity-pairs", type=int, default=8,
                    help="factors of the timed set checked against the FP64 oracle after "
                         "the timed region (0: none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU time budget of the oracle baseline sample")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-comparison", action="store_true",
                    help="skip the batched vs per-factor comparison")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--workload", choices=["global", "room", "corridor", "differentiable", "large",
                                           "covariances"],
                    default="global",
                    help="global (default): the global-map factor set; the others measure the "
                         "single-factor, odometry-window, autograd and large-map workloads")
    ap.add_argument("--resolution", type=float, default=0.0,
                    help="voxel resolution of the corridor workload (0: 0.25 m)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------

def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init_dist(backend):
    import torch.distributed as dist
    rank, world, _ = rank_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if "MASTER_PORT" not in os.environ:
            raise RuntimeError("WORLD_SIZE > 1 needs MASTER_PORT (launch with "
                               "torch.distributed.run, or pass --gpus N alone)")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Max of a float over all ranks (the step time of the slowest rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device="cpu") -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(args, rank):
    from paper_2202_00242_gb300 import synth
    w = synth.config_global_map(seed=args.seed + 1000 * rank, n_submaps=args.submaps,
                                neighbours=args.neighbours_per_submap)
    return synth.with_surface_covariances(w)


def workload_config(w, args, extra=None):
    sizes = w.clouds.sizes
    cfg = {
        "workload": f"global_map_{len(sizes)}submaps_{w.pairs.shape[0]}pairs_r{w.resolution:g}",
        "submaps": int(len(sizes)),
        "pairs": int(w.pairs.shape[0]),
        "points_per_submap": [int(sizes.min()), int(sizes.max())],
        "target_points": int(sizes.sum()),
        "source_points_per_step": int(w.source_points_per_step),
        "resolution_m": w.resolution,
        "neighbours": 1,
        "step": "rebuild all target voxel maps + batched linearization of all pairs",
        "covariances": "surface-normal Gaussians, eigenvalues (1, 1, 1e-3)",
        "l2": f"inputs larger than L2 ({w.clouds.points.nbytes * 3 / 1e9:.2f} GB of points+covs)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi every 100 ms."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid=None):
        self.uuid = (uuid or "").lower().replace("gpu-", "")
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0].lower():
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = sorted({self.REASONS[i] for _, _, r in rows for i in range(4)
                          if r[i].lower() == "active"})
        sm = [r[0] for r in rows]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)),
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch):
    try:
        return str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return None


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------------

def oracle_sample(w, budget_s, nthreads, start_pair=0, min_pairs=2):
    """Build the needed target maps and linearize pairs in order until the
    budget is spent.  Returns (source points, seconds, pairs done)."""
    import oracle
    oracle.build()
    pts_done = 0
    t0 = time.perf_counter()
    maps = {}
    p = start_pair
    done = 0
    while True:
        j, i = (int(x) for x in w.pairs[p % w.pairs.shape[0]])
        if j not in maps:
            tp, tc = w.clouds.cloud(j)
            maps[j] = oracle.build_voxelmap(tp, tc, w.resolution)
        sp, sc = w.clouds.cloud(i)
        oracle.linearize(maps[j], sp, sc, w.poses[p % w.pairs.shape[0]], nthreads=nthreads)
        pts_done += sp.shape[0]
        p += 1
        done += 1
        if done >= min_pairs and time.perf_counter() - t0 >= budget_s:
            break
    return pts_done, time.perf_counter() - t0, done


# ---------------------------------------------------------------------------
# parity of the measured results against the FP64 oracle (outside the timed region)
# ---------------------------------------------------------------------------

TOL = 1e-4


def near_face_points(points, T, r, tol=1e-5) -> int:
    """Source points whose binary64 position T mu lies within tol of a voxel face."""
    q = points.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    f = q / r - np.floor(q / r)
    return int((np.minimum(f, 1.0 - f).min(axis=1) * r < tol).sum())


def oracle_parity(w, out, inliers, poses, n_sample, neighbours=1, seed=0, grad=None,
                  planted=False):
    """Error of sampled factors against the FP64 oracle: H relative Frobenius,
    b plain relative and relative to max(|b|, sqrt(err |H|_F)), err relative,
    inlier mismatches and near-face points.  ``out`` (P, 43) and ``inliers`` (P,)
    are host arrays; with ``grad`` (P, 6) the gradient 2 J^T W d is checked
    against the oracle's 2 b instead of H and b, and ``out`` holds err only.
    ``planted``: the poses are the scenes' ground truth, where b nearly vanishes;
    b is then held to 1e-4 of the Cauchy-Schwarz scale, otherwise to plain 1e-4."""
    import oracle
    oracle.build()
    P = w.pairs.shape[0]
    sel = np.sort(np.random.default_rng(seed).choice(P, min(n_sample, P), replace=False))
    maps = {}
    eH, eb, ebc, ee, mism, near = [], [], [], [], 0, 0
    for p in sel:
        j, i = (int(x) for x in w.pairs[p])
        if j not in maps:
            maps[j] = oracle.build_voxelmap(*w.clouds.cloud(j), w.resolution)
        sp, sc = w.clouds.cloud(i)
        ref = oracle.linearize(maps[j], sp, sc, poses[p], neighbours=neighbours, nthreads=0)
        mism += int(int(inliers[p]) != ref.inliers)
        near += near_face_points(sp, poses[p], w.resolution)
        if grad is not None:
            g = np.asarray(grad[p], np.float64)
            eb.append(np.linalg.norm(g - 2 * ref.b) / max(np.linalg.norm(2 * ref.b), 1e-300))
            scale = max(np.linalg.norm(ref.b), np.sqrt(max(ref.err, 0.0) * np.linalg.norm(ref.H)))
            ebc.append(np.linalg.norm(g - 2 * ref.b) / max(2 * scale, 1e-300))
            ee.append(abs(float(out[p]) - ref.err) / max(abs(ref.err), 1e-300))
            continue
        o = np.asarray(out[p], np.float64)
        H, b, e = o[:36].reshape(6, 6), o[36:42], float(o[42])
        eH.append(np.linalg.norm(H - ref.H) / max(np.linalg.norm(ref.H), 1e-300))
        eb.append(np.linalg.norm(b - ref.b) / max(np.linalg.norm(ref.b), 1e-300))
        scale = max(np.linalg.norm(ref.b), np.sqrt(max(ref.err, 0.0) * np.linalg.norm(ref.H)))
        ebc.append(np.linalg.norm(b - ref.b) / max(scale, 1e-300))
        ee.append(abs(e - ref.err) / max(abs(ref.err), 1e-300))
    res = {"pairs_checked": int(len(sel)), "pairs_sampled_from": int(P),
           "neighbours": int(neighbours), "reference": "FP64 CPU oracle"}
    if grad is None:
        res["max_rel_fro_H"] = float(max(eH))
    key = "max_rel_grad_vs_2b" if grad is not None else "max_rel_b"
    res[key] = float(max(eb))
    res[key + "_cs_scale"] = float(max(ebc))
    res["max_rel_err"] = float(max(ee))
    res["inlier_mismatches"] = int(mism)
    res["near_face_points"] = int(near)
    res["tolerance"] = TOL
    res["poses"] = "planted (b held to the Cauchy-Schwarz scale)" if planted else "perturbed"
    bmax = max(ebc) if planted else max(eb)
    res["within_tolerance"] = bool(mism == 0 and bmax <= TOL and max(ee) <= TOL
                                   and (grad is not None or max(eH) <= TOL))
    return res


# ---------------------------------------------------------------------------
# ncu DRAM traffic of the linearize kernel, from the committed profile summary
# ---------------------------------------------------------------------------

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "linearize_global_map_traffic.txt")
KERNEL_SOURCES = ["paper_2202_00242_gb300/csrc/vgicp_linearize.cu",
                  "paper_2202_00242_gb300/csrc/vgicp_device.cuh",
                  "paper_2202_00242_gb300/csrc/vgicp_internal.h"]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(source_points: int):
    """dram__bytes_read.sum + dram__bytes_write.sum of one linearize launch, scaled
    to `source_points` from the captured launch, or None when there is no capture
    of the current kernel sources."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256") != kernel_sources_sha256():
            return None
        per_point = float(kv["dram_bytes_per_launch"]) / float(kv["source_points_per_launch"])
        return per_point * source_points
    except (OSError, KeyError, ValueError):
        return None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    init_dist("nccl")
    from paper_2202_00242_gb300 import _lib, api, build
    build.build()
    lib = _lib.load()
    dev = torch.device("cuda", local)

    w = make_workload(args, rank)
    off = w.clouds.offsets
    C = len(off) - 1
    pts = torch.from_numpy(w.clouds.points).to(dev)
    covs = torch.from_numpy(w.clouds.covs).to(dev)
    maps = api.build_voxelmaps(pts, covs, off, w.resolution)
    maps[0].status()
    if args.sources == "maps":
        srcs = maps
    else:
        srcs = [(pts[off[c]:off[c + 1]], covs[off[c]:off[c + 1]]) for c in range(C)]
    P = w.pairs.shape[0]
    out = torch.empty((P, api.RESULT_SIZE), dtype=torch.float64, device=dev)
    inl = torch.empty(P, dtype=torch.int64, device=dev)
    n_pts = w.source_points_per_step
    stream = torch.cuda.current_stream()

    # the factor set is fixed: its work list is planned once, the launch shape
    # autotuned on the GPU, and every step replays one CUDA graph
    plan = api.Plan(maps, srcs, w.pairs, tile=args.tile, variant=args.variant, grid=args.grid)
    tuned = plan.autotune(w.poses) if not (args.tile or args.variant) else plan.info()

    def step(ev=None):
        api.rebuild_voxelmaps(maps, pts, covs)
        plan.execute(w.poses, out=out, inliers=inl, events=ev)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    for m in maps:
        m.status()

    K = args.steps
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    for a, b in kev:  # create the underlying events before the library records them
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_uuid(torch))
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.vgicp_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(K):
        step(kev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = lib.vgicp_launch_count() - launches0
    clk = clocks.stop()
    ms_local = t_start.elapsed_time(t_end) / K
    kernel_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    ms = max_over_ranks(ms_local, world, dev)
    total_pts = sum_over_ranks(n_pts, world, dev)
    value = total_pts / (ms / 1e3)

    # batched vs per-factor on the same GPU (linearize only, the caller's clouds as
    # given): one vgicp_linearize launch pair per factor vs one batched plan
    comparison = None
    if not args.no_comparison:
        csrcs = [(pts[off[c]:off[c + 1]], covs[off[c]:off[c + 1]]) for c in range(C)]
        cplan = api.Plan(maps, csrcs, w.pairs, tile=tuned["item_points"], variant=tuned["variant"])
        cplan.execute(w.poses, out=out, inliers=inl)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            cplan.execute(w.poses, out=out, inliers=inl)
        e1.record(stream)
        torch.cuda.synchronize()
        batched_ms = e0.elapsed_time(e1) / 3
        cplan.close()
        outs = torch.empty((P, api.RESULT_SIZE), dtype=torch.float64, device=dev)
        inls = torch.empty(P, dtype=torch.int64, device=dev)

        def per_factor():
            for p_ in range(P):
                j, i = int(w.pairs[p_, 0]), int(w.pairs[p_, 1])
                api.linearize(maps[j], csrcs[i][0], csrcs[i][1], w.poses[p_], out=outs[p_],
                              inliers=inls[p_])

        per_factor()
        torch.cuda.synchronize()
        e0.record(stream)
        per_factor()
        e1.record(stream)
        torch.cuda.synchronize()
        pf_ms = e0.elapsed_time(e1)
        comparison = {"sources": "caller clouds as given", "step": "linearize only",
                      "batched_graph": {"ms": batched_ms, "value": n_pts / (batched_ms / 1e3)},
                      "per_factor_launches": {"ms": pf_ms, "value": n_pts / (pf_ms / 1e3),
                                              "launches": 2 * P}}

    # e2e through the public API: pinned host clouds in, results out, every step.
    # Step k+1's clouds are uploaded on a copy stream into the other of two device
    # buffers while step k rebuilds its maps and linearizes; every upload and
    # every read-back lies inside the timed region.
    pts_h = torch.from_numpy(w.clouds.points).pin_memory()
    covs_h = torch.from_numpy(w.clouds.covs).pin_memory()
    out_h = torch.empty_like(out, device="cpu").pin_memory()
    inl_h = torch.empty_like(inl, device="cpu").pin_memory()
    E = max(args.e2e_steps, 2)
    bufs = [(pts, covs), (torch.empty_like(pts), torch.empty_like(covs))]
    cstream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(b):
        cstream.wait_event(freed[b])
        with torch.cuda.stream(cstream):
            bufs[b][0].copy_(pts_h, non_blocking=True)
            bufs[b][1].copy_(covs_h, non_blocking=True)
        copied[b].record(cstream)

    def e2e_run(steps, start_event=None):
        for b in (0, 1):
            freed[b].record(stream)
        if start_event is not None:
            cstream.wait_event(start_event)
        upload(0)
        for k in range(steps):
            b = k % 2
            stream.wait_event(copied[b])
            if k + 1 < steps:
                upload(1 - b)
            api.rebuild_voxelmaps(maps, bufs[b][0], bufs[b][1])
            freed[b].record(stream)
            plan.execute(w.poses, out=out, inliers=inl)
            out_h.copy_(out, non_blocking=True)
            inl_h.copy_(inl, non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the pinned host-to-device bandwidth on its own (one upload, copy stream idle
    # otherwise): the end-to-end step hides the upload only while it is shorter
    # than the device step
    e0.record(cstream)
    with torch.cuda.stream(cstream):
        bufs[1][0].copy_(pts_h, non_blocking=True)
        bufs[1][1].copy_(covs_h, non_blocking=True)
    e1.record(cstream)
    torch.cuda.synchronize()
    h2d_alone_ms = e0.elapsed_time(e1)
    barrier(world)
    e0.record(stream)
    e2e_run(E, start_event=e0)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / E, world, dev)
    e2e_value = total_pts / (e2e_ms / 1e3)
    h2d = pts_h.numel() * 4 + covs_h.numel() * 4
    d2h = out_h.numel() * 8 + inl_h.numel() * 8

    # parity of the timed factor set: one more step, sampled factors against the oracle
    parity = None
    if args.parity_pairs > 0:
        step()
        torch.cuda.synchronize()
        parity = oracle_parity(w, out.cpu().numpy(), inl.cpu().numpy(), w.poses,
                               args.parity_pairs, seed=rank)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = BYTES_PER_POINT * n_pts / (kernel_ms / 1e3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        n_done, secs, pairs_done = oracle_sample(w, args.cpu_seconds, cores)
        n1, secs1, pairs1 = oracle_sample(w, min(3.0, args.cpu_seconds), 1)
        cpu = {"value": n_done / secs, "unit": "source pts/s", "cores": cores, "kind": "oracle",
               "sample": f"first {pairs_done} of {P} pairs in order (their target maps built by "
                         f"the oracle inside the timed sample), {n_done} source points, "
                         f"{secs:.1f} s, FP64, OpenMP over {cores} threads",
               "single_thread": {"value": n1 / secs1, "unit": "source pts/s",
                                 "sample": f"first {pairs1} pairs, {n1} source points, "
                                           f"{secs1:.1f} s, one thread"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "source pts/s", "n_gpus": world,
            "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded city-loop submaps; no dataset available)",
            "config": workload_config(w, args, {"parallelism": f"independent factor sets x{world}",
                                                "sources": args.sources,
                                                "launch": tuned,
                                                "autotuned": not (args.tile or args.variant),
                                                "cuda_graph": True}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": measured_traffic(n_pts),
                         "kernel": "linearize (1-neighbour), timed as its graph (status reset + "
                                   "linearize + per-pair reduce)", "kernel_ms": kernel_ms,
                         "algorithmic_bytes_per_launch": BYTES_PER_POINT * n_pts,
                         "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)"},
            "e2e": {"value": e2e_value, "unit": "source pts/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "h2d_alone": {"ms": h2d_alone_ms, "GB/s": h2d / (h2d_alone_ms / 1e3) / 1e9},
                    "pipelining": "upload of step k+1 (copy stream, second buffer) overlaps "
                                  "step k"},
            "batched_vs_per_factor": comparison,
            "parity": parity,
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    w = make_workload(args, 0)
    cores = host_cores()
    P = w.pairs.shape[0]
    per_step_pairs = 4
    for s in range(max(args.warmup, 3)):
        oracle_sample(w, 0.0, cores, start_pair=s * per_step_pairs, min_pairs=per_step_pairs)
    t0 = time.perf_counter()
    pts = 0
    for s in range(args.steps):
        n, _, _ = oracle_sample(w, 0.0, cores, start_pair=(s * per_step_pairs) % P,
                                min_pairs=per_step_pairs)
        pts += n
    secs = time.perf_counter() - t0
    value = pts / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "source pts/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded city-loop submaps; no dataset available)",
        "config": workload_config(w, args, {"parallelism": "host cores (oracle)"}),
        "cpu_baseline": {"value": value, "unit": "source pts/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step_pairs} consecutive pairs per step (target maps "
                                   f"built inside the step), FP64 oracle, OpenMP over {cores} "
                                   "threads"},
        "e2e": {"value": value, "unit": "source pts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads (one GPU; each line uses the same metric)
# ---------------------------------------------------------------------------

def _timed(torch, fn, steps, warmup):
    for _ in range(max(warmup, 3)):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_workload(args):
    import torch
    from paper_2202_00242_gb300 import _lib, api, autograd, build, synth
    build.build()
    lib = _lib.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    K = args.steps if args.steps != 200 else {"room": 200, "corridor": 200, "differentiable": 20,
                                               "large": 2, "covariances": 20}[args.workload]
    extra = {"covariances": "surface-normal Gaussians, eigenvalues (1, 1, 1e-3)"}
    if args.workload == "room":
        w = synth.with_surface_covariances(synth.config_room())
        tp, tc = w.clouds.cloud(0)
        sp, sc = w.clouds.cloud(1)
        tpd, tcd = torch.from_numpy(tp).to(dev), torch.from_numpy(tc).to(dev)
        spd, scd = torch.from_numpy(sp).to(dev), torch.from_numpy(sc).to(dev)
        vm = api.VoxelMap.build(tpd, tcd, w.resolution)
        out = torch.empty(api.RESULT_SIZE, dtype=torch.float64, device=dev)
        inl = torch.empty((), dtype=torch.int64, device=dev)
        T = w.poses[0]

        def step():
            api.rebuild_voxelmaps([vm], tpd, tcd)
            api.linearize(vm, spd, scd, T, out=out, inliers=inl)
        n_pts = sp.shape[0]
        name = "room_single_factor_8192x8192_r0.5"
        extra["step"] = "rebuild the target voxel map + one single-factor linearization"
    elif args.workload == "corridor":
        r = args.resolution or 0.25
        w = synth.with_surface_covariances(synth.config_corridor(resolution=r))
        Kf = len(w.clouds.offsets) - 2
        off = w.clouds.offsets
        pts = torch.from_numpy(w.clouds.points).to(dev)
        covs = torch.from_numpy(w.clouds.covs).to(dev)
        kp, kc = pts[:off[Kf]].contiguous(), covs[:off[Kf]].contiguous()
        maps = api.build_voxelmaps(kp, kc, off[:Kf + 1], r)
        src = [(pts[off[Kf]:off[Kf + 1]], covs[off[Kf]:off[Kf + 1]])]
        pairs = np.stack([np.arange(Kf), np.zeros(Kf, np.int64)], 1)
        plan = api.Plan(maps, src, pairs)
        plan.autotune(w.poses)

        def step():
            api.rebuild_voxelmaps(maps, kp, kc)
            plan.execute(w.poses)
        n_pts = Kf * int(off[Kf + 1] - off[Kf])
        name = f"corridor_window_1scan_vs_{Kf}keyframes_20000pts_r{r:g}"
        extra["step"] = "rebuild the 10 keyframe maps + batched linearization (CUDA graph)"
    elif args.workload == "differentiable":
        w = synth.with_surface_covariances(synth.config_differentiable())
        off = w.clouds.offsets
        C = len(off) - 1
        pts = torch.from_numpy(w.clouds.points).to(dev)
        covs = torch.from_numpy(w.clouds.covs).to(dev)
        maps = api.build_voxelmaps(pts, covs, off, w.resolution)
        srcs = [(pts[off[c]:off[c + 1]], covs[off[c]:off[c + 1]]) for c in range(C)]
        fs = autograd.FactorSet(maps, srcs, w.pairs, w.poses)
        xi = torch.zeros((w.pairs.shape[0], 6), dtype=torch.float64, device=dev,
                         requires_grad=True)

        def step():
            xi.grad = None
            fs.cost(xi).sum().backward()
        n_pts = int(w.source_points_per_step)
        name = f"differentiable_{w.pairs.shape[0]}pairs_20k-50k_r{w.resolution:g}"
        extra["step"] = ("forward (poses T0 Exp(xi) composed on the device, cost kernel) + "
                         "backward (gradient kernel, J_r^T and the incoming gradient applied "
                         "on the device) of the autograd Function over all factors, xi on the "
                         "GPU; points counted once")
    elif args.workload == "covariances":
        w = synth.config_global_map(n_submaps=args.submaps)
        pts = torch.from_numpy(w.clouds.points).to(dev)
        off = w.clouds.offsets

        def step():
            api.estimate_covariances(pts, offsets=off, k=10, eps=1e-3)
        n_pts = int(off[-1])
        name = f"knn_covariances_{len(off) - 1}clouds_{n_pts}pts_k10"
        extra["step"] = ("k = 10 nearest neighbours (exact, binary64 distances) and the "
                         "regularised covariance of every point, clouds searched separately")
        extra["unit_note"] = "points (not source points of factors) per second"
        extra["covariances"] = "computed by the step"
    else:  # large
        w = synth.with_surface_covariances(synth.config_large_map(n_submaps=args.submaps
                                                                   if args.submaps != 500
                                                                   else 2000))
        budget = 24 << 30
        state = {}
        pts_h = torch.from_numpy(w.clouds.points).pin_memory()  # the clouds stay on the host
        covs_h = torch.from_numpy(w.clouds.covs).pin_memory()

        def step():
            state["ev"] = []
            state["r"] = api.linearize_admitted(pts_h, covs_h, w.clouds.offsets,
                                                w.pairs, w.poses, w.resolution, budget=budget,
                                                neighbours=27, kernel_events=state["ev"],
                                                variant=args.variant, tile=args.tile)
        n_pts = int(w.source_points_per_step)
        name = (f"large_map_{len(w.clouds.offsets) - 1}submaps_x100k_{w.pairs.shape[0]}pairs"
                f"_r0.5_27neighbours")
        extra["step"] = ("admission batches under a 24 GB budget: per batch, upload the "
                         "submaps from host memory, build their maps, one batched "
                         "27-neighbour linearization")
        extra["inputs"] = "pinned host memory (7.2 GB of clouds, uploaded inside every step)"
    launches0 = lib.vgicp_launch_count()
    clocks = ClockSampler(gpu_uuid(torch))
    clocks.start()
    ms = _timed(torch, step, K, args.warmup)
    clk = clocks.stop()
    launches = lib.vgicp_launch_count() - launches0
    if args.workload == "large":
        extra["admission_batches"] = int(state["r"][2])
    if args.workload == "differentiable":
        # device time of the two evaluations one autograd step launches (cost,
        # then gradient with J_r^T and the incoming gradient), back to back
        x0 = torch.zeros((w.pairs.shape[0], 6), dtype=torch.float64, device=dev)
        ones = torch.ones(w.pairs.shape[0], dtype=torch.float64, device=dev)

        def two_evaluations():
            fs.plan.evaluate(fs.base, x0, mode=api.COST)
            fs.plan.evaluate(fs.base, x0, mode=api.GRADIENT, grad_scale=ones)
        extra["device_ms_cost_plus_gradient"] = _timed(torch, two_evaluations, K, args.warmup)

    # parity of the timed workload's results against the FP64 oracle (untimed)
    parity = None
    if args.parity_pairs > 0:
        if args.workload == "room":
            api.linearize(vm, spd, scd, T, out=out, inliers=inl)
            parity = oracle_parity(w, out.cpu().numpy()[None], inl.cpu().numpy()[None], w.poses,
                                   1)
        elif args.workload == "corridor":
            res = plan.execute(w.poses)
            parity = oracle_parity(w, res.out.cpu().numpy(), res.inliers.cpu().numpy(), w.poses,
                                   args.parity_pairs, planted=True)
        elif args.workload == "differentiable":
            g, err, inl_d = api.evaluate_batched(maps, srcs, w.pairs, w.poses, mode=api.GRADIENT)
            parity = oracle_parity(w, err.cpu().numpy(), inl_d.cpu().numpy(), w.poses,
                                   args.parity_pairs, grad=g.cpu().numpy())
        elif args.workload == "large":
            parity = oracle_parity(w, state["r"][0], state["r"][1], w.poses,
                                   min(args.parity_pairs, 4), neighbours=27)
    value = n_pts / (ms / 1e3)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = BYTES_PER_POINT * n_pts / (ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "whole step (36 B per source point over the step time)"}
    if args.workload == "large":
        # the 27-neighbour linearize kernel alone, over the last step's batches:
        # its HBM fraction (36 B per source point) and its FP32 fraction
        torch.cuda.synchronize()
        kms = float(sum(a.elapsed_time(b) for a, b in state["ev"]))
        terms = float(np.sum(state["r"][1]))  # point-voxel terms (27-neighbour inliers)
        flops = FLOPS_PER_TERM * terms + FLOPS_PER_POINT_27 * n_pts
        fp32_peak = fp32_peak_tflops(peaks)
        roofline = {"bound": "alu", "achieved": flops / (kms / 1e3) / 1e12, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": flops / (kms / 1e3) / 1e12 / fp32_peak,
                    "traffic": None,
                    "kernel": "27-neighbour linearize kernel alone (CUDA events around each "
                              "admission batch's launch, summed)",
                    "kernel_ms": kms, "terms": terms,
                    "flops": {"per_term": FLOPS_PER_TERM, "per_point": FLOPS_PER_POINT_27},
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                    "hbm": {"achieved": BYTES_PER_POINT * n_pts / (kms / 1e3) / 1e9,
                            "peak": peak, "unit": "GB/s",
                            "frac": BYTES_PER_POINT * n_pts / (kms / 1e3) / 1e9 / peak}}
    line = {
        "metric": METRIC, "value": value, "unit": "source pts/s", "n_gpus": 1, "steps": K,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded scenes; no dataset available)",
        "config": dict({"workload": name, "source_points_per_step": n_pts}, **extra),
        "roofline": roofline,
        "parity": parity, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def free_port() -> int:
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(args, argv) -> int:
    """--gpus N without a launcher: start N ranks of this script, one per GPU, with
    torch.distributed.run on this node (127.0.0.1, a free port).  Returns the
    launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1",
           "--nproc-per-node", str(args.gpus), "--master-addr", "127.0.0.1",
           "--master-port", str(free_port()), os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    args = parse_args(argv)
    env_world = os.environ.get("WORLD_SIZE")
    if env_world is None and args.gpus > 1:
        rc = launch_ranks(args, argv)
        if rc != 0:
            raise SystemExit(rc)
        return
    if env_world is not None and int(env_world) != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} disagrees with WORLD_SIZE={env_world}")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "global":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
