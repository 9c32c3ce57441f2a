"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank owns an independent factor set (weak scaling, no data-path collective);
the step time is the max over ranks and the throughput the sum of the ranks'
points over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w = bench.init_dist("gloo")
    ms = bench.max_over_ranks(10.0 + r, w)
    pts = bench.sum_over_ranks(1000.0 * (r + 1), w)
    args = bench.parse_args(["--submaps", "4", "--neighbours-per-submap", "2"])
    wl = bench.make_workload(args, r)
    bench.barrier(w)
    q.put((r, ms, pts, float(wl.clouds.points[0, 0]), wl.pairs.shape[0]))
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_max_time_sum_points_independent_workloads():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]       # slowest rank's step time
    assert [r[2] for r in res] == [3000.0, 3000.0]   # points of both ranks
    assert res[0][4] == res[1][4] == 8
    assert res[0][3] != res[1][3]                    # each rank its own seeded factor set


def _reference_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import contextlib
    import io
    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main(["--gpus", str(world), "--impl", "reference", "--submaps", "3",
                    "--neighbours-per-submap", "1", "--steps", "1", "--warmup", "3"])
    q.put((rank, buf.getvalue()))


@pytest.mark.timeout(300)
def test_reference_arm_prints_on_rank_zero_only():
    import json
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reference_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] == ""
    line = json.loads(res[0].strip())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.timeout(300)
def test_gpus_flag_starts_one_rank_per_gpu():
    """`bench.py --gpus 2` without a launcher starts two ranks itself
    (torch.distributed.run on 127.0.0.1, a free port); the reference arm then
    runs on rank 0 only and reports the world size."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2",
                        "--impl", "reference", "--submaps", "3", "--neighbours-per-submap", "1",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2


def test_gpus_flag_must_match_launcher_world_size(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(SystemExit):
        bench.main(["--gpus", "3", "--impl", "reference"])
