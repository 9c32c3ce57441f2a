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
        bench.main(["--impl", "reference", "--submaps", "3", "--neighbours-per-submap", "1",
                    "--steps", "1", "--warmup", "3"])
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
