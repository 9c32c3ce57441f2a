"""Failure paths, made without faulting the GPU: an allocation failure injected
on the host, and a bounded device wait that is made to run out.

  * an injected allocation failure makes each allocating entry point return
    VGICP_ERR_OOM, and the next calls on the same context still match the
    oracle;
  * a staged-kernel launch whose producer withholds a tile: the consumers'
    bounded mbarrier wait (20 ms for that launch) runs out, the launch's status
    word turns its outputs into NaN and its inlier count into -1, the kernel
    returns with no copy in flight, and the next launch on the same context is
    correct.
"""
import numpy as np
import pytest
import torch

import cases
import oracle
from paper_2202_00242_gb300 import api, synth
from paper_2202_00242_gb300._lib import VGICPError

from test_gpu_parity import check_factor, cu, dev  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

OOM = -2


@pytest.fixture
def lib(dev):  # noqa: F811
    from paper_2202_00242_gb300 import _lib
    L = _lib.load()
    yield L
    L.vgicp_test_fail_allocations(0)


def _expect_oom(lib, fn):
    assert lib.vgicp_test_fail_allocations(1) == 0
    with pytest.raises(VGICPError) as e:
        fn()
    assert e.value.code == OOM, e.value
    assert b"memory" in lib.vgicp_last_error_string().lower() or b"alloc" in \
        lib.vgicp_last_error_string().lower()


def test_injected_allocation_failure_returns_oom_and_context_stays_usable(lib):
    tp, tc, sp, sc, T_true, r = cases.room()
    T = synth.perturb_pose(np.random.default_rng(3), T_true, 0.05, 1.0)
    tpd, tcd, spd, scd = cu(tp), cu(tc), cu(sp), cu(sc)
    _expect_oom(lib, lambda: api.VoxelMap.build(tpd, tcd, r))
    vm = api.VoxelMap.build(tpd, tcd, r)
    vm.status()
    _expect_oom(lib, lambda: api.linearize(vm, spd, scd, T))
    _expect_oom(lib, lambda: api.linearize_batched([vm], [(spd, scd)], [[0, 0]], T[None]))
    _expect_oom(lib, lambda: api.Plan([vm], [(spd, scd)], [[0, 0]]))
    _expect_oom(lib, lambda: api.estimate_covariances(spd))
    _expect_oom(lib, lambda: api.downsample(spd, 0.2))
    assert lib.vgicp_test_fail_allocations(-1) == -1
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T)
    lin = api.linearize(vm, spd, scd, T)
    check_factor(lin.out, lin.inliers, ref)
    fresh = api.VoxelMap.build(tpd, tcd, r)
    lin = api.linearize(fresh, spd, scd, T)
    check_factor(lin.out, lin.inliers, ref)
    plan = api.Plan([vm], [(spd, scd)], [[0, 0]])
    res = plan.execute(T[None])
    check_factor(res.out[0], res.inliers[0], ref)
    plan.close()


def test_expired_device_wait_reports_status_and_next_call_is_correct(lib):
    tp, tc, sp, sc, T_true, r = cases.room()
    T = synth.perturb_pose(np.random.default_rng(3), T_true, 0.05, 1.0)
    vm = api.VoxelMap.build(cu(tp), cu(tc), r)
    vm.status()
    spd, scd = cu(sp), cu(sc)
    ref = oracle.linearize(oracle.build_voxelmap(tp, tc, r), sp, sc, T)
    assert lib.vgicp_test_expire_waits(0, 20_000_000) == 0
    bad = api.linearize(vm, spd, scd, T, variant=2, tile=1024)
    torch.cuda.synchronize()
    assert torch.isnan(bad.out).all() and int(bad.inliers) == -1
    # the hook is one-shot: the next staged launch waits normally
    good = api.linearize(vm, spd, scd, T, variant=2, tile=1024)
    check_factor(good.out, good.inliers, ref, "staged, after the expired wait")
    # a withheld tile in the middle of a CTA's stream, batched
    assert lib.vgicp_test_expire_waits(5, 20_000_000) == 0
    bat = api.linearize_batched([vm], [(spd, scd)], [[0, 0], [0, 0]], np.stack([T, T]),
                                variant=2, tile=4096)
    torch.cuda.synchronize()
    assert torch.isnan(bat.out).all() and (bat.inliers == -1).all()
    bat = api.linearize_batched([vm], [(spd, scd)], [[0, 0], [0, 0]], np.stack([T, T]),
                                variant=2, tile=4096)
    for p in range(2):
        check_factor(bat.out[p], bat.inliers[p], ref, f"batched pair {p}")
    lin = api.linearize(vm, spd, scd, T)
    check_factor(lin.out, lin.inliers, ref, "per-point kernel")
    assert lib.vgicp_test_expire_waits(-1, 1000) != 0
    assert lib.vgicp_test_expire_waits(0, 0) != 0
