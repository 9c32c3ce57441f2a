"""vgicp_linearize_noalloc: single-factor linearization that allocates nothing.

Who needs it: a caller whose device memory is fixed before its main loop starts
(a real-time mapping front-end that must not stall on the allocator, or a plugin
that a host framework hands a stream and forbids to allocate on) cannot use
vgicp_linearize, which takes its scratch from the stream-ordered allocator on
every call.  This entry point uses a fixed array in device memory instead.

The test calls it through the C ABI (ctypes on the shared library) and compares
its result with vgicp_linearize on the same inputs, twice in a row, because the
fixed array keeps the previous call's contents.  It builds its own inputs so it
passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import cases
from paper_2202_00242_gb300 import api, synth
from paper_2202_00242_gb300._lib import LinOpts

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_00242_gb300 import _lib, build
    build.build()
    return _lib.load()


def _call(lib, fn, vm, pts, covs, T, opts=None):
    out = torch.full((43,), float("nan"), dtype=torch.float64, device="cuda")
    inl = torch.full((), -7, dtype=torch.int64, device="cuda")
    Tn = np.ascontiguousarray(T, dtype=np.float64)
    rc = getattr(lib, fn)(vm.handle, ctypes.c_void_p(pts.data_ptr()),
                          ctypes.c_void_p(covs.data_ptr()), pts.shape[0],
                          Tn.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(inl.data_ptr()),
                          ctypes.byref(opts) if opts is not None else None,
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), int(inl.item())


def test_noalloc_matches_linearize_twice_in_a_row(lib):
    tp, tc, sp, sc, T_true, r = cases.room(seed=5, n_target=6000, n_source=7000)
    vm = api.VoxelMap.build(torch.from_numpy(tp).cuda(), torch.from_numpy(tc).cuda(), r)
    vm.status()
    pts, covs = torch.from_numpy(sp).cuda(), torch.from_numpy(sc).cuda()
    poses = [T_true, synth.perturb_pose(np.random.default_rng(2), T_true, 0.05, 1.0)]
    for T in poses:  # two calls in a row on the shared fixed scratch
        rc_ref, ref, inl_ref = _call(lib, "vgicp_linearize", vm, pts, covs, T)
        rc, got, inl = _call(lib, "vgicp_linearize_noalloc", vm, pts, covs, T)
        assert rc_ref == 0 and rc == 0, lib.vgicp_last_error_string()
        assert inl == inl_ref > 0
        H, Hr = got[:36].reshape(6, 6), ref[:36].reshape(6, 6)
        assert cases.rel_fro(H, Hr) <= TOL
        assert cases.b_error(got[36:42], ref[36:42], ref[42], Hr) <= TOL
        assert abs(got[42] - ref[42]) <= TOL * abs(ref[42])


def test_noalloc_rejects_more_items_than_its_scratch(lib):
    tp, tc, sp, sc, T, r = cases.room(seed=5, n_target=6000, n_source=7000)
    vm = api.VoxelMap.build(torch.from_numpy(tp).cuda(), torch.from_numpy(tc).cuda(), r)
    n = 5000
    pts = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    covs = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    opts = LinOpts(1, 1, 0, 0, None, None, None, None)  # 1 point per item -> 5000 items
    rc, out, inl = _call(lib, "vgicp_linearize_noalloc", vm, pts, covs, T, opts)
    assert rc == -1
    assert b"scratch" in lib.vgicp_last_error_string()
    assert np.isnan(out).all() and inl == -7  # nothing was launched
