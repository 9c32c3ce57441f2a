"""The C-ABI library loads and exports every entry point that include/vgicp.h
declares, and its host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(vgicp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_00242_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2202_00242_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_host_argument_checks_without_gpu(lib):
    from paper_2202_00242_gb300 import _lib
    assert lib.vgicp_version() == 10000
    h = ctypes.c_void_p()
    # invalid resolution is rejected before any device work
    rc = lib.vgicp_build_voxelmap(None, None, 0, -1.0, None, None, ctypes.byref(h))
    assert rc == -1 and b"resolution" in lib.vgicp_last_error_string()
    rc = lib.vgicp_build_voxelmap(None, None, -5, 0.5, None, None, ctypes.byref(h))
    assert rc == -1
    # misaligned cloud pointer
    rc = lib.vgicp_build_voxelmap(ctypes.c_void_p(2), ctypes.c_void_p(8), 1, 0.5, None, None,
                                  ctypes.byref(h))
    assert rc == -1 and b"aligned" in lib.vgicp_last_error_string()
    # null map / outputs
    rc = lib.vgicp_linearize(None, None, None, 0, None, None, None, None, None)
    assert rc == -1
    assert lib.vgicp_destroy_voxelmap(None) == 0
    # a null map is refused before any copy
    assert lib.vgicp_voxelmap_grouped_cloud(None, None, None, None) == -1
    opts = _lib.LinOpts(5, 0, 0, 0, None, None)
    rc = lib.vgicp_linearize_batched(None, 0, None, 0, None, 1, None, None, None,
                                     ctypes.byref(opts), None)
    assert rc == -1


def _i64(*v):
    return (ctypes.c_int64 * len(v))(*v)


def test_host_checks_of_covariance_downsample_and_overlap(lib):
    """Each rejected argument returns -1 with a message before any device work;
    an empty input succeeds without touching the device."""
    from paper_2202_00242_gb300 import _lib
    err = lambda: lib.vgicp_last_error_string()  # noqa: E731
    ok2 = _i64(0, 0)
    # k-nearest-neighbour covariances
    est = lib.vgicp_estimate_covariances
    assert est(None, ok2, 0, 20, 1e-3, 0.0, None, None, None) == -1
    assert est(None, ok2, 1, 0, 1e-3, 0.0, None, None, None) == -1 and b"k must" in err()
    assert est(None, ok2, 1, 33, 1e-3, 0.0, None, None, None) == -1
    assert est(None, ok2, 1, 20, 0.0, 0.0, None, None, None) == -1 and b"eps" in err()
    assert est(None, ok2, 1, 20, 1.5, 0.0, None, None, None) == -1
    assert est(None, ok2, 1, 20, 1e-3, -1.0, None, None, None) == -1 and b"cell" in err()
    assert est(None, ok2, 1, 20, 1e-3, float("nan"), None, None, None) == -1
    assert est(None, _i64(1, 4), 1, 20, 1e-3, 0.0, None, None, None) == -1
    assert b"offsets[0]" in err()
    assert est(None, _i64(0, 5, 3), 2, 20, 1e-3, 0.0, None, None, None) == -1
    assert b"non-decreasing" in err()
    assert est(None, _i64(0, 0, 0), 2, 20, 1e-3, 0.0, None, None, None) == 0
    # voxel-grid downsampling
    ds = lib.vgicp_downsample
    out = _i64(7, 7, 7)
    assert ds(None, None, ok2, 1, 0.0, 1.0, None, None, None, out, None) == -1
    assert b"resolution" in err()
    assert ds(None, None, ok2, 1, float("inf"), 1.0, None, None, None, out, None) == -1
    assert ds(None, None, ok2, 1, 0.5, 1.0, None, None, None, None, None) == -1
    assert ds(None, None, _i64(0, 3, 1), 2, 0.5, 1.0, None, None, None, out, None) == -1
    assert ds(None, None, ok2, 1, 0.5, float("nan"), None, None, None, out, None) == -1
    assert b"split" in err()
    assert ds(None, None, _i64(0, 0, 0), 2, 0.5, 1.0, None, None, None, out, None) == 0
    assert list(out) == [0, 0, 0]
    # non-null points with n > 0 still need aligned device buffers
    assert ds(None, None, _i64(0, 4), 1, 0.5, 1.0, None, None, None, out, None) == -1
    # overlap: the rate uses the one-neighbour lookup only
    opts = _lib.LinOpts(27, 0, 0, 0, None, None)
    ov = lib.vgicp_overlap_batched
    assert ov(None, 1, None, 1, None, 1, None, None, ctypes.byref(opts), None) == -1
    assert b"1-neighbour" in err()
    opts.neighbours = 1
    assert ov(None, 1, None, 1, None, 1, None, None, ctypes.byref(opts), None) == -1
    assert b"null" in err()
    assert ov(None, 0, None, 0, None, 0, None, None, None, None) == 0
    assert ov(None, 0, None, 0, None, -1, None, None, None, None) == -1


def test_host_checks_of_se3_and_admission(lib):
    d16 = (ctypes.c_double * 16)()
    d36 = (ctypes.c_double * 36)()
    d6 = (ctypes.c_double * 6)()
    assert lib.vgicp_se3_exp(None, d16) == -1
    assert lib.vgicp_se3_right_jacobian(d6, None) == -1
    assert lib.vgicp_pose_mul(d16, None, d16) == -1
    assert lib.vgicp_binary_factor(d36, d6, None, d36, d6) == -1
    # a zero H is not positive definite, with or without damping
    assert lib.vgicp_solve6(d36, d6, 0.0, d6) == -1 and b"positive definite" in \
        lib.vgicp_last_error_string()
    # the voxel map size bound grows with the point count
    sizes = [lib.vgicp_voxelmap_bytes(n, None) for n in (0, 1, 1000, 10 ** 6)]
    assert all(s > 0 for s in sizes) and sizes == sorted(sizes) and sizes[3] > 64 * 10 ** 6
    mb = _i64(100, 200)
    pairs = (ctypes.c_int32 * 2)(0, 2)
    bop = (ctypes.c_int32 * 1)()
    nb = ctypes.c_int32()
    sched = lib.vgicp_admission_schedule
    assert sched(mb, 2, None, 0, pairs, 1, 10 ** 6, 1, bop, ctypes.byref(nb)) == -1
    assert b"out of range" in lib.vgicp_last_error_string()
    pairs[1] = 1
    assert sched(mb, 2, None, 0, pairs, 1, 299, 1, bop, ctypes.byref(nb)) == -1
    assert b"exceeds" in lib.vgicp_last_error_string()
    assert sched(mb, 2, None, 0, pairs, 1, 300, 1, bop, ctypes.byref(nb)) == 0
    assert nb.value == 1 and bop[0] == 0
    assert sched(mb, 2, None, 0, pairs, 0, 300, 1, bop, ctypes.byref(nb)) == 0 and nb.value == 0


def test_host_checks_of_plans(lib):
    """Plan creation and use reject bad arguments before any device work."""
    from paper_2202_00242_gb300 import _lib
    err = lambda: lib.vgicp_last_error_string()  # noqa: E731
    h = ctypes.c_void_p()
    maps = (ctypes.c_void_p * 1)(ctypes.c_void_p(8))
    srcs = (_lib.Cloud * 1)()
    pairs = (ctypes.c_int32 * 2)(0, 0)
    create = lib.vgicp_plan_create
    assert create(maps, 1, srcs, 1, pairs, 1, None, None, None) == -1 and b"out" in err()
    assert create(None, 1, srcs, 1, pairs, 1, None, None, ctypes.byref(h)) == -1
    assert create(maps, 1, srcs, 1, pairs, 0, None, None, ctypes.byref(h)) == -1
    assert b"empty" in err() and not h.value
    for nb, tile, variant, msg in [(5, 0, 0, b"neighbours"), (1, 1024, 0, b"2048"),
                                   (1, 0, 7, b"variant")]:
        opts = _lib.LinOpts(nb, tile, 0, variant, None, None)
        assert create(maps, 1, srcs, 1, pairs, 1, ctypes.byref(opts), None,
                      ctypes.byref(h)) == -1
        assert msg in err() and not h.value
    opts = _lib.LinOpts(1, 0, 0, 0, ctypes.c_void_p(16), None)
    assert create(maps, 1, srcs, 1, pairs, 1, ctypes.byref(opts), None, ctypes.byref(h)) == -1
    assert b"single-factor" in err()
    poses = (ctypes.c_double * 16)()
    assert lib.vgicp_plan_execute(None, poses, None, None, None, None, None) == -1
    assert lib.vgicp_plan_autotune(None, poses, None) == -1
    assert lib.vgicp_plan_info(None, None, None, None, None) == -1
    assert lib.vgicp_plan_destroy(None) == 0
