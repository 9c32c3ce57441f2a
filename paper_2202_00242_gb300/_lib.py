"""ctypes binding of the C ABI declared in include/vgicp.h (argument marshalling only).

Every function of the header is bound here under the same name.  Loading fails
loudly when the compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
f64 = ctypes.c_double


class MapOpts(ctypes.Structure):
    _fields_ = [("max_probe", i32), ("capacity_factor", i32)]


class LinOpts(ctypes.Structure):
    _fields_ = [("neighbours", i32), ("tile", i32), ("grid", i32), ("variant", i32),
                ("corr_out", P), ("qkey_out", P), ("kernel_start", P), ("kernel_stop", P)]


class Cloud(ctypes.Structure):
    _fields_ = [("points", P), ("covs", P), ("n", i64), ("map", P)]


# name -> (restype, argtypes); mirrors include/vgicp.h
SIGNATURES = {
    "vgicp_last_error_string": (ctypes.c_char_p, []),
    "vgicp_version": (ctypes.c_int, []),
    "vgicp_launch_count": (i64, []),
    "vgicp_test_fail_allocations": (ctypes.c_int, [i32]),
    "vgicp_test_expire_waits": (ctypes.c_int, [i32, i64]),
    "vgicp_build_voxelmap": (ctypes.c_int, [P, P, i64, f64, ctypes.POINTER(MapOpts), P,
                                            ctypes.POINTER(P)]),
    "vgicp_build_voxelmaps": (ctypes.c_int, [P, P, P, i32, f64, ctypes.POINTER(MapOpts), P,
                                             ctypes.POINTER(P)]),
    "vgicp_rebuild_voxelmaps": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P, P]),
    "vgicp_destroy_voxelmap": (ctypes.c_int, [P]),
    "vgicp_voxelmap_status": (ctypes.c_int, [P, P]),
    "vgicp_voxelmap_info": (ctypes.c_int, [P, P, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "vgicp_voxelmap_export": (ctypes.c_int, [P, P, i64, P, P, P, P]),
    "vgicp_voxelmap_grouped_cloud": (ctypes.c_int, [P, P, P, P]),
    "vgicp_linearize": (ctypes.c_int, [P, P, P, i64, P, P, P, ctypes.POINTER(LinOpts), P]),
    "vgicp_linearize_noalloc": (ctypes.c_int, [P, P, P, i64, P, P, P, ctypes.POINTER(LinOpts),
                                               P]),
    "vgicp_linearize_batched": (ctypes.c_int, [ctypes.POINTER(P), i32, ctypes.POINTER(Cloud), i32,
                                               P, i64, P, P, P, ctypes.POINTER(LinOpts), P]),
    "vgicp_evaluate_batched": (ctypes.c_int, [ctypes.POINTER(P), i32, ctypes.POINTER(Cloud), i32,
                                              P, i64, P, i32, P, P, ctypes.POINTER(LinOpts), P]),
    "vgicp_backward_batched": (ctypes.c_int, [ctypes.POINTER(P), i32, ctypes.POINTER(Cloud), i32,
                                              P, i64, P, i32, P, P, ctypes.POINTER(LinOpts), P]),
    "vgicp_se3_exp": (ctypes.c_int, [P, P]),
    "vgicp_se3_right_jacobian": (ctypes.c_int, [P, P]),
    "vgicp_pose_mul": (ctypes.c_int, [P, P, P]),
    "vgicp_solve6": (ctypes.c_int, [P, P, f64, P]),
    "vgicp_binary_factor": (ctypes.c_int, [P, P, P, P, P]),
    "vgicp_overlap_batched": (ctypes.c_int, [ctypes.POINTER(P), i32, ctypes.POINTER(Cloud), i32,
                                             P, i64, P, P, ctypes.POINTER(LinOpts), P]),
    "vgicp_estimate_covariances": (ctypes.c_int, [P, P, i32, i32, f64, f64, P, P, P]),
    "vgicp_downsample": (ctypes.c_int, [P, P, P, i32, f64, f64, P, P, P, P, P]),
    "vgicp_voxelmap_bytes": (i64, [i64, ctypes.POINTER(MapOpts)]),
    "vgicp_admission_schedule": (ctypes.c_int, [P, i32, P, i32, P, i64, i64, i32, P, P]),
    "vgicp_plan_create": (ctypes.c_int, [ctypes.POINTER(P), i32, ctypes.POINTER(Cloud), i32, P,
                                         i64, ctypes.POINTER(LinOpts), P, ctypes.POINTER(P)]),
    "vgicp_plan_autotune": (ctypes.c_int, [P, P, P]),
    "vgicp_plan_execute": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "vgicp_plan_evaluate": (ctypes.c_int, [P, P, P, i32, P, P, P, P]),
    "vgicp_plan_info": (ctypes.c_int, [P, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32), ctypes.POINTER(i64)]),
    "vgicp_plan_destroy": (ctypes.c_int, [P]),
}

_lib = None


class VGICPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vgicp error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libvgicp_gb300.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_2202_00242_gb300.build` (CUDA extension required)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != 0:
        msg = load().vgicp_last_error_string()
        raise VGICPError(rc, msg.decode() if msg else "")
    return rc
