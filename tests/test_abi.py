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
    opts = _lib.LinOpts(5, 0, 0, 0, None, None)
    rc = lib.vgicp_linearize_batched(None, 0, None, 0, None, 1, None, None, None,
                                     ctypes.byref(opts), None)
    assert rc == -1
