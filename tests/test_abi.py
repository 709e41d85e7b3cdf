"""The C ABI library builds, loads and exports every function that
include/flycoo.h declares; argument checks that need no device answer with
their documented status codes.  No compute call runs here."""
import ctypes
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_09131_gb300 import build as B
    B.build()
    from paper_2309_09131_gb300 import _native
    return _native


def test_every_declared_function_is_exported(native):
    names = native.header_functions()
    assert "flycoo_create" in names and "flycoo_spmttkrp" in names and "flycoo_remap" in names
    L = native.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def test_binding_names_match_header(native):
    import paper_2309_09131_gb300 as P
    for n in native.header_functions():
        assert hasattr(native, n), n
        assert hasattr(P, n), n


def test_host_side_argument_checks(native):
    L = native.lib()
    h = ctypes.c_void_p()
    dims = (ctypes.c_uint64 * 3)(4, 4, 4)
    # NULL out handle
    assert L.flycoo_create(3, dims, 0, None, None, None, None, None) == 1
    # mode count outside the ABI range
    assert L.flycoo_create(9, dims, 0, None, None, None, None, ctypes.byref(h)) == 1
    # valid but not built
    assert L.flycoo_create(2, dims, 0, None, None, None, None, ctypes.byref(h)) == 8
    assert "not built" in native.flycoo_last_error()
    # zero-sized mode
    bad = (ctypes.c_uint64 * 3)(4, 0, 4)
    assert L.flycoo_create(3, bad, 0, None, None, None, None, ctypes.byref(h)) == 1
    # NULL data with nonzeros
    assert L.flycoo_create(3, dims, 5, None, None, None, None, ctypes.byref(h)) == 1
    # calls on a NULL handle
    assert L.flycoo_spmttkrp(None, 0, None, 0, 32, None, -1, None) == 1
    assert L.flycoo_remap(None, 0, None) == 1
    info = native.flycoo_info()
    assert L.flycoo_get_info(None, ctypes.byref(info)) == 1
    assert L.flycoo_timing_read(None, None, None) == 1
    L.flycoo_destroy(None)


def test_build_flags_target_sm103a():
    from paper_2309_09131_gb300 import build as B
    assert "arch=compute_103a,code=sm_103a" in B.ARCH
