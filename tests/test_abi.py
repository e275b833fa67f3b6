"""The C-ABI library builds, loads without a GPU and exports every function the
header declares; host-side argument checks reject bad calls before any launch."""
import ctypes

import pytest

from paper_2302_05002_gb300 import fastpoints as fp


def test_header_declares_the_boundary():
    names = fp.declared_functions()
    for n in ["fp_bounds", "fp_decimate", "fp_count", "fp_merge_chunks", "fp_distribute",
              "fp_build_chunk_octree", "fp_subsample", "fp_workspace_size", "fp_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = fp.load()
    for name in fp.declared_functions():
        assert hasattr(lib, name), name


def test_status_strings():
    lib = fp.load()
    assert lib.fp_status_string(0) == b"ok"
    assert b"workspace" in lib.fp_status_string(5)


def test_host_argument_checks_without_gpu():
    lib = fp.load()
    # null cube pointer: rejected on the host before anything touches a device
    assert lib.fp_bounds(None, 0, None, None, 0, None) == 1
    # too many points
    assert lib.fp_bounds(ctypes.c_void_p(16), 1 << 30, ctypes.c_void_p(16), None, 0, None) == 3
    # misaligned point array
    assert lib.fp_bounds(ctypes.c_void_p(8), 5, ctypes.c_void_p(16), None, 0, None) == 2
    # unsupported grid
    assert lib.fp_count(ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 9, ctypes.c_void_p(16), 0, None, 0, None) == 8
    bad = fp.params(grid_log2=7, sub_log2=7, max_level=16)     # max_level + sub_log2 > 22
    args = [None, None, 0] + [None] * 5 + [ctypes.byref(bad), None, 0, None, None, None, None, None, 0, None]
    assert lib.fp_build_chunk_octree(*args) == 8
