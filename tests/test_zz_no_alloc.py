"""fp_bounds_decimate_static: the bounds + preview pass for callers that cannot
allocate device memory (for instance a host application whose device memory
belongs to another allocator, or a real-time loop that must not wait on one).
It uses scratch held inside the library instead of a caller workspace; its
results must equal those of fp_bounds_decimate, bit for bit, call after call."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_points_equal, cube_np, dev_points

pytestmark = pytest.mark.gpu


def _static_fn(fp):
    f = fp.load().fp_bounds_decimate_static
    p, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    f.restype = ctypes.c_int
    f.argtypes = [p, u64, p, u64, u32, p, u64, p, p]
    return f


def test_static_scratch_matches_workspace_version(gpu_lib):
    fp = gpu_lib
    f = _static_fn(fp)
    stream = torch.cuda.current_stream()
    # two calls in a row, different sizes, the second reusing the library's scratch
    for seed, n, first in ((1, 3_000_000, 0), (2, 777_777, 12345)):
        pts = dev_points(synth.lidar(n, seed))
        cube_ref, prev_ref, cnt_ref = fp.fp_bounds_decimate(pts, first, 16)
        cube = torch.zeros(8, dtype=torch.int32, device="cuda")
        out = torch.zeros_like(prev_ref)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = f(fp._ptr(pts), n, fp._ptr(cube), first, 16, fp._ptr(out), out.shape[0], fp._ptr(cnt),
               ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(cube, cube_ref)
        k = int(cnt_ref.item())
        assert int(cnt.item()) == k
        assert torch.equal(out[:k], prev_ref[:k])
        # and against the oracle directly
        pts_np = synth.lidar(n, seed)
        assert cube_np(cube).tobytes() == oracle.bounds(pts_np).tobytes()
        want, _ = oracle.decimate(pts_np, first, 16)
        assert_points_equal(out, want, count=k)
    assert fp.get_device_error() == 0


def test_static_scratch_empty_and_capacity(gpu_lib):
    fp = gpu_lib
    f = _static_fn(fp)
    stream = torch.cuda.current_stream()
    S = ctypes.c_void_p(stream.cuda_stream)
    cube = torch.full((8,), 7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), 99, dtype=torch.int64, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    # an empty cloud: count 0, cube side 0, nothing written
    assert f(None, 0, fp._ptr(cube), 0, 16, fp._ptr(out), out.shape[0], fp._ptr(cnt), S) == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
    assert cube_np(cube)["S"][0] == 0
    assert fp.get_device_error() == 0
    # more kept points than out_cap: the count is the full count, the first out_cap
    # points are written, nothing beyond them, and the capacity bit is raised
    n, cap = 100_000, 1000
    pts_np = synth.uniform(n, 5)
    pts = dev_points(pts_np)
    out = torch.full((cap + 16, 4), -1, dtype=torch.int32, device="cuda")
    assert f(fp._ptr(pts), n, fp._ptr(cube), 0, 16, fp._ptr(out), cap, fp._ptr(cnt), S) == 0
    torch.cuda.synchronize()
    want, _ = oracle.decimate(pts_np, 0, 16)
    assert len(want) > cap
    assert int(cnt.item()) == len(want)
    assert_points_equal(out, want[:cap], count=cap)
    assert bool((out[cap:] == -1).all())
    assert fp.get_device_error() == 1 << 9   # FP_ERR_CAPACITY, cleared by the read
    assert fp.get_device_error() == 0


def test_static_scratch_rejects_oversized_input(gpu_lib):
    fp = gpu_lib
    f = _static_fn(fp)
    dummy = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    cube = torch.zeros(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = f(fp._ptr(dummy), (1 << 27) + 1, fp._ptr(cube), 0, 16, fp._ptr(dummy), 4, fp._ptr(cnt), None)
    assert rc == 3   # FP_ERR_TOO_LARGE, rejected on the host before any launch
