"""fp_bounds_decimate_static: the bounds + preview pass for callers that cannot
allocate device memory (for instance a host application whose device memory
belongs to another allocator, or a real-time loop that must not wait on one).
It uses scratch held inside the library instead of a caller workspace; its
results must equal those of fp_bounds_decimate, bit for bit, call after call."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import dev_points

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
    assert fp.get_device_error() == 0


def test_static_scratch_rejects_oversized_input(gpu_lib):
    fp = gpu_lib
    f = _static_fn(fp)
    dummy = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    cube = torch.zeros(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = f(fp._ptr(dummy), (1 << 27) + 1, fp._ptr(cube), 0, 16, fp._ptr(dummy), 4, fp._ptr(cnt), None)
    assert rc == 3   # FP_ERR_TOO_LARGE, rejected on the host before any launch
