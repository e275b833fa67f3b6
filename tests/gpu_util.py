"""Helpers of the GPU parity tests: run the CUDA path through the C-ABI binding
and bring results to the host in the oracle's record formats."""
import numpy as np
import torch

import oracle


def dev_points(pts_np):
    from paper_2302_05002_gb300 import fastpoints as fp
    return fp.as_points(pts_np, "cuda")


def host_points(t):
    a = t.detach().cpu().contiguous().numpy()
    return a.view(np.uint8).reshape(-1, 16).copy().view(oracle.POINT).reshape(-1)


def cube_np(cube_t):
    return cube_t.detach().cpu().numpy().view(np.uint8).copy().view(oracle.CUBE)


def assert_points_equal(got_t, want_np, count=None):
    got = host_points(got_t)
    if count is not None:
        got = got[:count]
    assert len(got) == len(want_np), (len(got), len(want_np))
    if len(want_np):
        g = got.view(np.uint32).reshape(-1, 4)
        w = np.ascontiguousarray(want_np).view(np.uint32).reshape(-1, 4)
        bad = np.flatnonzero((g != w).any(axis=1))
        assert bad.size == 0, "first mismatch at %d of %d" % (bad[0], len(want_np))
