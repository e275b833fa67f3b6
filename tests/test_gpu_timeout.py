"""The bounded waits: a look-back whose predecessor never publishes gives up,
raises FP_ERR_TIMEOUT in the device error word and lets the call finish (no
hang, no fault), and the next call is bit-exact again.  The missing publish is
made on purpose by the library's test hook (fp_debug_withhold_publish), never
by a device fault."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import dev_points

pytestmark = pytest.mark.gpu

TIMEOUT_BIT = 1 << 6


def test_withheld_publish_times_out_then_recovers(gpu_lib):
    fp = gpu_lib
    L = fp.load()
    # more than 2048 chunks: fp_distribute runs its radix passes, whose tiles look back
    n, g, T = 300_000, 7, 40
    pts_np = synth.uniform(n, 21)
    pts = dev_points(pts_np)
    cube = fp.fp_bounds(pts)
    counts = fp.fp_count(pts, cube, g)
    chunks, num_chunks, lut, offsets = fp.fp_merge_chunks(counts, g, T)
    torch.cuda.synchronize()
    assert int(num_chunks.item()) > 2048
    assert fp.get_device_error() == 0
    try:
        assert L.fp_debug_withhold_publish(3, 2000) == 0
        fp.fp_distribute(pts, cube, g, lut, offsets, num_chunks)
        torch.cuda.synchronize()             # returns: the wait is bounded
    finally:
        assert L.fp_debug_withhold_publish(0xFFFFFFFF, 0) == 0
    assert fp.get_device_error() & TIMEOUT_BIT
    assert fp.get_device_error() == 0        # cleared by the read
    # the next call, with every tile publishing, is exact
    dist, perm = fp.fp_distribute(pts, cube, g, lut, offsets, num_chunks)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    ocube = oracle.bounds(pts_np)
    ocounts = oracle.count(pts_np, ocube, g)
    _, olut, ooff = oracle.merge(ocounts, g, T)
    _, operm = oracle.distribute(pts_np, ocube, g, olut, ooff)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), operm)
