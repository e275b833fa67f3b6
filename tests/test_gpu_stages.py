"""Parity of the CUDA stages bounds, preview, count, merge and distribute with
the CPU oracle, element by element, bit-exact (integer and index work)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_points_equal, cube_np, dev_points, host_points

pytestmark = pytest.mark.gpu


def cloud(kind, n, seed):
    if kind == "uniform":
        return synth.uniform(n, seed)
    if kind == "lidar":
        return synth.lidar(n, seed)
    if kind == "dups":
        base = synth.uniform(max(1, n // 50), seed, bits=6)
        idx = (np.arange(n) * 7919) % len(base)
        return base[idx]
    if kind == "extremes":
        a = synth.uniform(n, seed, bits=32)
        a["x"][0], a["x"][min(1, n - 1)] = -2**31, 2**31 - 1
        return a
    raise ValueError(kind)


CASES = [
    ("uniform", 1_000_000, 1, 7, 100_000),     # the 1M-point uniform workload
    ("uniform", 300_001, 5, 7, 2_000),         # ragged tail, 512 chunks: one sweep with chunk digits
    ("lidar", 400_000, 2, 7, 1_000),           # 1409 chunks: one sweep with chunk digits
    ("uniform", 2_000_003, 12, 7, 1_000),      # 4096 chunks: two radix passes
    ("lidar", 50_000, 3, 7, 1),                # every cell its own chunk
    ("dups", 40_000, 4, 3, 50),
    ("extremes", 8_193, 6, 7, 100),
    ("uniform", 4_096, 7, 2, 10),
    ("uniform", 1, 8, 7, 100),
    ("uniform", 0, 9, 7, 100),
]


@pytest.mark.parametrize("kind,n,seed,g,T", CASES)
def test_stages_match_oracle(gpu_lib, kind, n, seed, g, T):
    fp = gpu_lib
    pts_np = cloud(kind, n, seed)
    pts = dev_points(pts_np)
    # bounds (fused and alone) and preview
    cube = fp.fp_bounds(pts)
    cube2, prev, prev_n = fp.fp_bounds_decimate(pts, 0, 16)
    prev3, prev3_n = fp.fp_decimate(pts, 0, 16)
    want_cube = oracle.bounds(pts_np)
    assert cube_np(cube).tobytes() == want_cube.tobytes()
    assert cube_np(cube2).tobytes() == want_cube.tobytes()
    want_prev, _ = oracle.decimate(pts_np, 0, 16)
    assert int(prev_n.item()) == len(want_prev) == int(prev3_n.item())
    assert_points_equal(prev, want_prev, len(want_prev))
    assert_points_equal(prev3, want_prev, len(want_prev))
    # count grid
    counts = fp.fp_count(pts, cube, g)
    want_counts = oracle.count(pts_np, want_cube, g)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), want_counts)
    # chunks
    chunks, num, lut, offsets = fp.fp_merge_chunks(counts, g, T)
    want_chunks, want_lut, want_off = oracle.merge(want_counts, g, T)
    K = int(num.item())
    assert K == len(want_chunks)
    got_chunks = fp.chunks_to_host(chunks, num)
    assert got_chunks.tobytes() == want_chunks.tobytes()
    assert np.array_equal(lut.cpu().numpy().view(np.uint32), want_lut)
    assert np.array_equal(offsets[:K + 1].cpu().numpy().view(np.uint64), want_off)
    # distribute
    out, perm = fp.fp_distribute(pts, cube, g, lut, offsets, num)
    want_out, want_perm = oracle.distribute(pts_np, want_cube, g, want_lut, want_off)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert_points_equal(out, want_out)
    out2, _ = fp.fp_distribute(pts, cube, g, lut, offsets, num, with_perm=False)
    assert_points_equal(out2, want_out)
    # the same two stages with the cells handed from the count to the distribution
    counts3, cells = fp.fp_count_cells(pts, cube, g)
    assert np.array_equal(counts3.cpu().numpy().view(np.uint32), want_counts)
    got_cells = cells[:n].cpu().numpy().view(np.uint32)
    if n <= 400_000:   # the oracle's cell of every point
        assert np.array_equal(got_cells, oracle.point_keys(pts_np, want_cube, g).astype(np.uint32))
    else:              # every cell as often as the oracle counts it
        assert np.array_equal(np.bincount(got_cells, minlength=1 << (3 * g)), want_counts)
    out4, perm4 = fp.fp_distribute_cells(pts, cells, cube, g, lut, offsets, num)
    assert np.array_equal(perm4.cpu().numpy().view(np.uint32), want_perm)
    assert_points_equal(out4, want_out)
    out5, _ = fp.fp_distribute_cells(pts, cells, cube, g, lut, offsets, num, with_perm=False)
    assert_points_equal(out5, want_out)
    assert fp.get_device_error() == 0


def test_preview_first_index_and_modulus(gpu_lib):
    fp = gpu_lib
    pts_np = synth.uniform(100_000, 12)
    pts = dev_points(pts_np)
    for first, m in ((0, 1), (12345, 16), (2**40, 7), (999, 1000)):
        out, cnt = fp.fp_decimate(pts, first, m)
        want, _ = oracle.decimate(pts_np, first, m)
        assert int(cnt.item()) == len(want)
        assert_points_equal(out, want, len(want))


def test_count_accumulate_over_pieces(gpu_lib):
    fp = gpu_lib
    pts_np = synth.lidar(200_000, 13)
    pts = dev_points(pts_np)
    cube = fp.fp_bounds(pts)
    counts = fp.fp_count(pts[:70_000], cube, 7)
    fp.fp_count(pts[70_000:], cube, 7, counts=counts, accumulate=True)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), oracle.count(pts_np, oracle.bounds(pts_np), 7))


def test_preview_capacity_is_reported(gpu_lib):
    fp = gpu_lib
    pts = dev_points(synth.uniform(50_000, 14))
    fp.get_device_error(clear=True)
    out = torch.empty((10, 4), dtype=torch.int32, device="cuda")
    _, cnt = fp.fp_decimate(pts, 0, 16, out=out)
    assert int(cnt.item()) > 10
    assert fp.get_device_error(clear=True) & (1 << 9)
