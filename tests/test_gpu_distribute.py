"""fp_distribute_cells at every chunk count around the boundaries of its paths
(with a 16-byte aligned cells array: 1..512 chunks the counting pass and the
sweep with per-warp histograms, 513..4096 the counting pass and the sweep that
sorts each tile, more the radix passes; without: 257..2048 the segmented sweeps,
else the radix passes), with a ragged last tile, against the
oracle's stable scatter given the same cell -> chunk table and offsets
(the paper's distribution, Sec. 4.4, is defined for any such table).  A cells
array that is not 16-byte aligned takes the paths without the sweep and gives
the same bytes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_points_equal, dev_points

pytestmark = pytest.mark.gpu

G = 7
N = 300_001   # 73 full tiles of 4096 points and a ragged one


@pytest.fixture(scope="module")
def cloud(gpu_lib):
    fp = gpu_lib
    pts_np = synth.uniform(N, 31)
    pts = dev_points(pts_np)
    cube = fp.fp_bounds(pts)
    want_cube = oracle.bounds(pts_np)
    cells_np = oracle.point_keys(pts_np, want_cube, G).astype(np.uint32)
    return fp, pts_np, pts, cube, want_cube, cells_np


def table(cells_np, K):
    """A cell -> chunk table with K chunks over the Morton order of the cells
    (every chunk occupied), and the chunk offsets of these points."""
    ncell = 1 << (3 * G)
    lut = ((np.arange(ncell, dtype=np.uint64) * K) >> (3 * G)).astype(np.uint32)
    counts = np.bincount(lut[cells_np], minlength=K).astype(np.uint64)
    assert (counts > 0).all()
    offsets = np.zeros(K + 1, np.uint64)
    offsets[1:] = np.cumsum(counts)
    return lut, offsets


@pytest.mark.parametrize("K", [1, 2, 255, 256, 257, 511, 512, 513, 2048, 2049, 3080, 4096, 4097])
@pytest.mark.parametrize("aligned", [True, False])
def test_distribute_cells_chunk_counts(cloud, K, aligned):
    fp, pts_np, pts, cube, want_cube, cells_np = cloud
    lut, offsets = table(cells_np, K)
    want_out, want_perm = oracle.distribute(pts_np, want_cube, G, lut, offsets)
    dev = pts.device
    lut_t = torch.from_numpy(lut.view(np.int32)).to(dev)
    off_t = torch.from_numpy(offsets.view(np.int64)).to(dev)
    num_t = torch.tensor([K], dtype=torch.int32, device=dev)
    if aligned:
        cells_t = torch.from_numpy(cells_np.view(np.int32)).to(dev)
    else:   # a view 4 bytes into a larger buffer
        big = torch.zeros(N + 4, dtype=torch.int32, device=dev)
        big[1:N + 1] = torch.from_numpy(cells_np.view(np.int32)).to(dev)
        cells_t = big[1:N + 1]
        assert cells_t.data_ptr() % 16 != 0
    out, perm = fp.fp_distribute_cells(pts, cells_t, cube, G, lut_t, off_t, num_t)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert_points_equal(out, want_out)
    out2, _ = fp.fp_distribute_cells(pts, cells_t, cube, G, lut_t, off_t, num_t, with_perm=False)
    assert_points_equal(out2, want_out)
    assert fp.get_device_error() == 0


def test_distribute_cells_small_clouds(gpu_lib):
    """Clouds of one partial tile and of exactly one full tile."""
    fp = gpu_lib
    for n, K in ((1, 1), (17, 3), (4095, 40), (4096, 512), (4097, 300), (4097, 1000), (8193, 3000)):
        pts_np = synth.uniform(n, 40 + n)
        pts = dev_points(pts_np)
        cube = fp.fp_bounds(pts)
        want_cube = oracle.bounds(pts_np)
        cells_np = oracle.point_keys(pts_np, want_cube, G).astype(np.uint32)
        ncell = 1 << (3 * G)
        # chunks by rank of the occupied cells, so that every one of the K chunks holds points
        occ = np.unique(cells_np)
        K = min(K, len(occ))
        lut = np.full(ncell, 0, np.uint32)
        rank = (np.arange(len(occ)) * K) // len(occ)
        lut[occ] = rank.astype(np.uint32)
        counts = np.bincount(lut[cells_np], minlength=K).astype(np.uint64)
        offsets = np.zeros(K + 1, np.uint64)
        offsets[1:] = np.cumsum(counts)
        want_out, want_perm = oracle.distribute(pts_np, want_cube, G, lut, offsets)
        dev = pts.device
        out, perm = fp.fp_distribute_cells(pts, torch.from_numpy(cells_np.view(np.int32)).to(dev), cube, G,
                                           torch.from_numpy(lut.view(np.int32)).to(dev),
                                           torch.from_numpy(offsets.view(np.int64)).to(dev),
                                           torch.tensor([K], dtype=torch.int32, device=dev))
        torch.cuda.synchronize()
        assert fp.get_device_error() == 0, n
        assert np.array_equal(perm[:n].cpu().numpy().view(np.uint32), want_perm), n
        assert_points_equal(out, want_out)
