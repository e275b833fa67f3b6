"""Preview variants against the oracle, bit-exact: the spatially constrained
random sampler (one point per occupied cell: the smallest index hash, Sec. 6)
and the point-budget modulus of the uniform preview (Sec. 5)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_points_equal, dev_points

pytestmark = pytest.mark.gpu


def cloud(kind, n, seed):
    return synth.lidar(n, seed) if kind == "lidar" else synth.uniform(n, seed)


@pytest.mark.parametrize("kind,n,seed,level,first", [
    ("lidar", 300_000, 31, 7, 0),
    ("uniform", 1_000_000, 32, 5, 0),
    ("uniform", 123_457, 33, 3, 1 << 33),   # ragged tail, global indices of a later piece
    ("lidar", 50_000, 34, 1, 17),
    ("uniform", 1, 35, 7, 0),
    ("uniform", 0, 36, 4, 0),
])
def test_spatial_matches_oracle(gpu_lib, kind, n, seed, level, first):
    fp = gpu_lib
    pts_np = cloud(kind, n, seed)
    pts = dev_points(pts_np) if n else torch.empty((0, 4), dtype=torch.int32, device="cuda")
    cube = fp.fp_bounds(pts)
    out, cnt = fp.fp_preview_spatial(pts, cube, level, first)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    want, _ = oracle.preview_spatial(pts_np, oracle.bounds(pts_np), level, first)
    k = int(cnt.item())
    assert k == len(want)
    assert_points_equal(out[:k], want)


def test_spatial_capacity_is_reported(gpu_lib):
    fp = gpu_lib
    pts_np = cloud("uniform", 200_000, 37)
    pts = dev_points(pts_np)
    cube = fp.fp_bounds(pts)
    out = torch.empty((100, 4), dtype=torch.int32, device="cuda")
    _, cnt = fp.fp_preview_spatial(pts, cube, 4, 0, out=out)
    torch.cuda.synchronize()
    want, _ = oracle.preview_spatial(pts_np, oracle.bounds(pts_np), 4)
    assert int(cnt.item()) == len(want) > 100
    assert fp.get_device_error() & (1 << 9)        # capacity bit
    assert_points_equal(out, want[:100])          # the first kept points are written


def test_spatial_rejects_bad_level(gpu_lib):
    fp = gpu_lib
    pts = dev_points(cloud("uniform", 1000, 38))
    cube = fp.fp_bounds(pts)
    with pytest.raises(fp.FastPointsError):
        fp.fp_preview_spatial(pts, cube, 8)


@pytest.mark.parametrize("n,target", [(1_000_000, 50_000), (777_777, 100_000), (300_000, 1_000_000)])
def test_budget_modulus_preview(gpu_lib, n, target):
    fp = gpu_lib
    m = fp.fp_preview_modulus(n, target)
    assert m == oracle.preview_modulus(n, target)
    pts_np = cloud("uniform", n, 39)
    out, cnt = fp.fp_decimate(dev_points(pts_np), 0, m)
    torch.cuda.synchronize()
    want, _ = oracle.decimate(pts_np, 0, m)
    assert int(cnt.item()) == len(want)
    assert_points_equal(out[:len(want)], want)
    assert abs(len(want) - n / m) < 6 * np.sqrt(n / m) + 1   # a binomial count around the budget
