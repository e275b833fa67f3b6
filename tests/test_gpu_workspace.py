"""Every stage stays inside the workspace fp_workspace_size() asks for.  Each call
gets a buffer of exactly that size followed by a canary region; the library may
carve only what the size query counted, so the canary must come back intact
(several cloud sizes with ragged last tiles, on every distribution path)."""
import pytest
import torch

import synth
from tests.gpu_util import dev_points

pytestmark = pytest.mark.gpu

CANARY = 1 << 20
FILL = 0xA5


def guarded(fp, stage, n, prm, dev):
    need = fp.workspace_size(stage, n, prm)
    buf = torch.full((need + CANARY,), FILL, dtype=torch.uint8, device=dev)
    return buf, need


def assert_canary(buf, need, what):
    torch.cuda.synchronize()
    bad = (buf[need:] != FILL).nonzero()
    assert bad.numel() == 0, "%s wrote %d bytes past its workspace (first at +%d)" % (
        what, bad.numel(), int(bad[0].item()))


@pytest.mark.parametrize("kind,n,T", [("lidar", 300_001, 20_000), ("uniform", 2_049, 1_000),
                                      ("uniform", 1_000_003, 300_000), ("lidar", 200_000, 300)])
def test_stages_stay_inside_their_workspace(gpu_lib, kind, n, T):
    fp = gpu_lib
    dev = torch.device("cuda")
    pts_np = synth.lidar(n, 51) if kind == "lidar" else synth.uniform(n, 52)
    pts = dev_points(pts_np)
    g = 7
    prm = fp.params(grid_log2=g, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=T,
                    node_capacity=min(2_000, T))
    fp.get_device_error(clear=True)

    def run(stage, stage_prm, f):
        buf, need = guarded(fp, stage, n, stage_prm, dev)
        out = f(buf)
        assert_canary(buf, need, stage)
        return out

    cube = run("bounds", None, lambda w: fp.fp_bounds(pts, ws=w))
    run("decimate", None, lambda w: fp.fp_decimate(pts, 0, 16, ws=w))
    run("bounds_decimate", None, lambda w: fp.fp_bounds_decimate(pts, 0, 16, ws=w))
    lvl = fp.params(grid_log2=6, sub_log2=6, max_level=6)
    run("preview_spatial", lvl, lambda w: fp.fp_preview_spatial(pts, cube, 6, ws=w))
    counts, cells = fp.fp_count_cells(pts, cube, g)
    merge_buf, merge_need = guarded(fp, "merge", 0, fp.params(grid_log2=g), dev)
    chunks, num_chunks, lut, offsets = fp.fp_merge_chunks(counts, g, T, ws=merge_buf)
    assert_canary(merge_buf, merge_need, "merge")
    dist, perm = run("distribute", fp.params(grid_log2=g),
                     lambda w: fp.fp_distribute(pts, cube, g, lut, offsets, num_chunks, ws=w))
    d2, p2 = run("distribute", fp.params(grid_log2=g),
                 lambda w: fp.fp_distribute_cells(pts, cells, cube, g, lut, offsets, num_chunks, ws=w))
    assert torch.equal(dist, d2) and torch.equal(perm, p2)
    nodes, num_nodes, leaf_pts, leaf_perm, owner = run(
        "octree", prm, lambda w: fp.fp_build_chunk_octree(dist, perm, cube, chunks, num_chunks, offsets, counts, prm,
                                                          ws=w))
    run("subsample", prm, lambda w: fp.fp_subsample(nodes, num_nodes, dist, perm, owner, chunks, num_chunks, offsets,
                                                    prm, ws=w))
    assert fp.get_device_error(clear=True) == 0
