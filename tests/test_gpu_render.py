"""Headless rendering against the oracle, bit-exact: the nodes a camera draws
(frustum and screen-size refinement over the node table) and the framebuffer
of their points (nearest point per pixel), for perspective cameras outside,
inside and facing away from the cloud, and an orthographic one."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import dev_points

pytestmark = pytest.mark.gpu


def centre_and_size(pts_np):
    lo = np.array([pts_np[a].min() for a in "xyz"], np.float64)
    hi = np.array([pts_np[a].max() for a in "xyz"], np.float64)
    return (lo + hi) / 2, float((hi - lo).max())


def cameras(fp, pts_np, W, H):
    c, size = centre_and_size(pts_np)
    out = []
    out.append(("outside", fp.view_projection(c + np.array([0.9, -1.2, 0.7]) * size, c, fovy_deg=50,
                                              aspect=W / H, near=size * 0.01, far=size * 10), 40.0))
    out.append(("inside", fp.view_projection(c + np.array([0.05, 0.02, 0.01]) * size, c + np.array([1, 0.3, 0]) * size,
                                             fovy_deg=70, aspect=W / H, near=size * 1e-4, far=size * 4), 25.0))
    out.append(("away", fp.view_projection(c + np.array([3.0, 0, 0]) * size, c + np.array([6.0, 0, 0]) * size,
                                           aspect=W / H, near=1.0, far=size * 10), 10.0))
    m = np.zeros(16, np.float32)   # orthographic over the bounding square
    lo = c - size / 2
    m[0], m[3] = 2 / size, -1 - 2 * lo[0] / size
    m[5], m[7] = 2 / size, -1 - 2 * lo[1] / size
    m[10], m[11], m[15] = 1 / size, -lo[2] / size, 1
    out.append(("ortho", m, 4.0))
    return out


def render_case(fp, pts_np, prm, W, H):
    pts = dev_points(pts_np)
    r = fp.build_octree(pts, prm)
    nodes_h = fp.nodes_to_host(r["nodes"], r["num_nodes"])
    M = len(nodes_h)
    cube = oracle.bounds(pts_np)
    fin = r["final"].cpu().numpy().view(np.uint8).reshape(-1, 16).copy().view(oracle.POINT).reshape(-1)
    nodes_d = r["nodes"][:M].contiguous()
    for name, m, minpx in cameras(fp, pts_np, W, H):
        cam = fp.camera(m, W, H, minpx)
        ids, nsel, npts = fp.fp_select_nodes(nodes_d, r["num_nodes"], r["cube"], cam)
        fb = fp.fp_rasterize(nodes_d, ids, nsel, r["final"], cam)
        torch.cuda.synchronize()
        assert fp.get_device_error() == 0
        ocam = oracle.camera(m, W, H, minpx)
        want_sel = oracle.render_select(nodes_h, cube, ocam)
        k = int(nsel.item())
        got_sel = ids[:k].cpu().numpy().view(np.uint32)
        assert np.array_equal(got_sel, want_sel), name
        assert int(npts.item()) == int(nodes_h["n_own"][want_sel].astype(np.int64).sum())
        want_fb = oracle.rasterize(nodes_h, want_sel, fin, ocam)
        got_fb = fb.cpu().numpy().view(np.uint64)
        bad = np.flatnonzero(got_fb.reshape(-1) != want_fb.reshape(-1))
        assert bad.size == 0, "%s: %d pixels differ, first %d" % (name, bad.size, bad[0])
        if name == "away":
            assert k == 0 and np.all(want_fb == np.uint64(0xFFFFFFFFFFFFFFFF))
        else:
            assert k > 0 and np.any(want_fb != np.uint64(0xFFFFFFFFFFFFFFFF))


@pytest.mark.parametrize("kind,n,seed,W,H", [("lidar", 400_000, 61, 640, 360), ("uniform", 150_000, 62, 333, 201)])
def test_render_matches_oracle(gpu_lib, kind, n, seed, W, H):
    fp = gpu_lib
    pts_np = synth.lidar(n, seed) if kind == "lidar" else synth.uniform(n, seed)
    prm = fp.params(grid_log2=6, sub_log2=7, max_level=14, decim_modulus=16, chunk_threshold=20_000,
                    node_capacity=1_500)
    render_case(fp, pts_np, prm, W, H)


def test_render_rejects_bad_camera(gpu_lib):
    fp = gpu_lib
    r = fp.build_octree(dev_points(synth.uniform(1000, 63)), fp.params())
    cam = fp.camera(np.eye(4, dtype=np.float32).reshape(16), 0, 10, 1.0)
    with pytest.raises(fp.FastPointsError):
        fp.fp_select_nodes(r["nodes"], r["num_nodes"], r["cube"], cam)
