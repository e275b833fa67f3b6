"""Host-side helpers of the binding, no GPU: the output bounds the binding sizes
buffers with, checked against what the oracle produces; the preview modulus rule;
the view-projection matrix."""
import numpy as np
import pytest

import oracle
import synth
from paper_2302_05002_gb300 import fastpoints as fp


def test_preview_modulus_closed_form():
    # a preview of about `target` points: every m-th hash class, m = max(1, ceil(n / target))
    for n in [0, 1, 2, 15, 16, 17, 999_999, 1_000_000, 1_000_001, 10 ** 9]:
        for target in [1, 7, 1_000_000]:
            assert fp.fp_preview_modulus(n, target) == max(1, -(-n // target)), (n, target)


@pytest.mark.parametrize("n,m,first", [(10, 2, 0), (1000, 16, 0), (100_000, 16, 12345), (200_000, 3, 7),
                                       (50_000, 1000, 0), (65_536, 1, 0)])
def test_preview_cap_holds_the_kept_points(n, m, first):
    # the hash rule keeps about n / m points; the buffer the binding allocates holds all of them
    kept, idx = oracle.decimate(synth.uniform(n, 1), first, m)
    assert len(kept) <= fp._preview_cap(n, m) <= n


CASES = [
    # kind, n, seed, g, s, lmax, T, C
    ("uniform", 20_000, 1, 4, 4, 10, 2_000, 50),
    ("uniform", 5_000, 2, 3, 3, 21 - 3, 100, 1),     # node capacity 1: every point its own leaf
    ("lidar", 30_000, 3, 5, 5, 14, 3_000, 40),
    ("uniform", 1, 4, 2, 2, 8, 1, 1),
]


@pytest.mark.parametrize("kind,n,seed,g,s,lmax,T,C", CASES)
def test_node_capacity_bound_covers_the_oracle_tree(kind, n, seed, g, s, lmax, T, C):
    pts = synth.uniform(n, seed) if kind == "uniform" else synth.lidar(n, seed)
    tree = oracle.octree_lod(pts, oracle.bounds(pts), oracle.params(g, s, lmax, 16, T, C))
    bound = fp.node_capacity_bound(n, fp.params(g, s, lmax, 16, T, C))
    assert len(tree["nodes"]) <= bound


def test_size_queries_grow_with_n():
    prm = fp.params()
    sizes = [(fp.node_capacity_bound(n, prm), fp.ooc_host_bytes(n, prm),
              fp.workspace_size("octree", n, prm), fp.workspace_size("subsample", n, prm))
             for n in (1, 1000, 10 ** 6, 10 ** 8)]
    for a, b in zip(sizes, sizes[1:]):
        assert all(y >= x for x, y in zip(a, b))
    # the out-of-core host store: points, indices, codes, owner ids and staging per point
    n = 10 ** 8
    assert fp.ooc_host_bytes(n, prm) >= 38 * n


def test_view_projection_maps_the_view_axis_to_the_centre():
    eye, target = np.array([10.0, -20.0, 5.0]), np.array([3.0, 4.0, 1.0])
    m = fp.view_projection(eye, target, fovy_deg=60.0, aspect=2.0, near=1.0, far=1e4).reshape(4, 4)

    def clip(p):
        return m.astype(np.float64) @ np.append(np.asarray(p, dtype=np.float64), 1.0)

    d = (target - eye) / np.linalg.norm(target - eye)
    for dist in (1.0, 50.0, 5_000.0):   # on the view axis: screen centre, depth in [0, w]
        c = clip(eye + dist * d)
        assert abs(c[0] / c[3]) < 1e-5 and abs(c[1] / c[3]) < 1e-5
        assert c[3] > 0 and 0.0 <= c[2] / c[3] <= 1.0 + 1e-6
    near, far = clip(eye + 1.0 * d), clip(eye + 1e4 * d)   # depth 0 at the near plane, 1 at the far one
    assert abs(near[2] / near[3]) < 1e-4 and abs(far[2] / far[3] - 1.0) < 1e-4
    assert clip(eye - 10.0 * d)[3] < 0                      # behind the eye
    # half the vertical field of view reaches the top edge of the screen
    up = np.cross(np.cross(d, [0.0, 0.0, 1.0]), d)
    up /= np.linalg.norm(up)
    top = clip(eye + 100.0 * d + 100.0 * np.tan(np.radians(30.0)) * up)
    assert abs(top[1] / top[3] - 1.0) < 1e-4
