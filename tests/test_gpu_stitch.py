"""The stitch at the shape of the 1B-point uniform workload, against the oracle
in full: uniform points, L_max = 8, 512 chunks of level 3, and the nodes above
the chunks (levels 0-2) keeping a large share of the points, merged across
chunks in original-index order (Sec. 4.4: the local octrees are stitched into
the global one).  Every node field and every point of the final layout,
including every point kept by a stitch node, is compared element by element;
the full-size tests can only check these by properties."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_build_matches_oracle, dev_points

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CASES = [
    # n, seed, T, C: 512 chunks of level 3 (n / 8^3 <= T < n / 8^2)
    # the 1B tree scaled down: chunks inner, leaves at level 5 (n / 8^5 <= C < n / 8^4)
    (8_000_000, 31, 50_000, 1_000),
    # node capacity of the 1B workload (C = 5e4): chunks are leaves, the stitch keeps most points
    (24_000_000, 32, 100_000, 50_000),
]


@pytest.mark.parametrize("n,seed,T,C", CASES)
def test_stitch_of_the_1B_shape_matches_oracle(gpu_lib, n, seed, T, C):
    fp = gpu_lib
    g, s, lmax = 7, 7, 8
    pts_np = synth.uniform(n, seed)
    prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    r = fp.build_octree(dev_points(pts_np), prm)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    assert int(r["num_chunks"].item()) == 512
    want = oracle.build_all(pts_np, oracle.params(g, s, lmax, 16, T, C))
    nodes = want["nodes"]
    stitch = nodes["level"] < 3
    assert stitch.sum() == 1 + 8 + 64
    kept_above = int(nodes["n_own"][stitch].sum())
    assert kept_above > n // 10, "the stitch nodes keep a large share of the points"
    M = int(r["num_nodes"].item())
    assert_build_matches_oracle(want, cube=r["cube"], nodes=r["nodes"][:M], final=r["final"],
                                final_perm=r["final_perm"])
    # the owner of every distributed point, the stitch nodes' included
    own_of_index = np.empty(n, np.int64)
    for k, nd in enumerate(nodes):
        own_of_index[want["final_perm"][int(nd["first"]):int(nd["first"]) + int(nd["n_own"])]] = k
    perm = r["perm"].cpu().numpy().view(np.uint32)
    assert np.array_equal(r["owner"].cpu().numpy().view(np.uint32), own_of_index[perm])
