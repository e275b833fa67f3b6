"""Parity of fp_build_chunk_octree and fp_subsample with the CPU oracle: node
table, leaf-grouped points, LOD owner of every point and the final layout,
bit-exact, across workloads and parameters (several tiles, ragged tails,
cells larger than one shared-memory piece, deep subtrees, duplicates)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_points_equal, dev_points

pytestmark = pytest.mark.gpu

NODE_FIELDS = ["key", "level", "count", "n_own", "n_desc", "child_mask", "is_leaf", "leaf_first", "first"]


def cloud(kind, n, seed):
    if kind == "uniform":
        return synth.uniform(n, seed)
    if kind == "lidar":
        return synth.lidar(n, seed)
    if kind == "dups":
        base = synth.uniform(max(1, n // 40), seed, bits=9)
        return base[(np.arange(n) * 7919) % len(base)]
    if kind == "clustered":      # one dense blob inside a sparse cube
        a = synth.uniform(n, seed)
        k = n // 2
        a["x"][:k] = 500_000 + (a["x"][:k] & 1023)
        a["y"][:k] = 500_000 + (a["y"][:k] & 1023)
        a["z"][:k] = 500_000 + (a["z"][:k] & 1023)
        return a
    raise ValueError(kind)


def run_case(fp, pts_np, g, s, lmax, T, C):
    prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    pts = dev_points(pts_np)
    r = fp.build_octree(pts, prm)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    oprm = oracle.params(g, s, lmax, 16, T, C)
    want = oracle.build_all(pts_np, oprm)
    perm = r["perm"].cpu().numpy().view(np.uint32)
    assert np.array_equal(perm, want["perm"])
    nodes = fp.nodes_to_host(r["nodes"], r["num_nodes"])
    assert len(nodes) == len(want["nodes"]), (len(nodes), len(want["nodes"]))
    for f in NODE_FIELDS:
        if not np.array_equal(nodes[f], want["nodes"][f]):
            bad = np.flatnonzero(nodes[f] != want["nodes"][f])[0]
            raise AssertionError("node field %s differs first at node %d: got %s want %s" %
                                 (f, bad, nodes[bad], want["nodes"][bad]))
    assert np.array_equal(r["leaf_perm"].cpu().numpy().view(np.uint32), want["leaf_perm"])
    assert_points_equal(r["leaf_pts"], want["leaf_pts"])
    # owner of every distributed point
    own_of_index = np.empty(len(pts_np), np.int64)
    for k, nd in enumerate(want["nodes"]):
        own_of_index[want["final_perm"][int(nd["first"]):int(nd["first"]) + int(nd["n_own"])]] = k
    got_owner = r["owner"].cpu().numpy().view(np.uint32)
    assert np.array_equal(got_owner, own_of_index[perm])
    assert np.array_equal(r["final_perm"].cpu().numpy().view(np.uint32), want["final_perm"])
    assert_points_equal(r["final"], want["final_pts"])
    return want


def chunk_subtree_sizes(want):
    """Nodes in the subtree of every chunk's node (the digits of the chunk in the
    chunk-by-chunk scatter of the leaf grouping; one more in the owner layout)."""
    nodes = want["nodes"]
    sizes = []
    for c in want["chunks"]:
        idx = np.flatnonzero((nodes["key"] == c["key"]) & (nodes["level"] == c["level"]))
        assert len(idx) == 1, "every chunk is a node of the tree"
        sizes.append(int(nodes["n_desc"][idx[0]]) + 1)
    return np.array(sizes)


CASES = [
    # kind, n, seed, g, s, lmax, T, C
    ("uniform", 1_000_000, 1, 7, 7, 15, 100_000, 20_000),     # the 1M-point uniform workload
    ("uniform", 200_003, 2, 7, 7, 8, 50_000, 5_000),
    ("lidar", 300_000, 3, 7, 7, 15, 10_000, 2_000),          # big cells, deep subtrees
    ("lidar", 100_000, 4, 4, 5, 12, 3_000, 300),
    ("clustered", 120_000, 5, 5, 6, 16, 4_000, 500),         # one dense blob: split tree, pieces
    ("dups", 50_000, 6, 3, 3, 9, 1_000, 40),                 # identical points: oversized leaves
    ("uniform", 2_000_000, 14, 5, 6, 8, 50_000, 2_000),      # leaves above the cells: level tables, 4 levels
    ("uniform", 1_500_000, 15, 5, 5, 9, 40_000, 2_000),      # ... 3 levels, many tables per unit
    ("uniform", 5_000, 7, 2, 2, 20, 100, 10),
    ("uniform", 1, 8, 7, 7, 15, 100, 10),
    ("uniform", 3, 9, 1, 1, 21, 1, 1),
]

# Chunk subtrees of every width the chunk-by-chunk scatter handles: up to 256
# digits, up to 2048 (with a chunk of many tiles and owners above the chunks),
# and beyond 2048, where the whole-array sort runs instead.
WIDTH_CASES = [
    # kind, n, seed, g, s, lmax, T, C, widest chunk subtree: (lower, upper]
    ("lidar", 300_000, 12, 5, 5, 14, 60_000, 300, (256, 2047)),
    ("uniform", 200_000, 11, 4, 4, 9, 200_000, 2_000, (256, 2047)),
    ("clustered", 200_000, 13, 5, 6, 16, 50_000, 150, (2047, 10 ** 9)),
    ("uniform", 300_000, 10, 3, 3, 10, 300_000, 200, (2047, 10 ** 9)),
]


@pytest.mark.parametrize("kind,n,seed,g,s,lmax,T,C,widest", WIDTH_CASES)
def test_octree_chunk_widths(gpu_lib, kind, n, seed, g, s, lmax, T, C, widest):
    want = run_case(gpu_lib, cloud(kind, n, seed), g, s, lmax, T, C)
    sizes = chunk_subtree_sizes(want)
    assert widest[0] < sizes.max() + 1 <= widest[1], sizes.max()


@pytest.mark.parametrize("kind,n,seed,g,s,lmax,T,C", CASES)
def test_octree_matches_oracle(gpu_lib, kind, n, seed, g, s, lmax, T, C):
    run_case(gpu_lib, cloud(kind, n, seed), g, s, lmax, T, C)


def test_result_does_not_depend_on_threshold(gpu_lib):
    fp = gpu_lib
    pts_np = synth.lidar(60_000, 11)
    pts = dev_points(pts_np)
    outs = []
    for T in (500, 1000, 20_000, 60_000):
        prm = fp.params(grid_log2=7, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=T, node_capacity=500)
        r = fp.build_octree(pts, prm)
        outs.append((fp.nodes_to_host(r["nodes"], r["num_nodes"]).tobytes(),
                     r["final_perm"].cpu().numpy().tobytes(), r["leaf_perm"].cpu().numpy().tobytes()))
    assert all(o == outs[0] for o in outs)


def test_repeatable(gpu_lib):
    fp = gpu_lib
    pts = dev_points(synth.lidar(80_000, 12))
    prm = fp.params(grid_log2=7, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=5_000, node_capacity=700)
    a = fp.build_octree(pts, prm)
    b = fp.build_octree(pts, prm)
    for k in ("nodes", "final", "final_perm", "leaf_pts", "owner"):
        assert torch.equal(a[k], b[k]), k
