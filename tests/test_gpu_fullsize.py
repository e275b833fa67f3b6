"""Parity at the benchmark's full sizes (100M-point LiDAR, 1B-point uniform),
through the same C-ABI calls and launch configuration the benchmark times.

* Whole-cloud outputs the oracle computes in one pass are compared in full:
  cube, preview, count grid, chunks, LUT, offsets, the distribution
  permutation.
* The octree is compared on sampled chunks.  Every node at or below a chunk's
  level, and the owner and leaf level of every point of the chunk, depend only
  on the chunk's points (cells at levels >= s >= g lie inside one level-g cell;
  an owner level at or below s collapses to the root either way) as long as
  every ancestor of the chunk stays inner, which holds when the chunk has more
  than C points.  So the oracle builds the tree of the chunk's points alone,
  with the whole cloud's cube, and the chunk's subtree, its leaf-grouped points,
  its final layout and its points' owner levels must match exactly.
* The rest is checked by properties that hold at any size: the final and
  leaf-grouped arrays are permutations of the cloud in node order with
  ascending original index inside each node, node counts add up, leaves obey
  the capacity rule.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import cube_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FULL = [
    # kind, n, seed, g, s, lmax, T, C  (the benchmark's 100M LiDAR and 1B uniform workloads)
    ("lidar", 100_000_000, 2, 7, 7, 15, 100_000, 20_000),
    ("uniform", 1_000_000_000, 3, 7, 7, 8, 5_000_000, 50_000),
]
BLOCK = 1 << 26


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def sampled_chunks(chunks, C, rng, k=4, spread=True):
    """The largest chunk above C points, plus (spread) the median and smallest
    of them, plus k random ones."""
    big = np.flatnonzero(chunks["count"] > C)
    assert big.size, "no chunk above the node capacity"
    order = big[np.argsort(chunks["count"][big], kind="stable")]
    pick = {int(order[-1])}
    if spread:
        pick.update((int(order[len(order) // 2]), int(order[0])))
    pick.update(int(x) for x in rng.choice(big, size=min(k, big.size), replace=False))
    return sorted(pick)


def node_index(nodes, level, key):
    idx = np.flatnonzero((nodes["level"] == level) & (nodes["key"] == key))
    assert idx.size == 1, (level, key, idx)
    return int(idx[0])


def check_chunk(fp, pts_np, cube, oprm, C, r, nodes, chunk, c_off, owner_dev, perm_np):
    """The chunk's subtree, leaf grouping, final layout and owners against the
    oracle's tree of the chunk's points alone."""
    lo, hi = int(c_off[0]), int(c_off[1])
    idx = perm_np[lo:hi].astype(np.int64)
    assert np.all(np.diff(idx) > 0), "distribution is not stable"
    pts_c = pts_np[idx]
    want = oracle.octree_lod(pts_c, cube, oprm)
    wn = want["nodes"]
    lev, key = int(chunk["level"]), int(chunk["key"])
    a = node_index(wn, lev, key)
    b = node_index(nodes, lev, key)
    m = int(wn["n_desc"][a]) + 1
    assert int(nodes["n_desc"][b]) + 1 == m
    gsub, wsub = nodes[b:b + m], wn[a:a + m]
    for f in ("key", "level", "count", "n_desc", "child_mask", "is_leaf", "n_own"):
        assert np.array_equal(gsub[f], wsub[f]), "chunk (%d, %d): node field %s" % (lev, key, f)
    assert np.array_equal(gsub["leaf_first"].astype(np.int64) - int(gsub["leaf_first"][0]),
                          wsub["leaf_first"].astype(np.int64) - int(wsub["leaf_first"][0]))
    # leaf-grouped points of the subtree
    l0, cnt = int(gsub["leaf_first"][0]), int(gsub["count"][0])
    wl0 = int(wsub["leaf_first"][0])
    got_leaf = u32(r["leaf_perm"][l0:l0 + cnt]).astype(np.int64)
    assert np.array_equal(got_leaf, idx[want["leaf_perm"][wl0:wl0 + cnt].astype(np.int64)])
    # final layout of every node of the subtree
    for k in range(m):
        no = int(gsub["n_own"][k])
        if no == 0:
            continue
        f0, w0 = int(gsub["first"][k]), int(wsub["first"][k])
        got = u32(r["final_perm"][f0:f0 + no]).astype(np.int64)
        assert np.array_equal(got, idx[want["final_perm"][w0:w0 + no].astype(np.int64)]), "node %d" % (b + k)
    # owner level of every point of the chunk
    _, _, own_lv = oracle.point_levels(pts_c, cube, oprm)
    got_owner = u32(owner_dev[lo:hi]).astype(np.int64)
    assert np.array_equal(nodes["level"][got_owner], own_lv)
    inside = own_lv >= lev
    assert np.all((got_owner[inside] >= b) & (got_owner[inside] < b + m))


def check_layout(fp, pts_dev, r, nodes, n, C, lmax):
    """Permutation, gather and node-order properties of the final and
    leaf-grouped arrays, on the device in blocks."""
    dev = pts_dev.device
    M = len(nodes)
    assert int(nodes["n_own"].astype(np.int64).sum()) == n
    first = np.concatenate([[0], np.cumsum(nodes["n_own"].astype(np.int64))[:-1]])
    assert np.array_equal(nodes["first"].astype(np.int64), first)
    # counts add up over children; leaves obey the capacity rule
    lvl = nodes["level"].astype(np.int64)
    cnt = nodes["count"].astype(np.int64)
    leaf = nodes["is_leaf"] != 0
    assert np.all(leaf == ((cnt <= C) | (lvl == lmax)))
    child_sum = np.zeros(M, np.int64)
    stack = []
    for i in range(M):   # parent of node i: the last open node one level up
        while stack and lvl[stack[-1]] >= lvl[i]:
            stack.pop()
        if stack:
            assert lvl[stack[-1]] == lvl[i] - 1
            child_sum[stack[-1]] += cnt[i]
        stack.append(i)
    assert np.array_equal(child_sum[~leaf], cnt[~leaf])
    assert int(cnt[0]) == n and lvl[0] == 0
    node_of_final = torch.repeat_interleave(torch.arange(M, device=dev, dtype=torch.int32),
                                            torch.from_numpy(nodes["n_own"].astype(np.int64)).to(dev))
    leaf_ids = np.flatnonzero(leaf)
    node_of_leaf = torch.repeat_interleave(torch.from_numpy(leaf_ids.astype(np.int32)).to(dev),
                                           torch.from_numpy(cnt[leaf_ids]).to(dev))
    for perm_key, pts_key, node_of in (("final_perm", "final", node_of_final), ("leaf_perm", "leaf_pts", node_of_leaf)):
        seen = torch.zeros(n, dtype=torch.uint8, device=dev)
        permt = r[perm_key][:n]
        for s0 in range(0, n, BLOCK):
            s1 = min(n, s0 + BLOCK)
            p = permt[s0:s1].long()
            seen[p] = 1
            assert torch.equal(r[pts_key][s0:s1], pts_dev[p]), "%s: points differ from the gather" % pts_key
            e = min(n, s1 + 1)
            q = permt[s0:e].long()
            nd = node_of[s0:e]
            same = nd[1:] == nd[:-1]
            assert bool(torch.all(~same | (q[1:] > q[:-1]))), "%s: not ascending inside a node" % perm_key
        assert bool(torch.all(seen == 1)), "%s is not a permutation" % perm_key
        del seen


def check_frame(fp, pts_np, r, nodes, cube):
    lo = np.array([pts_np[a].min() for a in "xyz"], np.float64)
    hi = np.array([pts_np[a].max() for a in "xyz"], np.float64)
    c, size = (lo + hi) / 2, float((hi - lo).max())
    m = fp.view_projection(c + np.array([0.45, -0.6, 0.25]) * size, c, fovy_deg=60, aspect=16 / 9,
                           near=size * 1e-3, far=size * 10)
    cam = fp.camera(m, 1920, 1080, 30.0)
    M = len(nodes)
    nd = r["nodes"][:M].contiguous()
    ids, nsel, _ = fp.fp_select_nodes(nd, r["num_nodes"], r["cube"], cam)
    fb = fp.fp_rasterize(nd, ids, nsel, r["final"], cam)
    torch.cuda.synchronize()
    ocam = oracle.camera(m, 1920, 1080, 30.0)
    want_sel = oracle.render_select(nodes, cube, ocam)
    k = int(nsel.item())
    assert np.array_equal(ids[:k].cpu().numpy().view(np.uint32), want_sel)
    fin = r["final"].cpu().numpy().view(np.uint8).reshape(-1, 16).copy().view(oracle.POINT).reshape(-1)
    assert np.array_equal(fb.cpu().numpy().view(np.uint64), oracle.rasterize(nodes, want_sel, fin, ocam))


@pytest.mark.parametrize("kind,n,seed,g,s,lmax,T,C", FULL)
def test_full_size(gpu_lib, kind, n, seed, g, s, lmax, T, C):
    fp = gpu_lib
    pts_np = synth.lidar(n, seed) if kind == "lidar" else synth.uniform(n, seed)
    pts = fp.as_points(pts_np, "cuda")
    prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    r = fp.build_octree(pts, prm)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    oprm = oracle.params(g, s, lmax, 16, T, C)

    # cube, preview, counts, chunks, offsets, distribution: the oracle in full
    cube = oracle.bounds(pts_np)
    assert cube_np(r["cube"]).tobytes() == cube.tobytes()
    prev, _ = oracle.decimate(pts_np, 0, 16)
    k = int(r["preview_count"].item())
    assert k == len(prev)
    got_prev = r["preview"][:k].cpu().numpy().view(np.uint32).reshape(-1, 4)
    assert np.array_equal(got_prev, np.ascontiguousarray(prev).view(np.uint32).reshape(-1, 4))
    del prev, got_prev
    counts = oracle.count(pts_np, cube, g)
    assert np.array_equal(u32(r["counts"]), counts)
    chunks, lut, offsets = oracle.merge(counts, g, T)
    K = int(r["num_chunks"].item())
    assert K == len(chunks)
    got_chunks = r["chunks"][:K].cpu().numpy().view(np.uint8).reshape(K, 16).copy().view(oracle.CHUNK).reshape(K)
    assert got_chunks.tobytes() == chunks.tobytes()
    assert np.array_equal(u32(r["lut"]), lut)
    assert np.array_equal(r["offsets"][:K + 1].cpu().numpy().view(np.uint64), offsets)
    dist_o, want_perm = oracle.distribute(pts_np, cube, g, lut, offsets)
    del dist_o
    perm_np = u32(r["perm"][:n])
    assert np.array_equal(perm_np, want_perm)
    del want_perm

    # spatial preview (one random point per occupied level-7 cell) on the same cloud
    if n <= 200_000_000:
        sp, sp_n = fp.fp_preview_spatial(pts, r["cube"], 7)
        want_sp, _ = oracle.preview_spatial(pts_np, cube, 7)
        k = int(sp_n.item())
        assert k == len(want_sp)
        assert np.array_equal(sp[:k].cpu().numpy().view(np.uint32).reshape(-1, 4),
                              np.ascontiguousarray(want_sp).view(np.uint32).reshape(-1, 4))
        del sp, want_sp

    # octree on sampled chunks
    nodes = fp.nodes_to_host(r["nodes"], r["num_nodes"])
    rng = np.random.default_rng(seed)
    # (the 1B cloud's chunks are all alike: two of them)
    for c in sampled_chunks(chunks, C, rng, *((1, False) if n > 500_000_000 else (4, True))):
        check_chunk(fp, pts_np, cube, oprm, C, r, nodes, chunks[c], offsets[c:c + 2], r["owner"], perm_np)
    del perm_np
    # layout properties of the whole cloud
    check_layout(fp, pts, r, nodes, n, C, lmax)
    # one headless frame of the whole octree (selection and framebuffer) against the oracle
    if n <= 200_000_000:
        check_frame(fp, pts_np, r, nodes, cube)
    assert fp.get_device_error() == 0
