"""Pins of the CPU oracle against what the definitions and mathematics fix:
published splitmix64 outputs, hand-worked fixtures, closed forms, library
routines (numpy min/max, bincount, stable argsort), a pure-Python brute force
written independently, and invariants.  No GPU."""
import json
import os
import random

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def make_pts(xyz, rgba=None):
    a = np.zeros(len(xyz), oracle.POINT)
    if len(xyz):
        xyz = np.asarray(xyz, dtype=np.int64)
        a["x"], a["y"], a["z"] = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    if rgba is not None:
        a["r"], a["g"], a["b"], a["a"] = rgba
    return a


def prm_of(d, modulus=16):
    return oracle.params(grid_log2=d["grid_log2"], sub_log2=d["sub_log2"], max_level=d["max_level"],
                         decim_modulus=modulus, chunk_threshold=d["chunk_threshold"],
                         node_capacity=d["node_capacity"])


# ------------------------------------------------------------------ splitmix64
def test_splitmix64_published_outputs():
    g = load("splitmix64_seed0.json")
    gamma = int(g["gamma"], 16)
    for k, v in enumerate(g["outputs"]):
        # output k of a generator seeded with 0 = first output of one seeded with k*gamma
        assert oracle.splitmix64((k * gamma) % (1 << 64)) == int(v, 16)


def test_preview_matches_independent_bigint_hash():
    n = 20000
    pts = synth.uniform(n, 11)
    prev, idx = oracle.decimate(pts, 0, 16)
    want = [i for i in range(n) if brute.splitmix64(i) % 16 == 0]
    assert idx.tolist() == want
    assert np.array_equal(prev, pts[want])
    # first_index shifts the hash argument, not the output order
    prev2, idx2 = oracle.decimate(pts[5000:], 5000, 16)
    assert idx2.tolist() == [i for i in want if i >= 5000]
    # modulus 1 keeps everything, a modulus larger than any hash keeps only h == 0
    assert len(oracle.decimate(pts[:100], 0, 1)[0]) == 100
    assert len(oracle.decimate(pts[:100], 0, 7)[1]) == sum(brute.splitmix64(i) % 7 == 0 for i in range(100))


def test_cloud_digest_bruteforce():
    pts = synth.lidar(300, 9)
    M = (1 << 64) - 1
    want = len(pts)
    for i, w in enumerate(pts.view(np.uint32).reshape(-1, 4).tolist()):
        a, b = w[0] | (w[1] << 32), w[2] | (w[3] << 32)
        want += brute.splitmix64(brute.splitmix64(i) ^ brute.splitmix64(a) ^ brute.splitmix64(b ^ 0x5851F42D4C957F2D))
    assert oracle.cloud_digest(pts) == want & M
    assert oracle.cloud_digest(pts[:0]) == 0
    swapped = pts.copy()
    swapped[[3, 4]] = swapped[[4, 3]]
    assert oracle.cloud_digest(swapped) != oracle.cloud_digest(pts)   # order matters
    moved = pts.copy()
    moved["x"][7] += 1
    assert oracle.cloud_digest(moved) != oracle.cloud_digest(pts)


def test_preview_modulus_closed_forms():
    # ceil(n / target), at least 1; the 1B-point cloud at a 1M-point budget keeps every 1000th hash
    assert oracle.preview_modulus(10 ** 9, 10 ** 6) == 1000
    assert oracle.preview_modulus(10 ** 9 + 1, 10 ** 6) == 1001
    assert oracle.preview_modulus(999_999, 10 ** 6) == 1
    assert oracle.preview_modulus(0, 10) == 1
    assert oracle.preview_modulus(10 ** 6, 0) == 1
    assert oracle.preview_modulus(1 << 40, 1) == 0xFFFFFFFF


@pytest.mark.parametrize("n,seed,level,first", [(300, 1, 1, 0), (500, 2, 2, 7), (800, 3, 3, 1 << 33), (1, 4, 7, 0),
                                                (0, 5, 4, 0)])
def test_preview_spatial_bruteforce(n, seed, level, first):
    rnd = random.Random(seed)
    xyz = [(rnd.randrange(-50, 50), rnd.randrange(0, 9), rnd.randrange(-3, 200)) for _ in range(n)]
    pts = make_pts(xyz)
    cube = oracle.bounds(pts)
    got, idx = oracle.preview_spatial(pts, cube, level, first)
    # independent: Python integers, a dictionary of the best (hash, index) per cell
    cb = brute.cube(xyz)
    best = {}
    for i, p in enumerate(xyz):
        k = brute.key(p, cb, level)
        h = brute.splitmix64(first + i)
        if k not in best or h < best[k][0]:
            best[k] = (h, i)
    want = sorted(i for _, i in best.values())
    assert [int(v) - first for v in idx] == want
    assert np.array_equal(got, pts[want]) if n else len(got) == 0


def test_preview_spatial_invariants():
    pts = synth.lidar(200_000, 8)
    cube = oracle.bounds(pts)
    for level in (4, 6):
        got, idx = oracle.preview_spatial(pts, cube, level)
        occupied = int((oracle.count(pts, cube, level) > 0).sum())
        assert len(got) == occupied                       # one point per occupied cell
        assert np.all(np.diff(idx.astype(np.int64)) > 0)  # ascending index
        keys = oracle.point_keys(pts[idx[:2000].astype(np.int64)], cube, level)
        assert len(set(keys.tolist())) == len(keys)       # distinct cells
    # every other point of a sampled cell has a larger hash than the kept one
    got, idx = oracle.preview_spatial(pts[:5000], oracle.bounds(pts[:5000]), 3)
    cb = oracle.bounds(pts[:5000])
    allkeys = oracle.point_keys(pts[:5000], cb, 3)
    for i in idx[:20].astype(np.int64):
        same = np.flatnonzero(allkeys == allkeys[i])
        assert min(same, key=lambda j: oracle.splitmix64(int(j))) == i


# ---------------------------------------------------------------------- cells
def test_cell_closed_forms():
    for level in (0, 1, 7, 13, 21):
        assert oracle.axis_cell(5, 5, 1, level) == 0                     # S = 1: one cell
        assert oracle.axis_cell(2**31 - 1, -2**31, 2**32, level) == 2**level - 1   # top of the cube
        assert oracle.axis_cell(0, -2**31, 2**32, level) == (2**level) // 2
        for S in (3, 1000, 2**20, 2**31):
            # the last coordinate of the cube: floor((S-1) 2^l / S) = 2^l - ceil(2^l / S)
            assert oracle.axis_cell(S - 1, 0, S, level) == 2**level - (2**level + S - 1) // S


def test_cell_exact_against_python_integers():
    rng = random.Random(7)
    for _ in range(3000):
        S = rng.choice([1, 2, 3, 7, 2**20, 2**31 + 11, 2**32, rng.randrange(1, 2**32 + 1)])
        d = rng.randrange(0, S)
        o = rng.randrange(-2**31, 2**31 - d) if d < 2**32 - 1 else -2**31
        if o + d > 2**31 - 1:
            continue
        for level in (0, 3, 7, 15, 21):
            assert oracle.axis_cell(o + d, o, S, level) == (d * 2**level) // S


def test_morton_digit_order():
    assert oracle.morton(1, 0, 0, 1) == 4       # x is the top bit of each digit
    assert oracle.morton(0, 1, 0, 1) == 2
    assert oracle.morton(0, 0, 1, 1) == 1
    assert oracle.morton(3, 0, 0, 2) == 36      # digits (4, 4)
    assert oracle.morton(2, 1, 0, 2) == 34      # digits (4, 2)
    assert oracle.morton(1, 1, 1, 2) == 7       # digits (0, 7)
    assert oracle.morton(127, 0, 0, 7) == 4 * (8**7 - 1) // 7


def test_nesting_of_levels():
    pts = synth.lidar(300, 3)
    cube = oracle.bounds(pts)
    for level in (1, 6, 7, 12, 20):
        a = oracle.point_keys(pts, cube, level)
        b = oracle.point_keys(pts, cube, level + 1)
        assert np.array_equal(a, b >> np.uint64(3))


def test_int32_extremes_fixture():
    g = load("hand_int32_extremes.json")
    pts = make_pts(g["points"])
    cube = oracle.bounds(pts)[0]
    assert cube["o"].tolist() == g["cube"]["o"] and cube["mx"].tolist() == g["cube"]["mx"]
    assert int(cube["S"]) == g["cube"]["S"]
    cb = oracle.bounds(pts)
    assert [oracle.axis_cell(int(p["x"]), int(cube["o"][0]), int(cube["S"]), 7) for p in pts] == g["level7_cells_x"]
    assert oracle.point_keys(pts, cb, 7).tolist() == g["level7_keys"]


# ---------------------------------------------------------------------- bounds
def test_bounds_against_numpy():
    for pts in (synth.uniform(5000, 2), synth.lidar(5000, 4), make_pts([[5, -9, 3]])):
        c = oracle.bounds(pts)[0]
        lo = [int(pts[a].min()) for a in "xyz"]
        hi = [int(pts[a].max()) for a in "xyz"]
        assert c["o"].tolist() == lo and c["mx"].tolist() == hi
        assert int(c["S"]) == max(h - l for h, l in zip(hi, lo)) + 1
    assert int(oracle.bounds(make_pts([]))[0]["S"]) == 0


# --------------------------------------------------------- count / merge / distribute
def test_count_against_bincount():
    pts = synth.lidar(20000, 5)
    cube = oracle.bounds(pts)
    for g in (1, 3, 7):
        counts = oracle.count(pts, cube, g)
        keys = oracle.point_keys(pts, cube, g).astype(np.int64)
        assert np.array_equal(counts, np.bincount(keys, minlength=8**g).astype(np.uint32))
        assert counts.sum() == len(pts)


def _check_chunks(counts, g, T, chunks, lut, offsets):
    n = int(counts.sum())
    assert offsets[0] == 0 and offsets[-1] == n
    assert np.array_equal(np.diff(offsets.astype(np.int64)), chunks["count"].astype(np.int64))
    covered = np.zeros(len(counts), bool)
    prev_start = -1
    for q, ch in enumerate(chunks):
        sh = 3 * (g - int(ch["level"]))
        b, e = int(ch["key"]) << sh, (int(ch["key"]) + 1) << sh
        assert b > prev_start                               # Morton preorder
        prev_start = b
        assert int(counts[b:e].sum()) == int(ch["count"]) > 0
        assert not covered[b:e].any()                       # disjoint
        covered[b:e] = True
        assert int(ch["count"]) <= T or int(ch["level"]) == g   # at or under T, or one finest cell
        if int(ch["level"]) > 0:                            # parent holds more than T
            psh = sh + 3
            pk = int(ch["key"]) >> 3
            assert int(counts[pk << psh:(pk + 1) << psh].sum()) > T
        nz = counts[b:e] > 0
        assert np.all(lut[b:e][nz] == q)
    assert np.all(covered[counts > 0])                      # covering
    assert np.all(lut[counts == 0] == 0xFFFFFFFF)


def test_merge_invariants_and_bruteforce():
    rng = random.Random(3)
    for trial in range(30):
        g = rng.choice([1, 2, 3])
        n = rng.randrange(0, 300)
        pts = synth.lidar(n, 100 + trial) if trial % 2 else synth.uniform(n, 100 + trial, bits=rng.choice([2, 5, 20]))
        cube = oracle.bounds(pts)
        counts = oracle.count(pts, cube, g)
        T = rng.choice([1, 2, 5, 17, 60, 1000])
        chunks, lut, offsets = oracle.merge(counts, g, T)
        _check_chunks(counts, g, T, chunks, lut, offsets)
        bp = [(int(p["x"]), int(p["y"]), int(p["z"])) for p in pts]
        bc = brute.cube(bp)
        want = brute.chunks(brute.counts(bp, bc, g), g, T)
        assert [(int(c["level"]), int(c["key"]), int(c["count"])) for c in chunks] == want
        dist, perm = oracle.distribute(pts, cube, g, lut, offsets)
        assert perm.tolist() == brute.distribute(bp, bc, g, want)


def test_merge_threshold_boundary():
    counts = np.zeros(8, np.uint32)
    counts[0], counts[5] = 3, 2
    ch, lut, off = oracle.merge(counts, 1, 5)       # root count 5 == T -> one chunk at the root
    assert [(int(c["level"]), int(c["key"]), int(c["count"])) for c in ch] == [(0, 0, 5)]
    ch, lut, off = oracle.merge(counts, 1, 4)       # 5 > 4 -> split
    assert [(int(c["level"]), int(c["key"]), int(c["count"])) for c in ch] == [(1, 0, 3), (1, 5, 2)]
    ch, lut, off = oracle.merge(counts, 1, 2)       # cell 0 overflows at the finest level
    assert [(int(c["level"]), int(c["key"]), int(c["count"])) for c in ch] == [(1, 0, 3), (1, 5, 2)]


def test_distribute_is_stable_argsort():
    pts = synth.lidar(30000, 9)
    cube = oracle.bounds(pts)
    counts = oracle.count(pts, cube, 7)
    chunks, lut, offsets = oracle.merge(counts, 7, 500)
    dist, perm = oracle.distribute(pts, cube, 7, lut, offsets)
    cid = lut[oracle.point_keys(pts, cube, 7).astype(np.int64)]
    want = np.argsort(cid, kind="stable")
    assert np.array_equal(perm, want)
    assert np.array_equal(dist, pts[want])


# ------------------------------------------------------------ golden fixtures
@pytest.mark.parametrize("name", ["hand_six_points.json", "hand_identical.json"])
def test_golden_fixture(name):
    gd = load(name)
    pts = make_pts(gd["points"])
    prm = prm_of(gd["params"])
    g = gd["params"]["grid_log2"]
    for form in (0, 1):
        r = oracle.build_all(pts, prm, lod_form=form)
        c = r["cube"][0]
        assert c["o"].tolist() == gd["cube"]["o"] and c["mx"].tolist() == gd["cube"]["mx"]
        assert int(c["S"]) == gd["cube"]["S"]
        nz = {str(k): int(v) for k, v in enumerate(r["counts"]) if v}
        assert nz == gd["counts_nonzero"]
        assert [[int(x["level"]), int(x["key"]), int(x["count"])] for x in r["chunks"]] == gd["chunks"]
        assert r["offsets"].tolist() == gd["offsets"]
        assert r["perm"].tolist() == gd["dist_perm"]
        nodes = r["nodes"]
        assert len(nodes) == len(gd["nodes"])
        for nd, want in zip(nodes, gd["nodes"]):
            for k, v in want.items():
                assert int(nd[k]) == v, (k, nd, want)
        assert r["leaf_perm"].tolist() == gd["leaf_perm"]
        assert r["final_perm"].tolist() == gd["final_perm"]
        assert np.array_equal(r["final_pts"], pts[gd["final_perm"]])
    lam, leaf, own = oracle.point_levels(pts, oracle.bounds(pts), prm)
    assert own.tolist() == gd["owner_level"]


# --------------------------------------------------------- hierarchy and LOD
def check_tree_invariants(pts, prm, r):
    n = len(pts)
    p = prm[0]
    C, Lmax, s = int(p["node_capacity"]), int(p["max_level"]), int(p["sub_log2"])
    nodes, fperm, lperm = r["nodes"], r["final_perm"], r["leaf_perm"]
    assert sorted(fperm.tolist()) == list(range(n))        # every point exactly once
    assert sorted(lperm.tolist()) == list(range(n))
    assert int(nodes["n_own"].sum()) == n if n else len(nodes) == 0
    cube = oracle.bounds(pts)
    keys = {l: oracle.point_keys(pts, cube, l) for l in range(0, 22)} if n else {}
    for i, nd in enumerate(nodes):
        L = int(nd["level"])
        b, e = int(nd["first"]), int(nd["first"]) + int(nd["n_own"])
        own = fperm[b:e]
        assert np.all(np.diff(own.astype(np.int64)) > 0)     # ascending index
        assert np.all(keys[L][own] == nd["key"])               # inside the node
        sub = lperm[int(nd["leaf_first"]):int(nd["leaf_first"]) + int(nd["count"])]
        assert np.all(keys[L][sub] == nd["key"]) and len(sub) == int(nd["count"])
        if nd["is_leaf"]:
            assert int(nd["count"]) <= C or L == Lmax or len(set(keys[21][sub].tolist())) == 1
            assert np.all(np.diff(sub.astype(np.int64)) > 0)
        else:
            assert int(nd["count"]) > C and L < Lmax
            # one owned point per occupied level-(L+s) cell, each the cell's minimum index
            ck = keys[L + s][own]
            assert len(set(ck.tolist())) == len(own)
            for q, c in zip(own, ck):
                assert q == np.flatnonzero(keys[L + s] == c).min()
            # the node and its ancestors together cover every occupied level-(L+s) cell
            anc = set(own.tolist())
            j = i
            while j > 0:
                j = max(k for k in range(j) if int(nodes[k]["n_desc"]) + k >= j and int(nodes[k]["level"]) < int(nodes[j]["level"]))
                pb = int(nodes[j]["first"])
                anc |= set(fperm[pb:pb + int(nodes[j]["n_own"])].tolist())
            covered = {int(keys[L + s][q]) for q in anc if keys[L][q] == nd["key"]}
            assert covered == set(keys[L + s][sub].tolist())


def random_cloud(rng, trial):
    n = rng.randrange(0, 250)
    kind = trial % 3
    if kind == 0:
        return synth.uniform(n, 500 + trial, bits=rng.choice([1, 3, 8, 20]))
    if kind == 1:
        return synth.lidar(n, 500 + trial)
    base = synth.uniform(max(n // 4, 1), 900 + trial, bits=4)          # many duplicates
    return base[np.array([rng.randrange(len(base)) for _ in range(n)], dtype=np.int64)] if n else base[:0]


def test_lod_forms_and_bruteforce_agree_small():
    rng = random.Random(11)
    for trial in range(45):
        pts = random_cloud(rng, trial)
        g = rng.choice([1, 2, 3])
        s = rng.choice([g, g + 1, g + 3])
        Lmax = rng.randrange(g, 22 - s + 1)
        C = rng.choice([1, 2, 3, 10, 40])
        T = C * rng.choice([1, 2, 7])
        prm = oracle.params(g, s, Lmax, 16, T, C)
        sim = oracle.build_all(pts, prm, lod_form=0)
        closed = oracle.octree_lod(pts, sim["cube"], prm, form=1)
        assert np.array_equal(sim["nodes"], closed["nodes"])
        assert np.array_equal(sim["final_perm"], closed["final_perm"])
        bp = [(int(p["x"]), int(p["y"]), int(p["z"])) for p in pts]
        b = brute.build(bp, g, s, Lmax, C, T)
        assert [(nd["level"], nd["key"], len(nd["members"])) for nd in b["nodes"]] == \
            [(int(x["level"]), int(x["key"]), int(x["count"])) for x in sim["nodes"]]
        assert sim["leaf_perm"].tolist() == b["leaf_perm"]
        assert sim["final_perm"].tolist() == b["final_perm"]
        assert sim["nodes"]["n_own"].tolist() == b["n_own"]
        check_tree_invariants(pts, prm, sim)


def test_lod_forms_agree_medium():
    for seed, gen in ((1, "uniform"), (2, "lidar")):
        pts = getattr(synth, gen)(40000, seed)
        prm = oracle.params(7, 7, 15, 16, 4000, 1000)
        cube = oracle.bounds(pts)
        a = oracle.octree_lod(pts, cube, prm, 0)
        b = oracle.octree_lod(pts, cube, prm, 1)
        assert np.array_equal(a["nodes"], b["nodes"])
        assert np.array_equal(a["final_perm"], b["final_perm"])
        assert np.array_equal(a["final_pts"], pts[a["final_perm"]])
        assert np.array_equal(a["leaf_pts"], pts[a["leaf_perm"]])


def test_lod_invariants_medium():
    pts = synth.lidar(3000, 21)
    prm = oracle.params(3, 4, 10, 16, 300, 100)
    r = oracle.build_all(pts, prm)
    check_tree_invariants(pts, prm, r)


def test_edge_cases():
    prm = oracle.params(7, 7, 15, 16, 100, 10)
    r = oracle.build_all(make_pts([]), prm)
    assert len(r["nodes"]) == 0 and len(r["chunks"]) == 0 and r["offsets"].tolist() == [0]
    r = oracle.build_all(make_pts([[4, 5, 6]]), prm)
    assert len(r["nodes"]) == 1 and int(r["nodes"][0]["is_leaf"]) == 1 and r["final_perm"].tolist() == [0]
    assert [(int(c["level"]), int(c["count"])) for c in r["chunks"]] == [(0, 1)]


def test_octree_independent_of_grid_and_threshold():
    """The hierarchy is defined by C and L_max alone and the LOD by s and the
    original indices, so the count grid g (g <= s, g <= L_max) and the chunk
    threshold T (T >= C) only change how the work is cut into chunks: the node
    table, the leaf grouping and the final layout are the same for all of them.
    The batched builder's tuner relies on this to pick g and T per cloud."""
    pts = synth.lidar(6000, 41)
    ref = None
    for g, T in [(1, 60), (2, 60), (3, 500), (4, 6000), (5, 100000)]:
        got = oracle.build_all(pts, oracle.params(g, 5, 12, 16, T, 60))
        key = (got["nodes"].tobytes(), got["leaf_perm"].tobytes(), got["final_perm"].tobytes())
        if ref is None:
            ref = key
        assert key == ref, (g, T)


# ------------------------------------------------------------------ rendering
def _ortho(sx, ox, sy, oy, sz, oz):
    """clip = (sx x + ox, sy y + oy, sz z + oz, 1): exact for power-of-two scales and integer inputs"""
    m = np.zeros(16, np.float32)
    m[0], m[3], m[5], m[7], m[10], m[11], m[15] = sx, ox, sy, oy, sz, oz, 1.0
    return m


def _cube_cloud(n, seed):
    """points in [0, 1024)^3 with the two corners present, so the cube is exactly [0, 1024)"""
    rnd = np.random.default_rng(seed)
    xyz = rnd.integers(0, 1024, size=(n, 3))
    xyz[0], xyz[1] = 0, 1023
    rgba = rnd.integers(0, 256, size=(n, 4))
    pts = make_pts(xyz.tolist())
    pts["r"], pts["g"], pts["b"], pts["a"] = rgba.T
    return pts


def _tree(pts, s=3, lmax=6, C=60):
    prm = oracle.params(2, s, lmax, 16, 10 ** 9, C)
    cube = oracle.bounds(pts)
    return cube, oracle.octree_lod(pts, cube, prm)


def test_render_orthographic_closed_form():
    pts = _cube_cloud(3000, 1)
    cube, t = _tree(pts)
    assert int(cube["S"][0]) == 1024
    cam = oracle.camera(_ortho(1 / 512, -1, 1 / 512, -1, 1 / 1024, 0), 64, 64, 0.0)
    sel = oracle.render_select(t["nodes"], cube, cam)
    assert sel.tolist() == list(range(len(t["nodes"])))   # in view, refined down to the leaves
    fb = oracle.rasterize(t["nodes"], sel, t["final_pts"], cam)
    # pixel = (x // 16, y // 16), depth = z / 1024 exactly; the smallest (depth, rgba) wins
    want = np.full((64, 64), np.uint64(0xFFFFFFFFFFFFFFFF))
    d = (pts["z"].astype(np.float32) / np.float32(1024)).view(np.uint32).astype(np.uint64)
    rgba = pts.view(np.uint32).reshape(-1, 4)[:, 3].astype(np.uint64)   # the record's fourth word
    key = (d << np.uint64(32)) | rgba
    for x, y, k in zip(pts["x"] // 16, pts["y"] // 16, key):
        want[y, x] = min(want[y, x], k)
    assert np.array_equal(fb, want)


def test_render_selection_frustum_and_size():
    pts = _cube_cloud(5000, 2)
    cube, t = _tree(pts)
    nodes = t["nodes"]
    # half the cube in view (x in [0, 512] maps to [-1, 1]): a node is drawn iff its box starts at x <= 512
    cam = oracle.camera(_ortho(1 / 256, -1, 1 / 512, -1, 1 / 1024, 0), 64, 64, 0.0)
    sel = set(oracle.render_select(nodes, cube, cam).tolist())
    for i, nd in enumerate(nodes):
        L = int(nd["level"])
        c = sum(((int(nd["key"]) >> (3 * b + 2)) & 1) << b for b in range(L))
        lo_x = -(-(c * 1024) // (1 << L))   # ceil(c S / 2^L)
        assert (i in sel) == (lo_x <= 512), (i, L, lo_x)
    # size threshold: a level-L box spans 1024 / 2^L - 1 units = (64 / 2^L - 1/16) pixels
    cam = oracle.camera(_ortho(1 / 512, -1, 1 / 512, -1, 1 / 1024, 0), 64, 64, 10.0)
    sel = oracle.render_select(nodes, cube, cam)
    assert sel.tolist() == [i for i, nd in enumerate(nodes) if nd["level"] <= 3]
    # nothing in view: the camera looks away (w < 0 everywhere)
    m = _ortho(1 / 512, -1, 1 / 512, -1, 1 / 1024, 0)
    m[15] = -1.0
    assert len(oracle.render_select(nodes, cube, oracle.camera(m, 64, 64, 0.0))) == 0
    # a huge threshold draws the root only
    assert oracle.render_select(nodes, cube, oracle.camera(_ortho(1 / 512, -1, 1 / 512, -1, 1 / 1024, 0), 64, 64,
                                                           1e9)).tolist() == [0]
