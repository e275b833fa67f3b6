"""fp_build_batched: a batch of clouds of uneven sizes and parameters, built on
several lanes in one call, gives every cloud exactly the outputs of the plain
calls (which the other GPU tests pin to the oracle), and the same again when the
batch is captured into a CUDA graph and replayed, and for any number of lanes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_build_matches_oracle

pytestmark = pytest.mark.gpu

KEYS = ["cube", "preview", "preview_count", "counts", "chunks", "num_chunks", "lut", "offsets", "dist", "perm",
        "num_nodes", "nodes", "leaf_pts", "leaf_perm", "owner", "final", "final_perm"]

# kind, n, seed, g, s, lmax, T, C
BATCH = [
    ("lidar", 300_000, 21, 7, 7, 15, 10_000, 2_000),
    ("uniform", 123_457, 22, 7, 7, 15, 100_000, 20_000),
    ("uniform", 0, 23, 7, 7, 15, 100_000, 20_000),
    ("lidar", 40_000, 24, 4, 5, 12, 3_000, 300),
    ("uniform", 1, 25, 7, 7, 15, 100, 10),
    ("uniform", 77_777, 26, 3, 3, 9, 1_000, 40),
    ("lidar", 5_000, 27, 5, 6, 16, 400, 50),
    ("uniform", 200_003, 28, 7, 7, 8, 50_000, 5_000),
    ("uniform", 3, 29, 1, 1, 21, 1, 1),
    ("lidar", 90_000, 30, 6, 7, 15, 20_000, 1_000),
]


def make_cloud(fp, kind, n, seed):
    a = synth.uniform(n, seed) if kind == "uniform" else synth.lidar(n, seed)
    return fp.as_points(a, "cuda")


def used(out, k):
    """The meaningful part of an output tensor (counts decide the lengths)."""
    t = out[k]
    if k == "preview":
        return t[: int(out["preview_count"].item())]
    if k == "chunks":
        return t[: int(out["num_chunks"].item())]
    if k == "offsets":
        return t[: int(out["num_chunks"].item()) + 1]
    if k == "nodes":
        return t[: int(out["num_nodes"].item())]
    if k in ("dist", "perm", "leaf_pts", "leaf_perm", "owner", "final", "final_perm"):
        return t[: out["n"]]
    return t


def plain(fp, pts, prm):
    r = fp.build_octree(pts, prm)
    r["n"] = pts.shape[0]
    return r


def assert_same(a, b, what):
    for k in KEYS:
        x, y = used(a, k).reshape(-1).view(torch.int32).cpu(), used(b, k).reshape(-1).view(torch.int32).cpu()
        assert x.shape == y.shape and torch.equal(x, y), "%s: output %s differs" % (what, k)


@pytest.fixture(scope="module")
def batch(gpu_lib):
    fp = gpu_lib
    clouds = []
    for kind, n, seed, g, s, lmax, T, C in BATCH:
        prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T,
                        node_capacity=C)
        clouds.append((make_cloud(fp, kind, n, seed), prm))
    ref = [plain(fp, p, prm) for p, prm in clouds]
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    return fp, clouds, ref


@pytest.mark.parametrize("nlanes", [1, 4, 7])
def test_batched_equals_plain(batch, nlanes):
    fp, clouds, ref = batch
    outs, _, _ = fp.build_batched(clouds, nlanes=nlanes)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    for i, (o, r) in enumerate(zip(outs, ref)):
        o["n"] = clouds[i][0].shape[0]
        assert_same(o, r, "cloud %d (%d lanes)" % (i, nlanes))


@pytest.mark.parametrize("threads,slots", [(256, 1024), (512, 0), (256, 4096)])
def test_fused_first_passes_equal_plain(batch, threads, slots):
    """The fused bounds + preview and count launches over all clouds of the
    batch, with each block size and hot-cell table the tuner may pick, give
    every cloud the plain calls' outputs."""
    fp, clouds, ref = batch
    opts = fp.batch_opts(nlanes=4, fused_first=1, count_threads=threads, count_slots=slots)
    outs, _, _ = fp.build_batched(clouds, opts=opts)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    for i, (o, r) in enumerate(zip(outs, ref)):
        o["n"] = clouds[i][0].shape[0]
        assert_same(o, r, "cloud %d (fused, %d threads, %d slots)" % (i, threads, slots))


def test_fused_first_passes_many_clouds_match_oracle(gpu_lib):
    """More clouds than one fused launch takes (300 > 256): two groups; every
    cloud's cube, preview, count grid and octree against the oracle."""
    fp = gpu_lib
    rng = np.random.default_rng(7)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(50), np.log(20_000), 300))]
    sizes[5] = 0
    prm = fp.params(grid_log2=5, sub_log2=6, max_level=12, decim_modulus=16, chunk_threshold=2_000, node_capacity=300)
    hosts = [synth.uniform(n, 900 + i) if i % 2 else synth.lidar(n, 900 + i) for i, n in enumerate(sizes)]
    clouds = [(fp.as_points(h, "cuda"), prm) for h in hosts]
    opts = fp.batch_opts(nlanes=8, fused_first=1, count_threads=512, count_slots=1024)
    outs, _, _ = fp.build_batched(clouds, opts=opts)
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    oprm = oracle.params(5, 6, 12, 16, 2_000, 300)
    for i in list(range(0, 300, 23)) + [5, 299]:
        want = oracle.build_all(hosts[i], oprm)
        o = outs[i]
        k = int(o["preview_count"].item())
        assert k == len(want["preview"])
        assert np.array_equal(o["counts"].cpu().numpy().view(np.uint32), want["counts"])
        M = int(o["num_nodes"].item())
        assert_build_matches_oracle(want, cube=o["cube"], preview=o["preview"][:k], nodes=o["nodes"][:M],
                                    final=o["final"][:sizes[i]], final_perm=o["final_perm"][:sizes[i]])


def test_batched_graph_replay(batch):
    fp, clouds, ref = batch
    outs, descs, ws = fp.build_batched(clouds, nlanes=5)   # first call (outside capture) creates the lanes
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        fp.fp_build_batched(descs, len(clouds), 5, ws, stream=side)
    for o in outs:   # wipe, then replay twice
        for k in ("final", "final_perm", "nodes", "leaf_pts", "owner"):
            o[k].fill_(-1)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert fp.get_device_error() == 0
    for i, (o, r) in enumerate(zip(outs, ref)):
        o["n"] = clouds[i][0].shape[0]
        assert_same(o, r, "cloud %d (graph replay)" % i)


def test_batched_matches_oracle(batch):
    """Two clouds of the batch straight against the oracle (node table, final layout)."""
    fp, clouds, _ = batch
    outs, _, _ = fp.build_batched(clouds, nlanes=3)
    torch.cuda.synchronize()
    for i in (3, 6):
        kind, n, seed, g, s, lmax, T, C = BATCH[i]
        a = synth.uniform(n, seed) if kind == "uniform" else synth.lidar(n, seed)
        want = oracle.build_all(a, oracle.params(g, s, lmax, 16, T, C))
        nodes = fp.nodes_to_host(outs[i]["nodes"], outs[i]["num_nodes"])
        for f in ("key", "level", "count", "n_own", "n_desc", "first", "leaf_first", "is_leaf", "child_mask"):
            assert np.array_equal(nodes[f], want["nodes"][f]), (i, f)
        got = outs[i]["final_perm"][:n].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want["final_perm"])


def test_batched_rejects_bad_descriptor(batch):
    fp, clouds, _ = batch
    outs = [fp.cloud_outputs(p, prm) for p, prm in clouds[:2]]
    descs = fp.batch_descs(clouds[:2], outs)
    descs[1].d_final = None   # a required output missing: nothing is enqueued
    ws = torch.empty(max(fp.batch_workspace_size(descs, 2, 2), 1), dtype=torch.uint8, device="cuda")
    st = fp.load().fp_build_batched(descs, 2, 2, ws.data_ptr(), ws.numel(), None)
    assert st == 1   # FP_ERR_INVALID


def test_side_stream_builds_match_oracle(gpu_lib):
    """Builds enqueued back to back on a side stream, each with its own grid
    resolution, as the tuner runs them: the binding's temporaries (workspaces,
    zero-filled outputs) belong to that stream, so none is reused while an
    earlier stage still runs, and every build equals the oracle's."""
    fp = gpu_lib
    pts_np = synth.lidar(526_150, 1000)
    pts = fp.as_points(pts_np, "cuda")
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    outs = []
    for g in (7, 6, 5, 4):
        prm = fp.params(grid_log2=g, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=100_000,
                        node_capacity=20_000)
        outs.append((g, fp.build_octree(pts, prm, stream=st)))
    st.synchronize()
    assert fp.get_device_error(stream=st) == 0
    for g, r in outs:
        want = oracle.build_all(pts_np, oracle.params(g, 7, 15, 16, 100_000, 20_000))
        M = int(r["num_nodes"].item())
        assert_build_matches_oracle(want, nodes=r["nodes"][:M], final=r["final"], final_perm=r["final_perm"])
