"""fp_build_batched: a batch of clouds of uneven sizes and parameters, built on
several lanes in one call, gives every cloud exactly the outputs of the plain
calls (which the other GPU tests pin to the oracle), and the same again when the
batch is captured into a CUDA graph and replayed, and for any number of lanes."""
import numpy as np
import pytest
import torch

import oracle
import synth

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
