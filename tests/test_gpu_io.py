"""The octree file and the build cache: the cloud digest against the oracle;
a saved octree read back by an independent numpy parser of the documented
layout and by fp_octree_load (whole and one node at a time) equals the device
outputs (which the other GPU tests pin to the oracle); a cloud built before is
loaded from the cache, a changed cloud or parameter set is rebuilt."""
import struct

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import dev_points

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,seed", [("lidar", 1_000_003, 51), ("uniform", 4097, 52), ("uniform", 1, 53),
                                         ("uniform", 0, 54)])
def test_digest_matches_oracle(gpu_lib, kind, n, seed):
    fp = gpu_lib
    pts_np = synth.lidar(n, seed) if kind == "lidar" else synth.uniform(n, seed)
    pts = dev_points(pts_np) if n else torch.empty((0, 4), dtype=torch.int32, device="cuda")
    assert fp.fp_cloud_digest(pts) == oracle.cloud_digest(pts_np)


def parse(path):
    """Independent reader of the documented file layout."""
    raw = open(path, "rb").read()
    magic, version, hbytes = struct.unpack_from("<8sII", raw, 0)
    n, M, flags, digest, no, po, qo = struct.unpack_from("<QIIQQQQ", raw, 80)
    assert magic == b"FPOCTREE" and version == 1 and hbytes == 160
    assert no % 4096 == 0 and po % 4096 == 0
    nodes = np.frombuffer(raw, oracle.NODE, M, no)
    pts = np.frombuffer(raw, np.uint32, 4 * n, po).reshape(n, 4)
    perm = np.frombuffer(raw, np.uint32, n, qo) if flags & 1 else None
    return dict(n=n, M=M, digest=digest, nodes=nodes, pts=pts, perm=perm, prm=np.frombuffer(raw, oracle.PARAMS, 1, 16),
                cube=np.frombuffer(raw, oracle.CUBE, 1, 48))


def test_save_parse_load(gpu_lib, tmp_path):
    fp = gpu_lib
    pts_np = synth.lidar(300_000, 55)
    pts = dev_points(pts_np)
    prm = fp.params(grid_log2=7, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=10_000, node_capacity=2_000)
    r = fp.build_octree(pts, prm)
    path = str(tmp_path / "a.fpo")
    small = torch.empty(8192, dtype=torch.uint8).pin_memory()   # many pieces through the two halves
    fp.octree_save(path, prm, r, digest=1234, staging=small)
    f = parse(path)
    nodes = fp.nodes_to_host(r["nodes"], r["num_nodes"])
    assert f["n"] == len(pts_np) and f["M"] == len(nodes) and f["digest"] == 1234
    assert f["nodes"].tobytes() == nodes.tobytes()
    assert np.array_equal(f["pts"], r["final"].cpu().numpy().view(np.uint32))
    assert np.array_equal(f["perm"], r["final_perm"].cpu().numpy().view(np.uint32))
    assert f["cube"].tobytes() == r["cube"].cpu().numpy().tobytes()
    assert int(f["prm"]["node_capacity"][0]) == 2_000
    # whole file back to the device
    back = fp.octree_load(path, staging=small)
    assert torch.equal(back["final"], r["final"]) and torch.equal(back["final_perm"], r["final_perm"])
    assert torch.equal(back["nodes"][: len(nodes)], r["nodes"][: len(nodes)])
    # one node's points, as the renderer loads them
    k = int(np.argmax(nodes["n_own"]))
    first, cnt = int(nodes["first"][k]), int(nodes["n_own"][k])
    part = fp.octree_load(path, nodes=False, first=first, count=cnt)
    assert torch.equal(part["final"], r["final"][first:first + cnt])
    assert torch.equal(part["final_perm"], r["final_perm"][first:first + cnt])


def test_file_errors(gpu_lib, tmp_path):
    fp = gpu_lib
    with pytest.raises(fp.FastPointsError):
        fp.octree_header(str(tmp_path / "missing.fpo"))
    bad = tmp_path / "bad.fpo"
    bad.write_bytes(b"NOTANOCTREEFILE" * 40)
    with pytest.raises(fp.FastPointsError):
        fp.octree_header(str(bad))
    pts = dev_points(synth.uniform(20_000, 56))
    prm = fp.params(grid_log2=4, sub_log2=5, max_level=10, decim_modulus=16, chunk_threshold=2_000, node_capacity=100)
    r = fp.build_octree(pts, prm)
    path = str(tmp_path / "b.fpo")
    fp.octree_save(path, prm, r, with_perm=False)
    L = fp.load()
    stg = torch.empty(1 << 16, dtype=torch.uint8).pin_memory()
    perm = torch.empty(10, dtype=torch.int32, device="cuda")
    st = L.fp_octree_load(path.encode(), None, 0, None, fp._ptr(perm), 0, 10, fp._ptr(stg), stg.numel(), None)
    assert st == 1   # the file holds no permutation: FP_ERR_INVALID
    few = torch.empty((4, 5), dtype=torch.int64, device="cuda")
    st = L.fp_octree_load(path.encode(), fp._ptr(few), 1, None, None, 0, 0, fp._ptr(stg), stg.numel(), None)
    assert st == 9   # node_cap below the file's node count: FP_ERR_CAPACITY


def test_cache(gpu_lib, tmp_path):
    fp = gpu_lib
    pts_np = synth.lidar(200_000, 57)
    pts = dev_points(pts_np)
    prm = fp.params(grid_log2=6, sub_log2=7, max_level=14, decim_modulus=16, chunk_threshold=20_000, node_capacity=3_000)
    a, hit_a = fp.cached_build(pts, prm, str(tmp_path))
    b, hit_b = fp.cached_build(pts, prm, str(tmp_path))
    assert not hit_a and hit_b
    M = int(a["num_nodes"].item())
    assert int(b["num_nodes"].item()) == M
    assert torch.equal(a["nodes"][:M], b["nodes"][:M])
    assert torch.equal(a["final"], b["final"]) and torch.equal(a["final_perm"], b["final_perm"])
    prm2 = fp.params(grid_log2=6, sub_log2=7, max_level=14, decim_modulus=16, chunk_threshold=20_000,
                     node_capacity=2_500)
    assert not fp.cached_build(pts, prm2, str(tmp_path))[1]          # other parameters
    moved = pts.clone()
    moved[5, 0] += 1
    assert not fp.cached_build(moved, prm, str(tmp_path))[1]         # another cloud
    assert fp.cached_build(pts, prm, str(tmp_path))[1]
