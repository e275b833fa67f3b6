"""Helpers of the GPU parity tests: run the CUDA path through the C-ABI binding
and bring results to the host in the oracle's record formats."""
import numpy as np
import torch

import oracle


def dev_points(pts_np):
    from paper_2302_05002_gb300 import fastpoints as fp
    return fp.as_points(pts_np, "cuda")


def host_points(t):
    a = t.detach().cpu().contiguous().numpy()
    return a.view(np.uint8).reshape(-1, 16).copy().view(oracle.POINT).reshape(-1)


def cube_np(cube_t):
    return cube_t.detach().cpu().numpy().view(np.uint8).copy().view(oracle.CUBE)


def assert_points_equal(got_t, want_np, count=None):
    got = host_points(got_t)
    if count is not None:
        got = got[:count]
    assert len(got) == len(want_np), (len(got), len(want_np))
    if len(want_np):
        g = got.view(np.uint32).reshape(-1, 4)
        w = np.ascontiguousarray(want_np).view(np.uint32).reshape(-1, 4)
        bad = np.flatnonzero((g != w).any(axis=1))
        assert bad.size == 0, "first mismatch at %d of %d" % (bad[0], len(want_np))


NODE_FIELDS = ["key", "level", "count", "n_own", "n_desc", "child_mask", "is_leaf", "leaf_first", "first"]


def node_records(nodes):
    """Node table (torch (M, 5) int64 or raw 40-byte rows) in the oracle's NODE format."""
    if isinstance(nodes, torch.Tensor):
        a = nodes.detach().cpu().contiguous().numpy().view(np.uint8)
    else:
        a = np.ascontiguousarray(nodes).view(np.uint8)
    return a.reshape(-1, 40).copy().view(oracle.NODE).reshape(-1)


def assert_nodes_equal(got, want):
    assert len(got) == len(want), (len(got), len(want))
    for f in NODE_FIELDS:
        if not np.array_equal(got[f], want[f]):
            bad = np.flatnonzero(got[f] != want[f])[0]
            raise AssertionError("node field %s differs first at node %d: got %s want %s" %
                                 (f, bad, got[bad], want[bad]))


def assert_build_matches_oracle(want, cube=None, preview=None, nodes=None, final=None, final_perm=None):
    """The outputs of one build (host or device tensors, any subset) against the
    oracle's build_all() of the same cloud, element by element."""
    if cube is not None:
        c = cube.detach().cpu().contiguous().view(torch.uint8).reshape(-1)[:32].numpy().copy().view(oracle.CUBE)
        assert c.tobytes() == want["cube"].tobytes(), (c, want["cube"])
    if preview is not None:
        assert_points_equal(preview, want["preview"], count=len(want["preview"]))
    if nodes is not None:
        assert_nodes_equal(node_records(nodes), want["nodes"])
    if final_perm is not None:
        fp_ = final_perm.detach().cpu().contiguous().numpy().view(np.uint32)[:len(want["final_perm"])]
        assert np.array_equal(fp_, want["final_perm"]), "final_perm differs first at %d" % \
            int(np.flatnonzero(fp_ != want["final_perm"])[0])
    if final is not None:
        assert_points_equal(final, want["final_pts"], count=len(want["final_pts"]))
