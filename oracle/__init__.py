"""CPU oracle for the octree-construction hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs may import this package.  The product path never does: the CUDA
library fails loudly when its extension is missing instead of falling back here.

Thin ctypes wrapper over ``fp_oracle.c`` (plain single-threaded C, built with
gcc).  Record dtypes are declared here independently of the CUDA binding; the
16-byte point record is the only format the two sides exchange.
"""
import ctypes
import os
import subprocess

import numpy as np

POINT = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                  ("r", "u1"), ("g", "u1"), ("b", "u1"), ("a", "u1")])
CUBE = np.dtype([("o", "<i4", (3,)), ("mx", "<i4", (3,)), ("S", "<u8")])
CHUNK = np.dtype([("key", "<u8"), ("count", "<u4"), ("level", "<u4")])
NODE = np.dtype([("key", "<u8"), ("first", "<u8"), ("leaf_first", "<u8"),
                 ("count", "<u4"), ("n_own", "<u4"), ("n_desc", "<u4"),
                 ("level", "u1"), ("child_mask", "u1"), ("is_leaf", "u1"), ("pad", "u1")])
PARAMS = np.dtype([("grid_log2", "<u4"), ("sub_log2", "<u4"), ("max_level", "<u4"),
                   ("decim_modulus", "<u4"), ("chunk_threshold", "<u8"), ("node_capacity", "<u8")])
assert (POINT.itemsize, CUBE.itemsize, CHUNK.itemsize, NODE.itemsize, PARAMS.itemsize) == (16, 32, 16, 40, 32)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "fp_oracle.c")]
_HDR = os.path.join(_HERE, "fp_oracle.h")
_LIB = os.path.join(_HERE, "lib", "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (portable C11, no target-specific flags)."""
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp] + _SRC +
                          ["-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        L.orc_splitmix64.argtypes = [u64]; L.orc_splitmix64.restype = u64
        L.orc_bounds.argtypes = [p, u64, p]
        L.orc_decimate.argtypes = [p, u64, u64, u32, p, p]; L.orc_decimate.restype = u64
        L.orc_preview_modulus.argtypes = [u64, u64]; L.orc_preview_modulus.restype = u32
        L.orc_cloud_digest.argtypes = [p, u64]; L.orc_cloud_digest.restype = u64
        L.orc_render_select.argtypes = [p, u32, p, p, p]; L.orc_render_select.restype = u32
        L.orc_rasterize.argtypes = [p, p, u32, p, p, p]
        L.orc_preview_spatial.argtypes = [p, u64, p, u32, u64, p, p]; L.orc_preview_spatial.restype = u64
        L.orc_axis_cell.argtypes = [ctypes.c_int32, ctypes.c_int32, u64, u32]; L.orc_axis_cell.restype = u64
        L.orc_morton.argtypes = [u64, u64, u64, u32]; L.orc_morton.restype = u64
        L.orc_point_key.argtypes = [p, p, u32]; L.orc_point_key.restype = u64
        L.orc_count.argtypes = [p, u64, p, u32, p]
        L.orc_merge.argtypes = [p, u32, u64, p, p, p]; L.orc_merge.restype = u32
        L.orc_distribute.argtypes = [p, u64, p, u32, p, p, p, p]
        L.orc_octree_lod.argtypes = [p, u64, p, p, p, u32, p, p, p, p, ctypes.c_int]
        L.orc_octree_lod.restype = u32
        L.orc_point_levels.argtypes = [p, u64, p, p, p, p, p]; L.orc_point_levels.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _pts(pts):
    a = np.ascontiguousarray(pts)
    if a.dtype != POINT:
        a = a.view(POINT).reshape(-1)
    return a


def params(grid_log2=7, sub_log2=7, max_level=15, decim_modulus=16,
           chunk_threshold=100000, node_capacity=20000):
    a = np.zeros(1, PARAMS)
    a["grid_log2"], a["sub_log2"], a["max_level"] = grid_log2, sub_log2, max_level
    a["decim_modulus"], a["chunk_threshold"], a["node_capacity"] = decim_modulus, chunk_threshold, node_capacity
    return a


def splitmix64(i):
    return int(_load().orc_splitmix64(i))


def axis_cell(p, o, S, level):
    return int(_load().orc_axis_cell(p, o, S, level))


def morton(cx, cy, cz, level):
    return int(_load().orc_morton(cx, cy, cz, level))


def bounds(pts):
    pts = _pts(pts)
    cube = np.zeros(1, CUBE)
    _load().orc_bounds(_p(pts), len(pts), _p(cube))
    return cube


def point_keys(pts, cube, level):
    pts = _pts(pts)
    L = _load()
    return np.array([L.orc_point_key(pts[i:i + 1].ctypes.data, _p(cube), level) for i in range(len(pts))],
                    dtype=np.uint64)


def decimate(pts, first_index=0, modulus=16):
    pts = _pts(pts)
    out = np.empty(max(len(pts), 1), POINT)
    idx = np.empty(max(len(pts), 1), np.uint64)
    k = _load().orc_decimate(_p(pts), len(pts), first_index, modulus, _p(out), _p(idx))
    return out[:k].copy(), idx[:k].copy()


def cloud_digest(pts):
    pts = _pts(pts)
    return int(_load().orc_cloud_digest(_p(pts), len(pts)))


def preview_modulus(n, target):
    return int(_load().orc_preview_modulus(n, target))


def preview_spatial(pts, cube, level, first_index=0):
    """One point per occupied level cell (smallest index hash), ascending index: (points, indices)."""
    pts = _pts(pts)
    out = np.empty(max(len(pts), 1), POINT)
    idx = np.empty(max(len(pts), 1), np.uint64)
    k = _load().orc_preview_spatial(_p(pts), len(pts), _p(cube), level, first_index, _p(out), _p(idx))
    if k == 0xFFFFFFFFFFFFFFFF:
        raise MemoryError("oracle allocation failed")
    return out[:k].copy(), idx[:k].copy()


CAMERA = np.dtype([("m", "<f4", (16,)), ("width", "<u4"), ("height", "<u4"), ("min_node_px", "<f4"),
                   ("reserved", "<u4")])


def camera(m, width, height, min_node_px):
    c = np.zeros(1, CAMERA)
    c["m"][0] = np.asarray(m, dtype=np.float32).reshape(16)
    c["width"], c["height"], c["min_node_px"] = width, height, min_node_px
    return c


def render_select(nodes, cube, cam):
    """Ids (preorder) of the nodes the camera draws."""
    nodes = np.ascontiguousarray(nodes)
    sel = np.empty(max(len(nodes), 1), np.uint32)
    k = _load().orc_render_select(_p(nodes), len(nodes), _p(cube), _p(cam), _p(sel))
    return sel[:k].copy()


def rasterize(nodes, sel, final_pts, cam):
    """Framebuffer (height, width) of uint64: (depth bits << 32 | rgba), all ones where empty."""
    fb = np.empty(int(cam["width"][0]) * int(cam["height"][0]), np.uint64)
    sel = np.ascontiguousarray(sel, dtype=np.uint32)
    _load().orc_rasterize(_p(np.ascontiguousarray(nodes)), _p(sel), len(sel), _p(_pts(final_pts)), _p(cam), _p(fb))
    return fb.reshape(int(cam["height"][0]), int(cam["width"][0]))


def count(pts, cube, g):
    pts = _pts(pts)
    counts = np.empty(1 << (3 * g), np.uint32)
    _load().orc_count(_p(pts), len(pts), _p(cube), g, _p(counts))
    return counts


def merge(counts, g, T):
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    cells = 1 << (3 * g)
    chunks = np.empty(cells, CHUNK)
    lut = np.empty(cells, np.uint32)
    offsets = np.empty(cells + 1, np.uint64)
    K = _load().orc_merge(_p(counts), g, T, _p(chunks), _p(lut), _p(offsets))
    return chunks[:K].copy(), lut, offsets[:K + 1].copy()


def distribute(pts, cube, g, lut, offsets):
    pts = _pts(pts)
    out = np.empty(max(len(pts), 1), POINT)
    perm = np.empty(max(len(pts), 1), np.uint32)
    _load().orc_distribute(_p(pts), len(pts), _p(cube), g, _p(np.ascontiguousarray(lut)),
                           _p(np.ascontiguousarray(offsets)), _p(out), _p(perm))
    return out[:len(pts)], perm[:len(pts)]


def octree_lod(pts, cube, prm, form=0):
    """Hierarchy + leaf-grouped points + LOD (form 0: move simulation, 1: closed form).
    Returns dict(nodes, leaf_pts, leaf_perm, final_pts, final_perm)."""
    pts = _pts(pts)
    n = len(pts)
    L = _load()
    m = max(n, 1)
    leaf_pts, leaf_perm = np.empty(m, POINT), np.empty(m, np.uint32)
    fin_pts, fin_perm = np.empty(m, POINT), np.empty(m, np.uint32)
    cap = 64
    while True:
        nodes = np.zeros(cap, NODE)
        M = L.orc_octree_lod(_p(pts), n, _p(cube), _p(prm), _p(nodes), cap,
                             _p(leaf_pts), _p(leaf_perm), _p(fin_pts), _p(fin_perm), form)
        if M == 0xFFFFFFFF:
            raise MemoryError("oracle allocation failed")
        if M <= cap:
            break
        cap = M
    return dict(nodes=nodes[:M].copy(), leaf_pts=leaf_pts[:n], leaf_perm=leaf_perm[:n],
                final_pts=fin_pts[:n], final_perm=fin_perm[:n])


def point_levels(pts, cube, prm):
    """Per point: (lambda, leaf level, owner level) of the closed-form LOD."""
    pts = _pts(pts)
    n = len(pts)
    lam, leaf, own = (np.empty(max(n, 1), np.uint8) for _ in range(3))
    if _load().orc_point_levels(_p(pts), n, _p(cube), _p(prm), _p(lam), _p(leaf), _p(own)):
        raise MemoryError("oracle allocation failed")
    return lam[:n], leaf[:n], own[:n]


def build_all(pts, prm, lod_form=0):
    """Every stage of the hot path, each from its own definition."""
    pts = _pts(pts)
    p = prm[0]
    g, T = int(p["grid_log2"]), int(p["chunk_threshold"])
    cube = bounds(pts)
    prev_pts, prev_idx = decimate(pts, 0, int(p["decim_modulus"]))
    counts = count(pts, cube, g)
    chunks, lut, offsets = merge(counts, g, T)
    dist, perm = distribute(pts, cube, g, lut, offsets)
    tree = octree_lod(pts, cube, prm, lod_form)
    out = dict(cube=cube, preview=prev_pts, preview_idx=prev_idx, counts=counts, chunks=chunks,
               lut=lut, offsets=offsets, dist=dist, perm=perm)
    out.update(tree)
    return out
