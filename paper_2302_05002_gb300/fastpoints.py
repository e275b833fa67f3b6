"""Python binding of libfastpoints (the C ABI in include/fastpoints.h).

Argument marshalling only: every stage runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  Points are int32 tensors of shape
(n, 4) on the device: x, y, z and the four colour bytes packed in the last
column (the 16-byte fp_point record).  Functions keep the C names; each raises
FastPointsError on a non-zero status.  There is no CPU path: without the built
library or a CUDA device the calls fail.
"""
import ctypes
import functools
import inspect
import os
import re

import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fastpoints.h")


class FastPointsError(RuntimeError):
    pass


class fp_params(ctypes.Structure):
    _fields_ = [("grid_log2", ctypes.c_uint32), ("sub_log2", ctypes.c_uint32), ("max_level", ctypes.c_uint32),
                ("decim_modulus", ctypes.c_uint32), ("chunk_threshold", ctypes.c_uint64),
                ("node_capacity", ctypes.c_uint64)]


class fp_cloud_desc(ctypes.Structure):
    _fields_ = [("d_pts", ctypes.c_void_p), ("n", ctypes.c_uint64), ("prm", fp_params), ("d_cube", ctypes.c_void_p),
                ("d_preview", ctypes.c_void_p), ("preview_cap", ctypes.c_uint64),
                ("d_preview_count", ctypes.c_void_p), ("d_counts", ctypes.c_void_p), ("d_chunks", ctypes.c_void_p),
                ("d_num_chunks", ctypes.c_void_p), ("d_lut", ctypes.c_void_p), ("d_offsets", ctypes.c_void_p),
                ("d_dist", ctypes.c_void_p), ("d_perm", ctypes.c_void_p), ("d_nodes", ctypes.c_void_p),
                ("node_cap", ctypes.c_uint32), ("d_num_nodes", ctypes.c_void_p), ("d_leaf_pts", ctypes.c_void_p),
                ("d_leaf_perm", ctypes.c_void_p), ("d_owner", ctypes.c_void_p), ("d_final", ctypes.c_void_p),
                ("d_final_perm", ctypes.c_void_p)]


class fp_cube(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int32 * 3), ("mx", ctypes.c_int32 * 3), ("S", ctypes.c_uint64)]


class fp_file_header(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32), ("header_bytes", ctypes.c_uint32),
                ("prm", fp_params), ("cube", fp_cube), ("n", ctypes.c_uint64), ("num_nodes", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("digest", ctypes.c_uint64), ("nodes_offset", ctypes.c_uint64),
                ("points_offset", ctypes.c_uint64), ("perm_offset", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 4)]


class fp_camera(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float * 16), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("min_node_px", ctypes.c_float), ("reserved", ctypes.c_uint32)]


FILE_HAS_PERM = 1
MAX_LANES = 32
PREVIEW_DONE = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
STAGE = dict(bounds=0, decimate=1, bounds_decimate=2, count=3, merge=4, distribute=5, octree=6, subsample=7,
             preview_spatial=8)
ERR_BITS = {1 << 6: "timeout", 1 << 9: "capacity"}
KERNEL = dict(none=0, bounds_decimate=1, count=2, distribute=3, cell_group=4, split_rounds=5, units=6, node_table=7,
              resolve=8, leaf_scatter=9, owner_scatter=10, stitch=11)
NODE_BYTES, CHUNK_BYTES, CUBE_BYTES = 40, 16, 32

_lib = None


def load():
    """Load libfastpoints.so (building it in-tree when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    p, u64, u32, sz, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "fp_workspace_size": (sz, [i32, u64, p]),
        "fp_status_string": (ctypes.c_char_p, [st]),
        "fp_node_capacity_bound": (u32, [u64, p]),
        "fp_get_device_error": (st, [p, p, i32]),
        "fp_get_device_error_sites": (st, [p, p]),
        "fp_time_kernel": (st, [i32, p, p]),
        "fp_debug_withhold_publish": (st, [u32, u32]),
        "fp_bounds": (st, [p, u64, p, p, sz, p]),
        "fp_decimate": (st, [p, u64, u64, u32, p, u64, p, p, sz, p]),
        "fp_preview_spatial": (st, [p, u64, p, u32, u64, p, u64, p, p, sz, p]),
        "fp_preview_modulus": (u32, [u64, u64]),
        "fp_bounds_decimate": (st, [p, u64, p, u64, u32, p, u64, p, p, sz, p]),
        "fp_count": (st, [p, u64, p, u32, p, i32, p, sz, p]),
        "fp_count_cells": (st, [p, u64, p, u32, p, i32, p, p, sz, p]),
        "fp_distribute_cells": (st, [p, p, u64, p, u32, p, p, p, p, p, p, sz, p]),
        "fp_merge_chunks": (st, [p, u32, u64, p, p, p, p, p, sz, p]),
        "fp_distribute": (st, [p, u64, p, u32, p, p, p, p, p, p, sz, p]),
        "fp_build_chunk_octree": (st, [p, p, u64, p, p, p, p, p, p, p, u32, p, p, p, p, p, sz, p]),
        "fp_subsample": (st, [p, p, u32, p, p, p, u64, p, p, p, p, p, p, sz, p]),
        "fp_batch_workspace_size": (sz, [p, u32, u32]),
        "fp_ooc_arena_min": (sz, [u64, p, u64]),
        "fp_ooc_host_bytes": (sz, [u64, p]),
        "fp_build_ooc": (st, [p, u64, p, u64, u64, p, sz, p, sz, p, p, u64, p, p, u32, p, p, p, PREVIEW_DONE, p, p]),
        "fp_build_batched": (st, [p, u32, u32, p, sz, p]),
        "fp_batch_workspace_size_ex": (sz, [p, u32, p]),
        "fp_build_batched_ex": (st, [p, u32, p, p, sz, p]),
        "fp_cloud_digest": (st, [p, u64, p, p]),
        "fp_render_workspace_size": (sz, [u32]),
        "fp_select_nodes": (st, [p, p, u32, p, p, p, p, p, p, sz, p]),
        "fp_rasterize": (st, [p, p, p, u32, p, u64, p, p, p, sz, p]),
        "fp_octree_save": (st, [ctypes.c_char_p, p, p, p, p, p, p, u64, u64, p, sz, p]),
        "fp_octree_read_header": (st, [ctypes.c_char_p, p]),
        "fp_octree_load": (st, [ctypes.c_char_p, p, u32, p, p, u64, u64, p, sz, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def declared_functions():
    """Names of the functions include/fastpoints.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:fp_status|size_t|uint32_t|const char\*)\s+(fp_\w+)\s*\(", text, re.M)))


def params(grid_log2=7, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=100000, node_capacity=20000):
    return fp_params(grid_log2, sub_log2, max_level, decim_modulus, chunk_threshold, node_capacity)


def _check(status, what):
    if status != 0:
        msg = load().fp_status_string(status).decode()
        raise FastPointsError("%s failed: %s (status %d)" % (what, msg, status))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _on_stream(fn):
    """Run a wrapper with its `stream` argument as torch's current stream, so that
    the temporaries it allocates (workspaces, outputs) belong to that stream:
    torch's caching allocator may hand a freed block to the next allocation at
    once, which is safe only when both are ordered on the same stream."""
    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def wrapper(*args, **kw):
        st = sig.bind_partial(*args, **kw).arguments.get("stream")
        if st is None:
            return fn(*args, **kw)
        with torch.cuda.stream(st):
            return fn(*args, **kw)
    return wrapper


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t):
    return t.device if t is not None else torch.device("cuda", torch.cuda.current_device())


def workspace_size(stage, n, prm=None):
    return int(load().fp_workspace_size(STAGE[stage], n, ctypes.byref(prm) if prm is not None else None))


def _ws(stage, n, prm, device, ws=None):
    need = workspace_size(stage, n, prm)
    if ws is not None and ws.numel() >= need:
        return ws, need
    return torch.empty(max(need, 1), dtype=torch.uint8, device=device), need


def as_points(x, device="cuda"):
    """numpy structured array / bytes / int32 (n, 4) tensor -> int32 (n, 4) CUDA tensor."""
    if isinstance(x, torch.Tensor):
        t = x
    else:
        import numpy as np
        a = np.ascontiguousarray(x).view(np.int32).reshape(-1, 4)
        t = torch.from_numpy(a)
    assert t.dtype == torch.int32 and t.dim() == 2 and t.shape[1] == 4
    return t.to(device).contiguous()


def time_kernel(kernel, start=None, stop=None):
    """Arm the kernel timing hook (fp_time_kernel): later calls that launch the
    named kernel record the two torch.cuda.Events around its launches."""
    k = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
    _check(load().fp_time_kernel(k, ctypes.c_void_p(start.cuda_event) if start is not None else None,
                                 ctypes.c_void_p(stop.cuda_event) if stop is not None else None), "fp_time_kernel")


def get_device_error_sites(stream=None):
    """Check sites (one bit each) that raised FP_ERR_CAPACITY since the last clear."""
    v = ctypes.c_uint32(0)
    _check(load().fp_get_device_error_sites(_stream(stream), ctypes.byref(v)), "fp_get_device_error_sites")
    return v.value


def get_device_error(stream=None, clear=True):
    v = ctypes.c_uint32(0)
    _check(load().fp_get_device_error(_stream(stream), ctypes.byref(v), int(clear)), "fp_get_device_error")
    return v.value


# ------------------------------------------------------------------ stages
@_on_stream
def fp_bounds(pts, stream=None, ws=None):
    n = pts.shape[0]
    cube = torch.empty(CUBE_BYTES // 4, dtype=torch.int32, device=_dev(pts))
    w, need = _ws("bounds", n, None, _dev(pts), ws)
    _check(load().fp_bounds(_ptr(pts), n, _ptr(cube), _ptr(w), w.numel(), _stream(stream)), "fp_bounds")
    return cube


def _preview_cap(n, modulus):
    # the kept count is a sum of n Bernoulli(1/m) draws: mean n/m, far below this bound
    return n if modulus <= 2 else min(n, n // modulus + 64 + 8 * int((n / modulus) ** 0.5 + 1) * 4)


@_on_stream
def fp_decimate(pts, first_index=0, modulus=16, out=None, stream=None, ws=None):
    n = pts.shape[0]
    cap = out.shape[0] if out is not None else _preview_cap(n, modulus)
    if out is None:
        out = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=_dev(pts))
    count = torch.zeros(1, dtype=torch.int64, device=_dev(pts))
    w, need = _ws("decimate", n, None, _dev(pts), ws)
    _check(load().fp_decimate(_ptr(pts), n, first_index, modulus, _ptr(out), cap, _ptr(count), _ptr(w), w.numel(),
                              _stream(stream)), "fp_decimate")
    return out, count


def fp_preview_modulus(n, target):
    """Modulus of a preview of about `target` points: max(1, ceil(n / target))."""
    return int(load().fp_preview_modulus(n, target))


@_on_stream
def fp_preview_spatial(pts, cube, level=7, first_index=0, out=None, stream=None, ws=None):
    """One random point (smallest index hash) per occupied cell of the 2^level
    grid, ascending index: (out, count)."""
    n = pts.shape[0]
    cap = out.shape[0] if out is not None else min(n, 1 << (3 * level))
    if out is None:
        out = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=_dev(pts))
    count = torch.zeros(1, dtype=torch.int64, device=_dev(pts))
    prm = params(grid_log2=level, sub_log2=level, max_level=level)
    w, need = _ws("preview_spatial", n, prm, _dev(pts), ws)
    _check(load().fp_preview_spatial(_ptr(pts), n, _ptr(cube), level, first_index, _ptr(out), cap, _ptr(count),
                                     _ptr(w), w.numel(), _stream(stream)), "fp_preview_spatial")
    return out, count


@_on_stream
def fp_bounds_decimate(pts, first_index=0, modulus=16, out=None, stream=None, ws=None):
    n = pts.shape[0]
    cap = out.shape[0] if out is not None else _preview_cap(n, modulus)
    if out is None:
        out = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=_dev(pts))
    cube = torch.empty(CUBE_BYTES // 4, dtype=torch.int32, device=_dev(pts))
    count = torch.zeros(1, dtype=torch.int64, device=_dev(pts))
    w, need = _ws("bounds_decimate", n, None, _dev(pts), ws)
    _check(load().fp_bounds_decimate(_ptr(pts), n, _ptr(cube), first_index, modulus, _ptr(out), cap, _ptr(count),
                                     _ptr(w), w.numel(), _stream(stream)), "fp_bounds_decimate")
    return cube, out, count


@_on_stream
def fp_count(pts, cube, grid_log2=7, counts=None, accumulate=False, stream=None):
    n = pts.shape[0]
    if counts is None:
        counts = torch.empty(1 << (3 * grid_log2), dtype=torch.int32, device=_dev(pts))
    _check(load().fp_count(_ptr(pts), n, _ptr(cube), grid_log2, _ptr(counts), int(accumulate), None, 0,
                           _stream(stream)), "fp_count")
    return counts


@_on_stream
def fp_count_cells(pts, cube, grid_log2=7, counts=None, cells=None, accumulate=False, stream=None):
    """fp_count that also returns every point's level-g Morton cell."""
    n = pts.shape[0]
    if counts is None:
        counts = torch.empty(1 << (3 * grid_log2), dtype=torch.int32, device=_dev(pts))
    if cells is None:
        cells = torch.empty(max(n, 1), dtype=torch.int32, device=_dev(pts))
    _check(load().fp_count_cells(_ptr(pts), n, _ptr(cube), grid_log2, _ptr(counts), int(accumulate), _ptr(cells),
                                 None, 0, _stream(stream)), "fp_count_cells")
    return counts, cells


@_on_stream
def fp_merge_chunks(counts, grid_log2, threshold, stream=None, ws=None):
    dev = counts.device
    cells = 1 << (3 * grid_log2)
    chunks = torch.empty((cells, CHUNK_BYTES // 8), dtype=torch.int64, device=dev)
    num = torch.zeros(1, dtype=torch.int32, device=dev)
    lut = torch.empty(cells, dtype=torch.int32, device=dev)
    offsets = torch.empty(cells + 1, dtype=torch.int64, device=dev)
    prm = params(grid_log2=grid_log2)
    w, need = _ws("merge", 0, prm, dev, ws)
    _check(load().fp_merge_chunks(_ptr(counts), grid_log2, threshold, _ptr(chunks), _ptr(num), _ptr(lut),
                                  _ptr(offsets), _ptr(w), w.numel(), _stream(stream)), "fp_merge_chunks")
    return chunks, num, lut, offsets


@_on_stream
def fp_distribute(pts, cube, grid_log2, lut, offsets, num_chunks, with_perm=True, out=None, perm=None,
                  stream=None, ws=None):
    n = pts.shape[0]
    dev = _dev(pts)
    if out is None:
        out = torch.empty_like(pts)
    if with_perm and perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=dev)
    prm = params(grid_log2=grid_log2)
    w, need = _ws("distribute", n, prm, dev, ws)
    _check(load().fp_distribute(_ptr(pts), n, _ptr(cube), grid_log2, _ptr(lut), _ptr(offsets), _ptr(num_chunks),
                                _ptr(out), _ptr(perm) if with_perm else None, _ptr(w), w.numel(), _stream(stream)),
           "fp_distribute")
    return out, perm


@_on_stream
def fp_distribute_cells(pts, cells, cube, grid_log2, lut, offsets, num_chunks, with_perm=True, out=None, perm=None,
                        stream=None, ws=None):
    """fp_distribute with the cells of fp_count_cells."""
    n = pts.shape[0]
    dev = _dev(pts)
    if out is None:
        out = torch.empty_like(pts)
    if with_perm and perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=dev)
    prm = params(grid_log2=grid_log2)
    w, need = _ws("distribute", n, prm, dev, ws)
    _check(load().fp_distribute_cells(_ptr(pts), _ptr(cells), n, _ptr(cube), grid_log2, _ptr(lut), _ptr(offsets),
                                      _ptr(num_chunks), _ptr(out), _ptr(perm) if with_perm else None, _ptr(w),
                                      w.numel(), _stream(stream)), "fp_distribute_cells")
    return out, perm


def node_capacity_bound(n, prm):
    return int(load().fp_node_capacity_bound(n, ctypes.byref(prm)))


@_on_stream
def fp_build_chunk_octree(sorted_pts, perm, cube, chunks, num_chunks, offsets, counts, prm, node_cap=None,
                          leaf=True, stream=None, ws=None):
    n = sorted_pts.shape[0]
    dev = _dev(sorted_pts)
    if node_cap is None:
        node_cap = node_capacity_bound(n, prm)
    nodes = torch.zeros((node_cap, NODE_BYTES // 8), dtype=torch.int64, device=dev)
    num_nodes = torch.zeros(1, dtype=torch.int32, device=dev)
    leaf_pts = torch.empty_like(sorted_pts) if leaf else None
    leaf_perm = torch.empty(n, dtype=torch.int32, device=dev) if leaf else None
    owner = torch.empty(n, dtype=torch.int32, device=dev)
    w, need = _ws("octree", n, prm, dev, ws)
    _check(load().fp_build_chunk_octree(_ptr(sorted_pts), _ptr(perm), n, _ptr(cube), _ptr(chunks), _ptr(num_chunks),
                                        _ptr(offsets), _ptr(counts), ctypes.byref(prm), _ptr(nodes), node_cap,
                                        _ptr(num_nodes), _ptr(leaf_pts), _ptr(leaf_perm), _ptr(owner), _ptr(w),
                                        w.numel(), _stream(stream)), "fp_build_chunk_octree")
    return nodes, num_nodes, leaf_pts, leaf_perm, owner


@_on_stream
def fp_subsample(nodes, num_nodes, sorted_pts, perm, owner, chunks, num_chunks, offsets, prm, stream=None, ws=None,
                 final=None, final_perm=None):
    """nodes must have been allocated with node_capacity_bound(n, prm) rows (the
    workspace size assumes that node_cap); chunks / num_chunks / offsets are
    fp_merge_chunks' outputs the points were distributed with."""
    n = sorted_pts.shape[0]
    dev = _dev(sorted_pts)
    if final is None:
        final = torch.empty_like(sorted_pts)
    if final_perm is None:
        final_perm = torch.empty(n, dtype=torch.int32, device=dev)
    w, need = _ws("subsample", n, prm, dev, ws)
    _check(load().fp_subsample(_ptr(nodes), _ptr(num_nodes), nodes.shape[0], _ptr(sorted_pts), _ptr(perm),
                               _ptr(owner), n, _ptr(chunks), _ptr(num_chunks), _ptr(offsets), _ptr(final),
                               _ptr(final_perm), _ptr(w), w.numel(), _stream(stream)),
           "fp_subsample")
    return final, final_perm


# ------------------------------------------------------------------ batches
def cloud_outputs(pts, prm, leaf=True):
    """Every output of the hot path for one cloud, allocated on the points' device
    (leaf=False: without the optional leaf-grouped points)."""
    n = pts.shape[0]
    dev = _dev(pts)
    cells = 1 << (3 * prm.grid_log2)
    ncap = node_capacity_bound(n, prm)
    cap = _preview_cap(n, prm.decim_modulus)
    i32 = dict(dtype=torch.int32, device=dev)
    return dict(cube=torch.zeros(8, **i32), preview=torch.empty((max(cap, 1), 4), **i32),
                preview_count=torch.zeros(1, dtype=torch.int64, device=dev), counts=torch.empty(cells, **i32),
                chunks=torch.empty((cells, 4), **i32), num_chunks=torch.zeros(1, **i32), lut=torch.empty(cells, **i32),
                offsets=torch.empty(cells + 1, dtype=torch.int64, device=dev), dist=torch.empty((max(n, 1), 4), **i32),
                perm=torch.empty(max(n, 1), **i32), nodes=torch.zeros((max(ncap, 1), 10), **i32),
                num_nodes=torch.zeros(1, **i32), leaf_pts=torch.empty((max(n, 1), 4), **i32) if leaf else None,
                leaf_perm=torch.empty(max(n, 1), **i32) if leaf else None, owner=torch.empty(max(n, 1), **i32),
                final=torch.empty((max(n, 1), 4), **i32), final_perm=torch.empty(max(n, 1), **i32),
                preview_cap=cap, node_cap=ncap)


def cloud_desc(pts, prm, out):
    d = fp_cloud_desc()
    P = lambda t: t.data_ptr() if t is not None else None
    d.d_pts, d.n, d.prm = P(pts), pts.shape[0], prm
    d.d_cube, d.d_preview, d.preview_cap, d.d_preview_count = P(out["cube"]), P(out["preview"]), out["preview_cap"], \
        P(out["preview_count"])
    d.d_counts, d.d_chunks, d.d_num_chunks = P(out["counts"]), P(out["chunks"]), P(out["num_chunks"])
    d.d_lut, d.d_offsets, d.d_dist, d.d_perm = P(out["lut"]), P(out["offsets"]), P(out["dist"]), P(out["perm"])
    d.d_nodes, d.node_cap, d.d_num_nodes = P(out["nodes"]), out["node_cap"], P(out["num_nodes"])
    d.d_leaf_pts, d.d_leaf_perm, d.d_owner = P(out["leaf_pts"]), P(out["leaf_perm"]), P(out["owner"])
    d.d_final, d.d_final_perm = P(out["final"]), P(out["final_perm"])
    return d


@_on_stream
def plain_calls(d, ws, stream=None):
    """The seven plain calls of one cloud (descriptor d), in order, on one stream."""
    L, S, W, Wn = load(), _stream(stream), _ptr(ws), ws.numel()
    g, T = d.prm.grid_log2, d.prm.chunk_threshold
    _check(L.fp_bounds_decimate(d.d_pts, d.n, d.d_cube, 0, d.prm.decim_modulus, d.d_preview, d.preview_cap,
                                d.d_preview_count, W, Wn, S), "fp_bounds_decimate")
    _check(L.fp_count(d.d_pts, d.n, d.d_cube, g, d.d_counts, 0, W, Wn, S), "fp_count")
    _check(L.fp_merge_chunks(d.d_counts, g, T, d.d_chunks, d.d_num_chunks, d.d_lut, d.d_offsets, W, Wn, S),
           "fp_merge_chunks")
    _check(L.fp_distribute(d.d_pts, d.n, d.d_cube, g, d.d_lut, d.d_offsets, d.d_num_chunks, d.d_dist, d.d_perm, W,
                           Wn, S), "fp_distribute")
    _check(L.fp_build_chunk_octree(d.d_dist, d.d_perm, d.n, d.d_cube, d.d_chunks, d.d_num_chunks, d.d_offsets,
                                   d.d_counts, ctypes.byref(d.prm), d.d_nodes, d.node_cap, d.d_num_nodes,
                                   d.d_leaf_pts, d.d_leaf_perm, d.d_owner, W, Wn, S), "fp_build_chunk_octree")
    _check(L.fp_subsample(d.d_nodes, d.d_num_nodes, d.node_cap, d.d_dist, d.d_perm, d.d_owner, d.n, d.d_chunks,
                          d.d_num_chunks, d.d_offsets, d.d_final, d.d_final_perm, W, Wn, S), "fp_subsample")


def batch_descs(clouds, outs):
    arr = (fp_cloud_desc * max(len(clouds), 1))()
    for i, ((pts, prm), out) in enumerate(zip(clouds, outs)):
        arr[i] = cloud_desc(pts, prm, out)
    return arr


class fp_batch_opts(ctypes.Structure):
    _fields_ = [("nlanes", ctypes.c_uint32), ("fused_first", ctypes.c_uint32), ("count_threads", ctypes.c_uint32),
                ("count_slots", ctypes.c_uint32)]


def batch_opts(nlanes=8, fused_first=0, count_threads=256, count_slots=1024):
    return fp_batch_opts(nlanes, int(fused_first), count_threads, count_slots)


def batch_workspace_size(descs, ncloud, nlanes):
    return int(load().fp_batch_workspace_size(descs, ncloud, nlanes))


def batch_workspace_size_ex(descs, ncloud, opts):
    return int(load().fp_batch_workspace_size_ex(descs, ncloud, ctypes.byref(opts)))


@_on_stream
def fp_build_batched_ex(descs, ncloud, opts, ws, stream=None):
    _check(load().fp_build_batched_ex(descs, ncloud, ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(stream)),
           "fp_build_batched_ex")


@_on_stream
def fp_build_batched(descs, ncloud, nlanes, ws, stream=None):
    _check(load().fp_build_batched(descs, ncloud, nlanes, _ptr(ws), ws.numel(), _stream(stream)), "fp_build_batched")


@_on_stream
def build_batched(clouds, nlanes=8, stream=None, outs=None, ws=None, opts=None):
    """clouds: list of (points tensor, fp_params).  Builds all of them with
    fp_build_batched (fp_build_batched_ex when opts is given); returns (list of
    output dicts, descriptors, workspace)."""
    if outs is None:
        outs = [cloud_outputs(p, prm) for p, prm in clouds]
    descs = batch_descs(clouds, outs)
    need = batch_workspace_size_ex(descs, len(clouds), opts) if opts is not None else \
        batch_workspace_size(descs, len(clouds), nlanes)
    dev = _dev(clouds[0][0]) if clouds else None
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    if opts is not None:
        fp_build_batched_ex(descs, len(clouds), opts, ws, stream=stream)
    else:
        fp_build_batched(descs, len(clouds), nlanes, ws, stream=stream)
    return outs, descs, ws


# ------------------------------------------------------------------ out of core
def ooc_host_bytes(n, prm):
    return int(load().fp_ooc_host_bytes(n, ctypes.byref(prm)))


def ooc_arena_min(n, prm, piece_points=1 << 23):
    return int(load().fp_ooc_arena_min(n, ctypes.byref(prm), piece_points))


def ooc_outputs(n, prm):
    """Pinned host outputs of fp_build_ooc for a cloud of n points."""
    ncap = node_capacity_bound(n, prm)
    cap = _preview_cap(n, prm.decim_modulus)
    pin = lambda *shape, dtype=torch.int32: torch.empty(shape, dtype=dtype).pin_memory()
    return dict(cube=pin(8), preview=pin(max(cap, 1), 4), preview_count=torch.zeros(1, dtype=torch.int64).pin_memory(),
                nodes=pin(max(ncap, 1), 10), num_nodes=torch.zeros(1, dtype=torch.int32).pin_memory(),
                final=pin(max(n, 1), 4), final_perm=pin(max(n, 1)), preview_cap=cap, node_cap=ncap)


@_on_stream
def build_ooc(host_pts, prm, arena, piece_points=1 << 23, group_points=0, scratch=None, out=None, on_preview=None,
              stream=None):
    """Out-of-core build of a cloud in pinned host memory ((n, 4) int32 CPU
    tensor) inside the device arena (uint8 CUDA tensor).  Blocks until done;
    on_preview() is called from a CUDA callback thread when the preview is in
    out["preview"].  Returns the pinned host outputs."""
    n = host_pts.shape[0]
    if out is None:
        out = ooc_outputs(n, prm)
    need = ooc_host_bytes(n, prm)
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(need, dtype=torch.uint8).pin_memory()
    cb = PREVIEW_DONE((lambda _u: on_preview()) if on_preview is not None else 0)
    st = load().fp_build_ooc(_ptr(host_pts), n, ctypes.byref(prm), piece_points, group_points, _ptr(arena),
                             arena.numel(),
                             _ptr(scratch), scratch.numel(), _ptr(out["cube"]), _ptr(out["preview"]),
                             out["preview_cap"], _ptr(out["preview_count"]), _ptr(out["nodes"]), out["node_cap"],
                             _ptr(out["num_nodes"]), _ptr(out["final"]), _ptr(out["final_perm"]), cb, None,
                             _stream(stream))
    _check(st, "fp_build_ooc")
    return out


# ------------------------------------------------------------------ decoding
def cube_to_host(cube):
    import numpy as np
    b = cube.cpu().numpy().view(np.uint8)
    o = b[0:12].view(np.int32)
    mx = b[12:24].view(np.int32)
    S = int(b[24:32].view(np.uint64)[0])
    return o.tolist(), mx.tolist(), S


def chunks_to_host(chunks, num):
    import numpy as np
    K = int(num.item())
    a = chunks[:K].cpu().numpy().view(np.uint8).reshape(K, 16)
    dt = np.dtype([("key", "<u8"), ("count", "<u4"), ("level", "<u4")])
    return a.copy().view(dt).reshape(K)


def nodes_to_host(nodes, num):
    import numpy as np
    M = int(num.item())
    a = nodes[:M].cpu().numpy().view(np.uint8).reshape(M, 40)
    dt = np.dtype([("key", "<u8"), ("first", "<u8"), ("leaf_first", "<u8"), ("count", "<u4"), ("n_own", "<u4"),
                   ("n_desc", "<u4"), ("level", "u1"), ("child_mask", "u1"), ("is_leaf", "u1"), ("pad", "u1")])
    return a.copy().view(dt).reshape(M)


@_on_stream
def build_octree(pts, prm, stream=None):
    """The whole hot path on one cloud (int32 (n, 4) CUDA tensor); returns a dict
    of device tensors: cube, preview (+count), counts, chunks (+count), lut,
    offsets, distributed points + perm, nodes (+count), leaf-grouped points +
    perm, owner per distributed point, final points + perm."""
    n = pts.shape[0]
    cube, prev, prev_n = fp_bounds_decimate(pts, 0, prm.decim_modulus, stream=stream)
    counts = fp_count(pts, cube, prm.grid_log2, stream=stream)
    chunks, num_chunks, lut, offsets = fp_merge_chunks(counts, prm.grid_log2, prm.chunk_threshold, stream=stream)
    dist, perm = fp_distribute(pts, cube, prm.grid_log2, lut, offsets, num_chunks, stream=stream)
    nodes, num_nodes, leaf_pts, leaf_perm, owner = fp_build_chunk_octree(dist, perm, cube, chunks, num_chunks, offsets,
                                                                         counts, prm, stream=stream)
    final, final_perm = fp_subsample(nodes, num_nodes, dist, perm, owner, chunks, num_chunks, offsets, prm,
                                     stream=stream)
    return dict(cube=cube, preview=prev, preview_count=prev_n, counts=counts, chunks=chunks, num_chunks=num_chunks,
                lut=lut, offsets=offsets, dist=dist, perm=perm, nodes=nodes, num_nodes=num_nodes, leaf_pts=leaf_pts,
                leaf_perm=leaf_perm, owner=owner, final=final, final_perm=final_perm)


# ------------------------------------------------------- octree file, cache
@_on_stream
def fp_cloud_digest(pts, stream=None):
    """64-bit digest of a cloud (every point and the order): the cache key."""
    d = torch.zeros(1, dtype=torch.int64, device=_dev(pts))
    _check(load().fp_cloud_digest(_ptr(pts), pts.shape[0], _ptr(d), _stream(stream)), "fp_cloud_digest")
    return int(d.item()) & 0xFFFFFFFFFFFFFFFF


def _staging(staging, nbytes=64 << 20):
    return staging if staging is not None else torch.empty(nbytes, dtype=torch.uint8).pin_memory()


@_on_stream
def octree_save(path, prm, out, digest=0, with_perm=True, staging=None, stream=None):
    """Writes the octree of build_octree() (device outputs: cube, nodes,
    num_nodes, final, final_perm) to one file."""
    stg = _staging(staging)
    n = out["final"].shape[0] if out.get("n") is None else out["n"]
    _check(load().fp_octree_save(os.fsencode(path), ctypes.byref(prm), _ptr(out["cube"]), _ptr(out["nodes"]),
                                 _ptr(out["num_nodes"]), _ptr(out["final"]),
                                 _ptr(out["final_perm"]) if with_perm else None, n, digest & 0xFFFFFFFFFFFFFFFF,
                                 _ptr(stg), stg.numel(), _stream(stream)), "fp_octree_save")


def octree_header(path):
    h = fp_file_header()
    _check(load().fp_octree_read_header(os.fsencode(path), ctypes.byref(h)), "fp_octree_read_header")
    return h


@_on_stream
def octree_load(path, nodes=True, first=0, count=None, perm=True, device=None, staging=None, stream=None):
    """Node table and final points [first, first + count) (all by default) of an
    octree file, as device tensors: dict(header, nodes, num_nodes, final, final_perm)."""
    h = octree_header(path)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    count = h.n - first if count is None else count
    stg = _staging(staging)
    d_nodes = torch.zeros((max(h.num_nodes, 1), NODE_BYTES // 8), dtype=torch.int64, device=dev) if nodes else None
    pts = torch.empty((max(count, 1), 4), dtype=torch.int32, device=dev)
    prm_ = torch.empty(max(count, 1), dtype=torch.int32, device=dev) if perm and (h.flags & FILE_HAS_PERM) else None
    _check(load().fp_octree_load(os.fsencode(path), _ptr(d_nodes), h.num_nodes, _ptr(pts), _ptr(prm_), first, count,
                                 _ptr(stg), stg.numel(), _stream(stream)), "fp_octree_load")
    num = torch.tensor([h.num_nodes], dtype=torch.int32, device=dev)
    return dict(header=h, nodes=d_nodes, num_nodes=num, final=pts[:count], final_perm=None if prm_ is None else prm_[:count])


def cache_path(cache_dir, digest, prm):
    key = "%016x_g%d_s%d_l%d_m%d_t%d_c%d" % (digest, prm.grid_log2, prm.sub_log2, prm.max_level, prm.decim_modulus,
                                             prm.chunk_threshold, prm.node_capacity)
    return os.path.join(cache_dir, key + ".fpo")


@_on_stream
def cached_build(pts, prm, cache_dir, stream=None, staging=None):
    """The octree of a cloud, from the cache when this cloud was built before
    with these parameters (same digest, same n), else built and saved.
    Returns (outputs, hit): outputs hold nodes, num_nodes, final, final_perm."""
    digest = fp_cloud_digest(pts, stream)
    path = cache_path(cache_dir, digest, prm)
    if os.path.exists(path):
        try:
            h = octree_header(path)
            if h.n == pts.shape[0] and h.digest == digest:
                return octree_load(path, device=pts.device, staging=staging, stream=stream), True
        except FastPointsError:
            pass   # unreadable entry: rebuilt and replaced below
    out = build_octree(pts, prm, stream=stream)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    octree_save(tmp, prm, out, digest=digest, staging=staging, stream=stream)
    os.replace(tmp, path)
    return out, False


# ------------------------------------------------------ rendering, headless
def view_projection(eye, target, up=(0.0, 0.0, 1.0), fovy_deg=60.0, aspect=16 / 9, near=1.0, far=1e7):
    """Row-major 4x4 perspective view-projection (clip z in [0, w]) as 16 fp32 values."""
    import numpy as np
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = r, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    proj = np.zeros((4, 4))
    proj[0, 0], proj[1, 1] = t / aspect, t
    proj[2, 2], proj[2, 3] = far / (near - far), near * far / (near - far)
    proj[3, 2] = -1.0
    return (proj @ view).astype(np.float32).reshape(16)


def camera(m, width, height, min_node_px):
    c = fp_camera()
    for i, v in enumerate(m):
        c.m[i] = float(v)
    c.width, c.height, c.min_node_px = width, height, min_node_px
    return c


def render_workspace_size(node_cap):
    return int(load().fp_render_workspace_size(node_cap))


@_on_stream
def fp_select_nodes(nodes, num_nodes, cube, cam, ws=None, stream=None):
    """(selected ids, count, total kept points) of the nodes the camera draws."""
    cap = nodes.shape[0]
    dev = nodes.device
    ids = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    npts = torch.zeros(1, dtype=torch.int64, device=dev)
    w = ws if ws is not None else torch.empty(max(render_workspace_size(cap), 1), dtype=torch.uint8, device=dev)
    _check(load().fp_select_nodes(_ptr(nodes), _ptr(num_nodes), cap, _ptr(cube), ctypes.byref(cam), _ptr(ids),
                                  _ptr(nsel), _ptr(npts), _ptr(w), w.numel(), _stream(stream)), "fp_select_nodes")
    return ids, nsel, npts


@_on_stream
def fp_rasterize(nodes, ids, nsel, final, cam, fb=None, ws=None, stream=None):
    """Framebuffer (height, width) int64: (depth bits << 32 | rgba) of the nearest point, -1 where empty."""
    cap = nodes.shape[0]
    dev = nodes.device
    if fb is None:
        fb = torch.empty((cam.height, cam.width), dtype=torch.int64, device=dev)
    w = ws if ws is not None else torch.empty(max(render_workspace_size(cap), 1), dtype=torch.uint8, device=dev)
    _check(load().fp_rasterize(_ptr(nodes), _ptr(ids), _ptr(nsel), cap, _ptr(final), final.shape[0],
                               ctypes.byref(cam), _ptr(fb), _ptr(w), w.numel(), _stream(stream)), "fp_rasterize")
    return fb
