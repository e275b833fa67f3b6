"""Seeded synthetic point clouds for tests and benchmarks.

Holds no octree arithmetic: it only writes 16-byte point records
(int32 x, y, z, uint8 r, g, b, a) that both the CUDA library and the oracle
receive unchanged.  The generators are plain C (``fp_synth.c``), threaded,
counter-based, so any slice of a cloud can be produced on its own.

Workloads (the synthetic stand-ins for the paper's NEON / Great Hall /
Oplontis scans, Sec. 5, which are not available here):
  * ``uniform(n, seed, bits=20)``  x, y, z uniform in [0, 2^bits)^3, RGBA uniform
  * ``lidar(n, seed)``             scanner scene, density ~ 1/r^2 (see fp_synth.c)
  * ``batch_sizes(count, seed, lo, hi)`` log-uniform cloud sizes for batched runs
"""
import ctypes
import math
import os
import subprocess

import numpy as np

POINT_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                        ("r", "u1"), ("g", "u1"), ("b", "u1"), ("a", "u1")])
assert POINT_DTYPE.itemsize == 16

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fp_synth.c")
_LIB = os.path.join(_HERE, "lib", "libfpsynth.so")
_lib = None


def build(force=False):
    """Compile the generator library with gcc (portable C, no -march flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-pthread", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, ptr = ctypes.c_uint64, ctypes.c_void_p
        lib.syn_uniform.argtypes = [u64, u64, u64, ctypes.c_uint32, ptr, ctypes.c_int]
        lib.syn_lidar.argtypes = [u64, u64, u64, ptr, ctypes.c_int]
        lib.syn_draw.argtypes = [u64, u64, ctypes.c_uint]
        lib.syn_draw.restype = u64
        _lib = lib
    return _lib


def _threads(threads):
    return threads if threads else max(1, min(64, os.cpu_count() or 1))


def _out(n, out):
    if out is None:
        return np.empty(n, dtype=POINT_DTYPE)
    arr = np.asarray(out)
    assert arr.nbytes >= 16 * n and arr.flags["C_CONTIGUOUS"]
    return arr


def _ptr(arr):
    return arr.ctypes.data if isinstance(arr, np.ndarray) else int(arr)


def uniform(n, seed, bits=20, first=0, out=None, threads=None):
    """n points with x, y, z uniform in [0, 2^bits); point i of the cloud is
    the same bytes whatever slice it is generated in."""
    arr = _out(n, out)
    _load().syn_uniform(seed, first, n, bits, _ptr(arr), _threads(threads))
    return arr


def lidar(n, seed, first=0, out=None, threads=None):
    """n points of the synthetic scanner scene with the given seed."""
    arr = _out(n, out)
    _load().syn_lidar(seed, first, n, _ptr(arr), _threads(threads))
    return arr


def uniform_into(ptr, n, seed, bits=20, first=0, threads=None):
    """Write into raw host memory (e.g. a pinned torch tensor's data_ptr())."""
    _load().syn_uniform(seed, first, n, bits, ctypes.c_void_p(ptr), _threads(threads))


def lidar_into(ptr, n, seed, first=0, threads=None):
    _load().syn_lidar(seed, first, n, ctypes.c_void_p(ptr), _threads(threads))


def draw(seed, i, k):
    """k-th counter-based draw for item i of stream `seed` (64-bit)."""
    return int(_load().syn_draw(seed, i, k))


def batch_sizes(count, seed, lo, hi):
    """Cloud sizes n_i = floor(exp(U(ln lo, ln hi))) and a generator choice per
    cloud (0 = uniform cube, 1 = lidar), from the counter-based stream."""
    sizes, kinds = [], []
    for i in range(count):
        u = (draw(seed, i, 0) >> 11) / float(1 << 53)
        sizes.append(int(math.floor(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
        kinds.append(int(draw(seed, i, 1) & 1))
    return sizes, kinds


def to_bytes(arr):
    return np.ascontiguousarray(arr).view(np.uint8).reshape(-1, 16)
