"""Multithreaded CPU R-tree renderer (HiVision's pixel-driven method on the
host cores): a reported baseline for the benchmark, not part of the GPU
library and not the parity oracle.  Built with g++ into
``cpu_baseline/_build/librtree_mt.so``."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtree_mt.cpp")
_SO = os.path.join(_HERE, "_build", "librtree_mt.so")
_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.cpu_rtree_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]
        L.cpu_rtree_build.restype = ctypes.c_void_p
        L.cpu_rtree_free.argtypes = [ctypes.c_void_p]
        L.cpu_rtree_render_rgba.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_uint64] + [ctypes.c_void_p] * 2
        L.cpu_rtree_render_rgba.restype = ctypes.c_int
        _lib = L
    return _lib


class PointTree:
    """Packed Hilbert R-tree of points in host memory."""

    def __init__(self, xy, threads=0):
        xy = np.ascontiguousarray(xy, dtype=np.int32)
        self._h = _load().cpu_rtree_build(xy.ctypes.data, xy.shape[0], threads)

    def render_rgba(self, reqs, rgb):
        """(n, 4) [z, x, y, r16] -> (n, 262144) RGBA; returns (tiles, threads)."""
        r = np.ascontiguousarray(np.asarray(reqs, dtype=np.uint32).reshape(-1, 4))
        c = np.ascontiguousarray(np.asarray(rgb, dtype=np.uint8)[:3])
        out = np.zeros((r.shape[0], 262144), dtype=np.uint8)
        th = _load().cpu_rtree_render_rgba(self._h, r.ctypes.data, r.shape[0], c.ctypes.data, out.ctypes.data)
        return out, th

    def close(self):
        if self._h:
            _load().cpu_rtree_free(self._h)
            self._h = None

    def __del__(self):
        self.close()
