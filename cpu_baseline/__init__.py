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
        P = ctypes.c_void_p
        L.cpu_rtree_build.argtypes = [P, ctypes.c_uint64, ctypes.c_int]
        L.cpu_rtree_build.restype = P
        L.cpu_rtree_build_lines.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int]
        L.cpu_rtree_build_lines.restype = P
        L.cpu_rtree_build_polygons.argtypes = [P, P, P, ctypes.c_uint64, ctypes.c_int]
        L.cpu_rtree_build_polygons.restype = P
        L.cpu_rtree_free.argtypes = [P]
        L.cpu_rtree_render.argtypes = [P, P, ctypes.c_uint64, P, P]
        L.cpu_rtree_render.restype = ctypes.c_int
        L.cpu_rtree_render_rgba.argtypes = [P, P, ctypes.c_uint64, P, P]
        L.cpu_rtree_render_rgba.restype = ctypes.c_int
        _lib = L
    return _lib


class _Tree:
    _h = None

    def render(self, reqs, style):
        """(n, 4) [z, x, y, r16] -> (n, 262144) RGBA with style (line r, g, b,
        a, fill r, g, b, a); returns (tiles, threads)."""
        r = np.ascontiguousarray(np.asarray(reqs, dtype=np.uint32).reshape(-1, 4))
        st = np.zeros(8, dtype=np.uint8)
        st[:len(style)] = np.asarray(style, dtype=np.uint8)[:8]
        out = np.zeros((r.shape[0], 262144), dtype=np.uint8)
        th = _load().cpu_rtree_render(self._h, r.ctypes.data, r.shape[0], st.ctypes.data, out.ctypes.data)
        return out, th

    def close(self):
        if self._h:
            _load().cpu_rtree_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


class PointTree(_Tree):
    """Packed Hilbert R-tree of points in host memory."""

    def __init__(self, xy, threads=0):
        xy = np.ascontiguousarray(xy, dtype=np.int32)
        self._h = _load().cpu_rtree_build(xy.ctypes.data, xy.shape[0], threads)

    def render_rgba(self, reqs, rgb):
        """(n, 4) [z, x, y, r16] -> (n, 262144) RGBA in the line colour."""
        return self.render(reqs, tuple(rgb[:3]) + (0, 0, 0, 0, 0))


class LineTree(_Tree):
    """Linestrings (vertices xy, line offsets) as a packed R-tree of segments."""

    def __init__(self, xy, line_off, threads=0):
        self._xy = np.ascontiguousarray(xy, dtype=np.int32)
        self._off = np.ascontiguousarray(line_off, dtype=np.uint64)
        self._h = _load().cpu_rtree_build_lines(self._xy.ctypes.data, self._off.ctypes.data,
                                                len(self._off) - 1, threads)


class PolygonTree(_Tree):
    """Polygons (vertices, ring offsets, per-polygon ring offsets): an R-tree of
    edges for the outline and one of polygon boxes for the fill."""

    def __init__(self, xy, ring_off, poly_ring_off, threads=0):
        self._xy = np.ascontiguousarray(xy, dtype=np.int32)
        self._ro = np.ascontiguousarray(ring_off, dtype=np.uint64)
        self._po = np.ascontiguousarray(poly_ring_off, dtype=np.uint64)
        self._h = _load().cpu_rtree_build_polygons(self._xy.ctypes.data, self._ro.ctypes.data,
                                                   self._po.ctypes.data, len(self._po) - 1, threads)
