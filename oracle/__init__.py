"""Parity oracle for the display-driven tile renderer.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
Nothing here is imported by the product package, and nothing here imports it.

Two independent implementations of the same definition (HiVision Sec. 3.2,
Algorithm 1 for points / lines / outlines, Algorithm 2 for polygon fill):

* ``hv_oracle.c`` (wrapped below): data driven, one pass over the objects,
  exact int64 / unsigned 128-bit arithmetic, single threaded.
* ``brute.py``: pixel driven, pure-Python integers and fractions, for tiny
  layers and small pixel windows.  It pins the C oracle (brute force on tiny
  inputs must agree byte for byte).

Requests are ``(n, 4)`` uint32 arrays with columns ``z, x, y, r16``.
Output is ``(n, tile_bytes(mode))`` uint8, the same byte layout the library
documents for its output buffers.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "hv_oracle.c")
_SO = os.path.join(_BUILD, "liboracle.so")

MODE_MASK, MODE_COVERAGE, MODE_RGBA = 0, 1, 2
TILE = 256

_lib = None


def compile_source(src: str, so: str) -> str:
    """Compile a C oracle source file into a shared library."""
    tmp = so + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                           "-Wextra", "-o", tmp, src])
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_source(_SRC, _SO)
    return _SO


def bind(path: str):
    """Load an oracle shared library and declare its entry points."""
    lib = ctypes.CDLL(path)
    p = ctypes.c_void_p
    u64 = ctypes.c_uint64
    i64 = ctypes.c_int64
    lib.oracle_render_points.argtypes = [p, u64, p, p, p, p, u64, ctypes.c_int, p, p]
    lib.oracle_render_lines.argtypes = [p, u64, p, u64, p, p, p, p, u64, ctypes.c_int, p, p]
    lib.oracle_render_polygons.argtypes = [p, u64, p, u64, p, u64, p, p, p, p, u64,
                                           ctypes.c_int, p, p]
    lib.oracle_render_points_r.argtypes = [p, u64, p, p, p, p, u64, i64, ctypes.c_int, p, p]
    lib.oracle_render_lines_r.argtypes = [p, u64, p, u64, p, p, p, p, u64, i64, ctypes.c_int, p, p]
    lib.oracle_render_polygons_r.argtypes = [p, u64, p, u64, p, u64, p, p, p, p, u64, i64,
                                             ctypes.c_int, p, p]
    lib.oracle_render_polygons_styled.argtypes = [p, u64, p, u64, p, u64, p, p, p, p, u64, i64, ctypes.c_int,
                                                  p, ctypes.c_int, p, ctypes.c_uint32, ctypes.c_uint32, p]
    lib.oracle_render_polygons_styled.restype = ctypes.c_int
    for f in (lib.oracle_render_points, lib.oracle_render_lines, lib.oracle_render_polygons,
              lib.oracle_render_points_r, lib.oracle_render_lines_r, lib.oracle_render_polygons_r):
        f.restype = ctypes.c_int
    lib.oracle_tile_bytes.argtypes = [ctypes.c_int]
    lib.oracle_tile_bytes.restype = u64
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def tile_bytes(mode: int) -> int:
    return {MODE_MASK: TILE * TILE // 8, MODE_COVERAGE: TILE * TILE, MODE_RGBA: TILE * TILE * 4}[mode]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _req_cols(reqs):
    r = np.ascontiguousarray(np.asarray(reqs, dtype=np.uint32).reshape(-1, 4))
    return [np.ascontiguousarray(r[:, k]) for k in range(4)], r.shape[0]


def _style(style):
    s = np.zeros(8, dtype=np.uint8)
    if style is not None:
        s[:] = np.asarray(style, dtype=np.uint8).reshape(8)
    return s


def _check(rc):
    if rc == -2:
        raise ValueError("oracle: request or coordinate out of range")
    if rc != 0:
        raise MemoryError("oracle: allocation failed")


def render_points(xy, reqs, mode, style=None, lib=None, R_units=None):
    """Points ``xy`` (n, 2) int32 -> (n_req, tile_bytes) uint8.  ``R_units``:
    one radius in grid units for every request (buffer analysis) instead of
    each request's r16."""
    lib = _load(lib)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    cols, n = _req_cols(reqs)
    st = _style(style)
    out = np.zeros((n, tile_bytes(mode)), dtype=np.uint8)
    args = (_ptr(xy), xy.shape[0], *[_ptr(c) for c in cols], n)
    if R_units is None:
        _check(lib.oracle_render_points(*args, mode, _ptr(st), _ptr(out)))
    else:
        _check(lib.oracle_render_points_r(*args, int(R_units), mode, _ptr(st), _ptr(out)))
    return out


def render_lines(xy, line_off, reqs, mode, style=None, lib=None, R_units=None):
    """Linestrings: vertices ``xy`` (V, 2), line l = vertices [off[l], off[l+1])."""
    lib = _load(lib)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    off = np.ascontiguousarray(np.asarray(line_off, dtype=np.uint64))
    cols, n = _req_cols(reqs)
    st = _style(style)
    out = np.zeros((n, tile_bytes(mode)), dtype=np.uint8)
    args = (_ptr(xy), xy.shape[0], _ptr(off), off.shape[0] - 1, *[_ptr(c) for c in cols], n)
    if R_units is None:
        _check(lib.oracle_render_lines(*args, mode, _ptr(st), _ptr(out)))
    else:
        _check(lib.oracle_render_lines_r(*args, int(R_units), mode, _ptr(st), _ptr(out)))
    return out


def render_polygons(xy, ring_off, poly_ring_off, reqs, mode, style=None, lib=None, R_units=None, aa=False,
                    pattern=None):
    """Polygons: ring r = vertices [ring_off[r], ring_off[r+1]) (closed implicitly),
    polygon p = rings [poly_ring_off[p], poly_ring_off[p+1]).  ``aa``: the
    fill decided at the four super-samples (COVERAGE byte = v | f << 4);
    ``pattern``: (h, w, 4) uint8 RGBA texels over the global pixel grid."""
    lib = _load(lib)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    ro = np.ascontiguousarray(np.asarray(ring_off, dtype=np.uint64))
    po = np.ascontiguousarray(np.asarray(poly_ring_off, dtype=np.uint64))
    cols, n = _req_cols(reqs)
    st = _style(style)
    out = np.zeros((n, tile_bytes(mode)), dtype=np.uint8)
    args = (_ptr(xy), xy.shape[0], _ptr(ro), ro.shape[0] - 1, _ptr(po), po.shape[0] - 1,
            *[_ptr(c) for c in cols], n)
    if aa or pattern is not None:
        pat = None if pattern is None else np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8))
        ph, pw = (0, 0) if pat is None else pat.shape[:2]
        _check(lib.oracle_render_polygons_styled(*args, -1 if R_units is None else int(R_units), mode, _ptr(st),
                                                 int(bool(aa)), None if pat is None else _ptr(pat), pw, ph,
                                                 _ptr(out)))
    elif R_units is None:
        _check(lib.oracle_render_polygons(*args, mode, _ptr(st), _ptr(out)))
    else:
        _check(lib.oracle_render_polygons_r(*args, int(R_units), mode, _ptr(st), _ptr(out)))
    return out


def mask_bits(tile_mask_bytes):
    """Unpack one MASK tile (8192 bytes) into a (256, 256) bool array [row, col]."""
    words = np.frombuffer(np.asarray(tile_mask_bytes, dtype=np.uint8).tobytes(), dtype="<u4")
    words = words.reshape(TILE, TILE // 32)
    bits = (words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(TILE, TILE).astype(bool)
