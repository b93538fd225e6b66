"""ctypes binding of libhivision (argument marshalling only).

Every function has the name of the C entry point it calls (include/hivision.h)
and raises ``HVError`` when the call returns a non-zero status.  Array
arguments may be numpy arrays (host memory), torch tensors (host or device;
their ``data_ptr()`` is passed) or raw integer addresses.  Streams may be a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2005_12489_gb300.build``); there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhivision.so")

HV_OK, HV_EINVAL, HV_ERANGE, HV_ENOMEM, HV_ECUDA, HV_ETIMEOUT, HV_EBUSY, HV_ESTATE = range(8)
STATUS_NAMES = ["HV_OK", "HV_EINVAL", "HV_ERANGE", "HV_ENOMEM", "HV_ECUDA", "HV_ETIMEOUT",
                "HV_EBUSY", "HV_ESTATE"]
HV_MODE_MASK, HV_MODE_COVERAGE, HV_MODE_RGBA = 0, 1, 2
HV_LAYER_POINTS, HV_LAYER_LINES, HV_LAYER_POLYGONS = 0, 1, 2
HV_INDEX_RTREE, HV_INDEX_LEARNED = 1, 2
HV_OVERLAY_AND, HV_OVERLAY_OR, HV_OVERLAY_XOR, HV_OVERLAY_DIFF = 0, 1, 2, 3
HV_FILL_AA = 1
HV_LEARNED_NO_MLP = 0xFFFFFFFF     # hv_build_opts.learned_hidden: linear pieces only
HV_PLACE_DEVICE, HV_PLACE_HOST = 0, 1

REQ_DTYPE = np.dtype([("x", "<u4"), ("y", "<u4"), ("r16", "<u2"), ("z", "u1"), ("mode", "u1"),
                      ("layer", "<u4")])
assert REQ_DTYPE.itemsize == 16


class HVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


class hv_style(ctypes.Structure):
    _fields_ = [("line_rgba", ctypes.c_uint8 * 4), ("fill_rgba", ctypes.c_uint8 * 4)]


class hv_fill_style(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("pattern_w", ctypes.c_uint32), ("pattern_h", ctypes.c_uint32),
                ("pattern_rgba", ctypes.c_void_p)]


class hv_build_opts(ctypes.Structure):
    _fields_ = [("learned_segments", ctypes.c_uint32), ("learned_hidden", ctypes.c_uint32),
                ("learned_steps", ctypes.c_uint32), ("learned_seed", ctypes.c_uint32),
                ("max_error", ctypes.c_uint32), ("object_placement", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


class hv_layer_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("indexes", ctypes.c_uint32),
                ("n_objects", ctypes.c_uint64), ("n_polygons", ctypes.c_uint64),
                ("mbr", ctypes.c_int32 * 4), ("tree_levels", ctypes.c_uint32),
                ("tree_nodes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("learned_error", ctypes.c_int64), ("learned_outliers", ctypes.c_uint64),
                ("build_ms", ctypes.c_double), ("train_ms", ctypes.c_double),
                ("learned_error_linear", ctypes.c_int64), ("learned_error_mlp", ctypes.c_int64),
                ("learned_mean_error", ctypes.c_double), ("learned_pieces", ctypes.c_uint32),
                ("learned_mlp", ctypes.c_uint32), ("learned_halo", ctypes.c_int32),
                ("piece_extent", ctypes.c_int32), ("index_records", ctypes.c_uint64),
                ("learned_mean_window", ctypes.c_double), ("learned_mean_window_linear", ctypes.c_double),
                ("host_bytes", ctypes.c_uint64)]


class hv_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("queue_capacity", ctypes.c_uint32),
                ("scratch_bytes", ctypes.c_uint64), ("index_kind", ctypes.c_uint32),
                ("use_graphs", ctypes.c_uint32), ("style", hv_style), ("pool", ctypes.c_void_p)]


class hv_pool_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("hits", "misses", "inserts", "evictions", "expirations",
                                                "rejected", "entries", "bytes", "capacity")]


class hv_done(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("bytes", ctypes.c_uint32),
                ("data", ctypes.c_void_p), ("t_submit_us", ctypes.c_double),
                ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


_lib = None
P = ctypes.c_void_p
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
I32 = ctypes.c_int

SIGNATURES = {
    "hv_create": [ctypes.POINTER(P), I32, U64],
    "hv_lonlat_to_grid": [P, U64, P],
    "hv_route_tiles": [P, U64, U32, P],
    "hv_destroy": [P],
    "hv_last_error": [],
    "hv_ctx_device_bytes": [P, ctypes.POINTER(U64)],
    "hv_layer_load_points": [P, P, U64, ctypes.POINTER(P)],
    "hv_layer_load_linestrings": [P, P, U64, P, U64, ctypes.POINTER(P)],
    "hv_layer_load_polygons": [P, P, U64, P, U64, P, U64, ctypes.POINTER(P)],
    "hv_layer_build_index": [P, U32, P],
    "hv_layer_info_get": [P, ctypes.POINTER(hv_layer_info)],
    "hv_layer_keys": [P, I32, P, U64],
    "hv_learned_lookup": [P, I32, P, U32, P, ctypes.POINTER(U64), P],
    "hv_layer_free": [P],
    "hv_layer_save": [P, ctypes.c_char_p],
    "hv_layer_load_file": [P, ctypes.c_char_p, ctypes.POINTER(P)],
    "hv_tile_bytes": [I32],
    "hv_render_tiles": [P, P, U32, I32, I32, P, P, U64, P],
    "hv_render_tiles_static": [P, P, U32, I32, I32, P, P, U64, P],
    "hv_layer_take_status": [P, P, ctypes.POINTER(U32)],
    "hv_render_tiles_counted": [P, P, U32, I32, I32, P, P, U64, P, U64, P, P],
    "hv_render_tiles_phases": [P, P, U32, I32, I32, P, P, U64, P, P],
    "hv_render_launches": [P, I32, ctypes.POINTER(U32)],
    "hv_render_buffer": [P, P, U32, I32, I32, ctypes.c_int32, P, P, U64, P],
    "hv_render_tiles_styled": [P, P, U32, I32, I32, P, P, P, U64, P],
    "hv_overlay_tiles": [P, ctypes.c_int32, P, ctypes.c_int32, I32, P, U32, I32, P, U64, P],
    "hv_server_start": [P, P, U32, ctypes.POINTER(hv_server_opts), ctypes.POINTER(P)],
    "hv_server_submit": [P, P, U64],
    "hv_server_poll": [P, ctypes.POINTER(hv_done), U32, ctypes.POINTER(U32)],
    "hv_server_stop": [P],
    "hv_server_replay": [P, P, P, U64, P, ctypes.POINTER(ctypes.c_double)],
    "hv_server_replay_detail": [P, P, P, U64, P, P, ctypes.POINTER(ctypes.c_double)],
    "hv_server_stats": [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U32)],
    "hv_server_shortcuts": [P, ctypes.POINTER(U64), ctypes.POINTER(U64)],
    "hv_result_pool_create": [U64, U32, ctypes.POINTER(P)],
    "hv_result_pool_destroy": [P],
    "hv_result_pool_put": [P, P, P, P, U64],
    "hv_result_pool_get": [P, P, P, P, U64, ctypes.POINTER(U32)],
    "hv_result_pool_stats": [P, ctypes.POINTER(hv_pool_stats)],
    "hv_result_pool_clear": [P],
}


def lib():
    """Load libhivision.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhivision.so is not built (%s); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.hv_last_error.restype = ctypes.c_char_p
        L.hv_tile_bytes.restype = U64
        _lib = L
    return _lib


def _check(rc):
    if rc != HV_OK:
        raise HVError(rc, lib().hv_last_error().decode(errors="replace"))


def ptr(a):
    """Address of a numpy array, torch tensor, ctypes object or int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    return ctypes.addressof(a)


def stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hv_last_error():
    return lib().hv_last_error().decode(errors="replace")


def hv_tile_bytes(mode):
    return int(lib().hv_tile_bytes(mode))


def hv_lonlat_to_grid(lonlat):
    """(n, 2) degrees (lon, lat) -> (n, 2) int32 grid coordinates."""
    a = np.ascontiguousarray(np.asarray(lonlat, dtype=np.float64).reshape(-1, 2))
    out = np.zeros(a.shape, dtype=np.int32)
    _check(lib().hv_lonlat_to_grid(ptr(a), a.shape[0], ptr(out)))
    return out


def hv_route_tiles(reqs, n_ranks):
    """Rank (0..n_ranks-1) of every request: a hash of its (layer, z, x, y)."""
    r = reqs if isinstance(reqs, np.ndarray) and reqs.dtype == REQ_DTYPE else make_requests(reqs)
    r = np.ascontiguousarray(r)
    out = np.zeros(len(r), dtype=np.uint32)
    _check(lib().hv_route_tiles(ptr(r), len(r), n_ranks, ptr(out)))
    return out


def hv_create(device=0, mem_budget=0):
    out = P()
    _check(lib().hv_create(ctypes.byref(out), device, mem_budget))
    return out.value


def hv_destroy(ctx):
    _check(lib().hv_destroy(ctx))


def hv_ctx_device_bytes(ctx):
    out = U64()
    _check(lib().hv_ctx_device_bytes(ctx, ctypes.byref(out)))
    return out.value


def _i32xy(xy):
    if isinstance(xy, np.ndarray):
        return np.ascontiguousarray(xy, dtype=np.int32)
    return xy


def _u64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def hv_layer_load_points(ctx, xy, n=None):
    xy = _i32xy(xy)
    n = (xy.shape[0] if n is None else n)
    out = P()
    _check(lib().hv_layer_load_points(ctx, ptr(xy), n, ctypes.byref(out)))
    return out.value


def hv_layer_load_linestrings(ctx, xy, line_off):
    xy = _i32xy(xy)
    off = _u64(line_off)
    out = P()
    _check(lib().hv_layer_load_linestrings(ctx, ptr(xy), int(off[-1]), ptr(off), off.shape[0] - 1,
                                           ctypes.byref(out)))
    return out.value


def hv_layer_load_polygons(ctx, xy, ring_off, poly_ring_off):
    xy = _i32xy(xy)
    ro, po = _u64(ring_off), _u64(poly_ring_off)
    out = P()
    _check(lib().hv_layer_load_polygons(ctx, ptr(xy), int(ro[-1]), ptr(ro), ro.shape[0] - 1, ptr(po),
                                        po.shape[0] - 1, ctypes.byref(out)))
    return out.value


def hv_layer_build_index(layer, kinds=HV_INDEX_RTREE, opts=None):
    _check(lib().hv_layer_build_index(layer, kinds, ctypes.byref(opts) if opts is not None else None))


def hv_layer_info_get(layer):
    info = hv_layer_info()
    _check(lib().hv_layer_info_get(layer, ctypes.byref(info)))
    return info


def hv_layer_keys(layer, which, out, n):
    _check(lib().hv_layer_keys(layer, which, ptr(out), n))


def hv_learned_lookup(layer, which, keys, n, out, stream=None):
    """Returns the number of lookups answered by the full-search fallback."""
    fb = U64()
    _check(lib().hv_learned_lookup(layer, which, ptr(keys), n, ptr(out), ctypes.byref(fb),
                                   stream_handle(stream)))
    return fb.value


def info_dict(layer):
    i = hv_layer_info_get(layer)
    return {name: (list(getattr(i, name)) if name == "mbr" else getattr(i, name)) for name, _ in i._fields_}


def hv_layer_free(layer):
    _check(lib().hv_layer_free(layer))


def hv_layer_save(layer, path):
    _check(lib().hv_layer_save(layer, os.fsencode(path)))


def hv_layer_load_file(ctx, path):
    out = P()
    _check(lib().hv_layer_load_file(ctx, os.fsencode(path), ctypes.byref(out)))
    return out.value


def make_requests(zxyr, mode=0, layer=0):
    """(n, 4) [z, x, y, r16] -> packed hv_tile_req records (numpy)."""
    a = np.asarray(zxyr, dtype=np.int64).reshape(-1, 4)
    r = np.zeros(a.shape[0], dtype=REQ_DTYPE)
    r["z"], r["x"], r["y"], r["r16"] = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    r["mode"] = mode
    r["layer"] = layer
    return r


def make_style(line=(0, 0, 0), fill=(0, 0, 0)):
    s = hv_style()
    for k in range(3):
        s.line_rgba[k] = line[k]
        s.fill_rgba[k] = fill[k]
    return s


def hv_render_tiles(layer, reqs, n, mode, index_kind, style, out, out_bytes, stream=None):
    """reqs / out: numpy arrays, torch tensors or addresses (host or device)."""
    _check(lib().hv_render_tiles(layer, ptr(reqs), n, mode, index_kind,
                                 ctypes.byref(style) if style is not None else None, ptr(out),
                                 out_bytes, stream_handle(stream)))


def hv_render_tiles_counted(layer, reqs, n, mode, index_kind, style, out, out_bytes, log, log_cap,
                            log_count, stream=None):
    _check(lib().hv_render_tiles_counted(layer, ptr(reqs), n, mode, index_kind,
                                         ctypes.byref(style) if style is not None else None, ptr(out),
                                         out_bytes, ptr(log), log_cap, ptr(log_count),
                                         stream_handle(stream)))


PHASE_NAMES = ["total", "prologue", "cull", "bin", "blocks_cta", "blocks_warp", "leaf", "descend", "encode",
               "ctas", "blocks", "leaf_visits", "node_visits", "frontier_tests", "leaf_empty", "leaf_decided"]
HV_PHASE_COUNT = 16


def hv_render_tiles_phases(layer, reqs, n, mode, index_kind, style, out, out_bytes, phases, stream=None):
    """Instrumented render: adds per-phase warp-cycles into `phases` (device,
    HV_PHASE_COUNT uint64, twice that for polygon layers)."""
    _check(lib().hv_render_tiles_phases(layer, ptr(reqs), n, mode, index_kind,
                                        ctypes.byref(style) if style is not None else None, ptr(out),
                                        out_bytes, ptr(phases), stream_handle(stream)))


def hv_render_tiles_static(layer, reqs, n, mode, index_kind, style, out, out_bytes, stream=None):
    """Allocation-free rendering: `out` must be device memory (see the header)."""
    _check(lib().hv_render_tiles_static(layer, ptr(reqs), n, mode, index_kind,
                                        ctypes.byref(style) if style is not None else None, ptr(out),
                                        out_bytes, stream_handle(stream)))


def make_fill_style(aa=False, pattern=None):
    """A fill style: anti-aliased fill and / or a (h, w, 4) uint8 RGBA pattern.
    The returned structure keeps the pattern array alive."""
    f = hv_fill_style()
    f.flags = HV_FILL_AA if aa else 0
    if pattern is not None:
        pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8))
        f.pattern_h, f.pattern_w = pat.shape[:2]
        f.pattern_rgba = pat.ctypes.data
        f._pattern = pat
    return f


def hv_render_tiles_styled(layer, reqs, n, mode, index_kind, style, fill, out, out_bytes, stream=None):
    _check(lib().hv_render_tiles_styled(layer, ptr(reqs), n, mode, index_kind,
                                        ctypes.byref(style) if style is not None else None,
                                        ctypes.byref(fill) if fill is not None else None, ptr(out), out_bytes,
                                        stream_handle(stream)))


def hv_render_buffer(layer, reqs, n, mode, index_kind, radius_units, style, out, out_bytes, stream=None):
    """hv_render_tiles with one radius in grid units for every tile."""
    _check(lib().hv_render_buffer(layer, ptr(reqs), n, mode, index_kind, radius_units,
                                  ctypes.byref(style) if style is not None else None, ptr(out), out_bytes,
                                  stream_handle(stream)))


def hv_overlay_tiles(layer_a, radius_a, layer_b, radius_b, op, reqs, n, index_kind, out, out_bytes, stream=None):
    """MASK tiles of op(buffer of layer_a at radius_a, buffer of layer_b at radius_b)."""
    _check(lib().hv_overlay_tiles(layer_a, radius_a, layer_b, radius_b, op, ptr(reqs), n, index_kind, ptr(out),
                                  out_bytes, stream_handle(stream)))


def hv_layer_take_status(layer, stream=None):
    out = U32()
    _check(lib().hv_layer_take_status(layer, stream_handle(stream), ctypes.byref(out)))
    return out.value


def hv_render_launches(layer, index_kind=HV_INDEX_RTREE):
    out = U32()
    _check(lib().hv_render_launches(layer, index_kind, ctypes.byref(out)))
    return out.value


def hv_server_start(ctx, layers, opts):
    arr = (P * len(layers))(*layers)
    out = P()
    _check(lib().hv_server_start(ctx, arr, len(layers), ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def hv_server_submit(srv, req, tag):
    """Returns the raw status (HV_OK or HV_EBUSY); raises on other errors."""
    rc = lib().hv_server_submit(srv, ptr(req), tag)
    if rc not in (HV_OK, HV_EBUSY):
        _check(rc)
    return rc


def hv_server_poll(srv, buf):
    n = U32()
    _check(lib().hv_server_poll(srv, buf, len(buf), ctypes.byref(n)))
    return n.value


def hv_server_stop(srv):
    _check(lib().hv_server_stop(srv))


def hv_server_replay(srv, reqs, arrival_us):
    """Open-loop replay; returns (latency_us array, wall_us)."""
    arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
    lat = np.zeros(len(reqs), dtype=np.float64)
    wall = ctypes.c_double()
    _check(lib().hv_server_replay(srv, ptr(reqs), ptr(arr), len(reqs), ptr(lat), ctypes.byref(wall)))
    return lat, wall.value


def hv_server_replay_detail(srv, reqs, arrival_us):
    """Open-loop replay; returns (latency_us, parts_us (n, 4): pre-submit wait,
    task-pool wait, service, hand-out), wall_us)."""
    arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
    lat = np.zeros(len(reqs), dtype=np.float64)
    parts = np.zeros((len(reqs), 4), dtype=np.float64)
    wall = ctypes.c_double()
    _check(lib().hv_server_replay_detail(srv, ptr(reqs), ptr(arr), len(reqs), ptr(lat), ptr(parts),
                                         ctypes.byref(wall)))
    return lat, parts, wall.value


def hv_server_stats(srv):
    b, t, g, s = U64(), U64(), U64(), U32()
    _check(lib().hv_server_stats(srv, ctypes.byref(b), ctypes.byref(t), ctypes.byref(g), ctypes.byref(s)))
    return {"batches": b.value, "tiles": t.value, "graph_launches": g.value, "slots": s.value}


def hv_server_shortcuts(srv):
    h, e = U64(), U64()
    _check(lib().hv_server_shortcuts(srv, ctypes.byref(h), ctypes.byref(e)))
    return {"pool_hits": h.value, "empty_tiles": e.value}


def make_server_opts(max_batch=64, queue_capacity=0, scratch_bytes=0, index_kind=HV_INDEX_RTREE,
                     use_graphs=1, style=None, pool=None):
    o = hv_server_opts()
    o.max_batch, o.queue_capacity, o.scratch_bytes = max_batch, queue_capacity, scratch_bytes
    o.index_kind, o.use_graphs = index_kind, use_graphs
    if style is not None:
        o.style = style
    o.pool = pool
    return o


# ---- result pool ---------------------------------------------------------------

def hv_result_pool_create(capacity_bytes, ttl_ms=0):
    out = P()
    _check(lib().hv_result_pool_create(capacity_bytes, ttl_ms, ctypes.byref(out)))
    return out.value


def hv_result_pool_destroy(pool):
    _check(lib().hv_result_pool_destroy(pool))


def hv_result_pool_put(pool, req, style, data, nbytes=None):
    """req: one hv_tile_req record (numpy REQ_DTYPE); data: host bytes."""
    n = data.nbytes if nbytes is None else nbytes
    _check(lib().hv_result_pool_put(pool, ptr(req), ctypes.byref(style) if style is not None else None,
                                    ptr(data), n))


def hv_result_pool_get(pool, req, style, out):
    """Returns True on a hit (the tile is copied into `out`)."""
    hit = U32()
    _check(lib().hv_result_pool_get(pool, ptr(req), ctypes.byref(style) if style is not None else None,
                                    ptr(out), out.nbytes, ctypes.byref(hit)))
    return bool(hit.value)


def hv_result_pool_stats(pool):
    st = hv_pool_stats()
    _check(lib().hv_result_pool_stats(pool, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in st._fields_}


def hv_result_pool_clear(pool):
    _check(lib().hv_result_pool_clear(pool))


# ---- convenience: render host arrays into a numpy result --------------------

def render(layer, zxyr, mode, style=None, index_kind=HV_INDEX_RTREE):
    """Render tiles with host requests into a host array (n, tile_bytes)."""
    reqs = make_requests(zxyr)
    n = reqs.shape[0]
    tb = hv_tile_bytes(mode)
    out = np.zeros((max(n, 1), tb), dtype=np.uint8)
    hv_render_tiles(layer, reqs, n, mode, index_kind, style, out, n * tb)
    return out[:n]
