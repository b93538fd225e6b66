"""Served tiles of the full-size serving workload against the oracle.

The serving workload (HiVision Exp. 3 shape, Sec. 5.3, served through the
MTVS / IMMF / HPVE pipeline of Sec. 4): resident layers of 1B clustered points
and 200M random-walk segments, a pan/zoom request trace (Zipf start tiles,
zoom 2-18, layer 50/50) with the radius fixed at one of four values per
request, served by the server with continuous batching, once through the
learned index (captured graphs) and once through the R-tree.  2,000 sampled
responses of each run are compared with the oracle byte for byte.

A tile of a billion-object layer at low zoom holds up to 10^8 objects, more
than the oracle can splat in a test; such a response is checked on a window
of its pixels instead (the whole tile whenever the objects that can reach it
number at most a few million, else the largest aligned square window of 256,
64, 16, 4 or 1 pixels that does).  The oracle is given every object whose box
meets the window's box widened by R plus a pixel, which contains every
object within R of any of the window's samples, so its values there are its
values over the whole layer.
"""
import time

import numpy as np
import pytest

import oracle
from cellgrid import PointGrid, SegmentGrid, segments_of_lines
from oracle_par import map_threads
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE = ((230, 40, 20), (30, 90, 200))
STYLE_T = STYLE[0] + (0,) + STYLE[1] + (0,)
R16_FIXED = (16, 24, 32, 48)
N_REQ = 20_000
N_SAMPLE = 2_000
CAP = 3_000_000          # objects handed to one oracle call


def serve(ctx, layers, reqs, index, graphs, keep):
    """Serve every request (all submitted as fast as the queue allows) and
    return the tile bytes of the tags in `keep`."""
    opts = hv.make_server_opts(max_batch=64, queue_capacity=1 << 16, scratch_bytes=2 << 30,
                               index_kind=index, use_graphs=graphs, style=hv.make_style(*STYLE))
    srv = hv.hv_server_start(ctx, layers, opts)
    got = {}
    buf = (hv.hv_done * 512)()
    try:
        nxt, done = 0, 0
        t0 = time.time()
        while done < len(reqs):
            while nxt < len(reqs) and hv.hv_server_submit(srv, reqs[nxt:nxt + 1], nxt) == hv.HV_OK:
                nxt += 1
            n = hv.hv_server_poll(srv, buf)
            for i in range(n):
                d = buf[i]
                assert d.status == hv.HV_OK, d.status
                if d.tag in keep:
                    got[d.tag] = np.ctypeslib.as_array((hv.ctypes.c_uint8 * d.bytes).from_address(d.data)).copy()
            done += n
            if not n:
                time.sleep(0.0002)
            assert time.time() - t0 < 600, "server did not finish"
        stats = hv.hv_server_stats(srv)
        short = hv.hv_server_shortcuts(srv)
    finally:
        hv.hv_server_stop(srv)
    # tiles no object reaches complete at submission, without a launch
    assert stats["tiles"] + short["empty_tiles"] == len(reqs) and stats["batches"] < len(reqs)
    return got


def window_of(req, grid, rng):
    """The window (i0, j0, w) of a response to check, the box in grid units
    of the objects that can reach it, and those objects: the largest aligned
    window of w in (256, 64, 16, 4, 1) pixels, placed at random, whose box
    holds at most CAP objects."""
    z, tx, ty, r16 = (int(v) for v in req)
    ps = 1 << (23 - z)
    R = r16 << (19 - z)
    X0 = -(1 << 30) + (tx << (31 - z))
    Y0 = -(1 << 30) + (ty << (31 - z))
    for w in (256, 64, 16, 4, 1):
        i0 = int(rng.integers(0, 256 // w)) * w
        j0 = int(rng.integers(0, 256 // w)) * w
        # samples lie inside the pixels; an object within R of one lies in
        # this box (one pixel of slack on each side)
        box = (X0 + i0 * ps - R - ps, Y0 + j0 * ps - R - ps, X0 + (i0 + w) * ps + R + ps,
               Y0 + (j0 + w) * ps + R + ps)
        # the cell counts bound the population from above; count exactly
        # when the bound is close
        if grid.upper_count(*box) <= 20 * CAP or w == 1:
            sub = grid.query(*box)
            if len(sub) <= CAP or w == 1:
                return (i0, j0, w), sub


def test_served_trace_full_size_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    t0 = time.time()
    pts = gen.gmm_points(1_000_000_000, seed=5, k=64)
    xy, off = gen.walk_lines(20_000_000, 200_000_000, seed=55)
    ctx = hv.hv_create(0)
    try:
        layers = [hv.hv_layer_load_points(ctx, pts), hv.hv_layer_load_linestrings(ctx, xy, off)]
        for L in layers:
            hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
        anchors = [pts[::500], gen.segment_midpoints(xy, off, 2_000_000, seed=56)]
        tr = gen.pan_zoom_trace(anchors, N_REQ, seed=700)
        rng = np.random.default_rng(701)
        reqs = np.zeros(N_REQ, dtype=hv.REQ_DTYPE)
        reqs["z"], reqs["x"], reqs["y"], reqs["layer"] = tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 4]
        reqs["r16"] = np.asarray(R16_FIXED)[rng.integers(0, len(R16_FIXED), N_REQ)]
        reqs["mode"] = hv.HV_MODE_RGBA
        keep = set(rng.choice(N_REQ, N_SAMPLE, replace=False).tolist())
        served = {"learned": serve(ctx, layers, reqs, hv.HV_INDEX_LEARNED, 1, keep),
                  "rtree": serve(ctx, layers, reqs, hv.HV_INDEX_RTREE, 0, keep)}
        for L in layers:
            hv.hv_layer_free(L)
    finally:
        hv.hv_destroy(ctx)
    t_serve = time.time() - t0
    grids = [PointGrid(pts), SegmentGrid(segments_of_lines(xy, off))]
    del pts, xy, off
    tags = sorted(keep)

    def check(t):
        r = reqs[t]
        layer = int(r["layer"])
        req = np.array([[r["z"], r["x"], r["y"], r["r16"]]], dtype=np.uint32)
        (i0, j0, w), sub = window_of(req[0], grids[layer], np.random.default_rng(702 + t))
        if layer == 0:
            ref = oracle.render_points(sub, req, hv.HV_MODE_RGBA, STYLE_T)[0]
        else:
            off2 = np.arange(0, 2 * len(sub) + 1, 2, dtype=np.uint64)
            ref = oracle.render_lines(sub.reshape(-1, 2), off2, req, hv.HV_MODE_RGBA, STYLE_T)[0]
        ref = ref.reshape(256, 256, 4)[j0:j0 + w, i0:i0 + w]
        bad = [k for k, got in served.items()
               if not np.array_equal(got[t].reshape(256, 256, 4)[j0:j0 + w, i0:i0 + w], ref)]
        return t, w, len(sub), bad

    res = map_threads(check, tags)
    t_all = time.time() - t0
    widths = np.array([w for _, w, _, _ in res])
    bad = [(t, b) for t, _, _, b in res if b]
    print("config-5 check: %d responses x 2 indexes, full tiles %d, windows %s, objects per call max %d, "
          "serve %.0f s, total %.0f s" % (len(res), int((widths == 256).sum()),
                                          {int(w): int((widths == w).sum()) for w in (64, 16, 4, 1)},
                                          max(n for _, _, n, _ in res), t_serve, t_all))
    assert len(res) == N_SAMPLE
    assert set(int(reqs[t]["r16"]) for t in tags) == set(R16_FIXED)
    assert not bad, "served tiles differ from the oracle: %s" % bad[:10]
