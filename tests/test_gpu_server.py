"""Serving loop: continuous batching must not change any pixel.

Every tile served in a mix of layers, zooms, radii and modes, with many
requests in flight, must equal the oracle's tile for the same request, the
same request served alone, and the same tile rendered by hv_render_tiles
(HiVision Sec. 4: tasks are independent; the MTVS / IMMF / HPVE pipeline only
schedules them).
"""
import time

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE = ((230, 40, 20), (30, 90, 200))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


@pytest.fixture(scope="module")
def layers(ctx):
    pts = gen.gmm_points(400_000, seed=51, k=16)
    xy, off = gen.walk_lines(20_000, 150_000, seed=52, n_cities=30)
    pxy, ro, po = gen.star_polygons(5_000, seed=53, k=16, rho_median=6e-4)
    Ls = [hv.hv_layer_load_points(ctx, pts), hv.hv_layer_load_linestrings(ctx, xy, off),
          hv.hv_layer_load_polygons(ctx, pxy, ro, po)]
    for L in Ls:
        hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    anchors = [pts, gen.segment_midpoints(xy, off, 2000), gen.polygon_centres(pxy, ro, po)]
    src = [("points", pts), ("lines", xy, off), ("polygons", pxy, ro, po)]
    yield Ls, anchors, src
    for L in Ls:
        hv.hv_layer_free(L)


def mixed_requests(anchors, n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for k in range(n):
        layer = int(rng.integers(0, 3))
        z = int(rng.integers(2, 16))
        a = anchors[layer][int(rng.integers(0, len(anchors[layer])))].astype(np.int64)
        x, y = (a + (1 << 30)) >> (31 - z)
        rows.append((x, y, int(rng.integers(8, 49)), z, int(rng.integers(0, 3)), layer))
    r = np.zeros(n, dtype=hv.REQ_DTYPE)
    r["x"], r["y"], r["r16"], r["z"], r["mode"], r["layer"] = zip(*rows)
    return r


def poll_all(srv, want, timeout=120.0):
    buf = (hv.hv_done * 256)()
    got = {}
    t0 = time.time()
    while len(got) < want:
        n = hv.hv_server_poll(srv, buf)
        for i in range(n):
            d = buf[i]
            assert d.status == hv.HV_OK, d.status
            got[d.tag] = bytes(np.ctypeslib.as_array((hv.ctypes.c_uint8 * d.bytes).from_address(d.data)))
        if not n:
            time.sleep(0.0002)
        assert time.time() - t0 < timeout, "server did not finish"
    return got


def oracle_tiles(src, reqs):
    """The oracle's tile for every request, one oracle call per (layer, mode)."""
    out = {}
    zxyr = np.stack([reqs["z"], reqs["x"], reqs["y"], reqs["r16"]], 1).astype(np.uint32)
    for layer in np.unique(reqs["layer"]):
        for mode in np.unique(reqs["mode"]):
            idx = np.nonzero((reqs["layer"] == layer) & (reqs["mode"] == mode))[0]
            if not idx.size:
                continue
            s = src[int(layer)]
            st = STYLE[0] + (0,) + STYLE[1] + (0,)
            if s[0] == "points":
                ref = oracle.render_points(s[1], zxyr[idx], int(mode), st)
            elif s[0] == "lines":
                ref = oracle.render_lines(s[1], s[2], zxyr[idx], int(mode), st)
            else:
                ref = oracle.render_polygons(s[1], s[2], s[3], zxyr[idx], int(mode), st)
            for k, i in enumerate(idx):
                out[int(i)] = ref[k].tobytes()
    return out


def direct(Ls, reqs, style):
    out = {}
    for i, r in enumerate(reqs):
        one = hv.make_requests([[int(r["z"]), int(r["x"]), int(r["y"]), int(r["r16"])]])
        tb = hv.hv_tile_bytes(int(r["mode"]))
        buf = np.zeros((1, tb), dtype=np.uint8)
        hv.hv_render_tiles(Ls[int(r["layer"])], one, 1, int(r["mode"]), hv.HV_INDEX_RTREE, style, buf, tb)
        out[i] = buf.tobytes()
    return out


@pytest.mark.parametrize("graphs,index", [(1, hv.HV_INDEX_RTREE), (0, hv.HV_INDEX_RTREE), (1, hv.HV_INDEX_LEARNED)])
def test_alone_equals_mix(ctx, layers, graphs, index):
    Ls, anchors, src = layers
    style = hv.make_style(*STYLE)
    reqs = mixed_requests(anchors, 240, seed=54 + graphs + index)
    opts = hv.make_server_opts(max_batch=16, scratch_bytes=16 * 262144 * 6, index_kind=index,
                               use_graphs=graphs, style=style)
    srv = hv.hv_server_start(ctx, Ls, opts)
    try:
        alone = {}
        for i in range(0, len(reqs), 8):                 # one request at a time
            assert hv.hv_server_submit(srv, reqs[i:i + 1], i) == hv.HV_OK
            alone.update(poll_all(srv, 1))
        for i in range(len(reqs)):                       # everything in flight at once
            while hv.hv_server_submit(srv, reqs[i:i + 1], 1000 + i) == hv.HV_EBUSY:
                time.sleep(0.0001)
        mix = poll_all(srv, len(reqs))
        stats = hv.hv_server_stats(srv)
    finally:
        hv.hv_server_stop(srv)
    ref = oracle_tiles(src, reqs)
    rendered = direct(Ls, reqs, style)
    for i in range(0, len(reqs), 8):
        assert alone[i] == ref[i], "alone %d" % i
    for i in range(len(reqs)):
        assert mix[1000 + i] == ref[i], "mix %d differs from the oracle" % i
        assert rendered[i] == ref[i], "hv_render_tiles %d" % i
    assert stats["batches"] < stats["tiles"]             # requests were batched
    if graphs:
        assert stats["graph_launches"] == stats["batches"]


def test_submit_errors_and_back_pressure(ctx, layers):
    Ls, anchors, _ = layers
    opts = hv.make_server_opts(max_batch=1, queue_capacity=4, scratch_bytes=262144 + 64)
    srv = hv.hv_server_start(ctx, Ls[:1], opts)
    try:
        bad = mixed_requests(anchors, 1, 5)
        bad["layer"] = 0
        bad["z"] = 20
        with pytest.raises(hv.HVError) as e:
            hv.hv_server_submit(srv, bad, 0)
        assert e.value.status == hv.HV_ERANGE
        bad["z"], bad["x"], bad["y"], bad["layer"] = 3, 0, 0, 7
        with pytest.raises(hv.HVError) as e:
            hv.hv_server_submit(srv, bad, 0)
        assert e.value.status == hv.HV_EINVAL
        ok = np.zeros(1, dtype=hv.REQ_DTYPE)
        ok["z"], ok["x"], ok["y"], ok["r16"], ok["mode"] = 9, 300, 200, 1024, hv.HV_MODE_RGBA
        codes = [hv.hv_server_submit(srv, ok, k) for k in range(2000)]
        assert hv.HV_EBUSY in codes
        accepted = codes.count(hv.HV_OK)
        assert len(poll_all(srv, accepted)) == accepted
        assert hv.hv_server_stats(srv)["slots"] == 1
    finally:
        hv.hv_server_stop(srv)


def test_open_loop_replay(ctx, layers):
    Ls, anchors, _ = layers
    reqs = mixed_requests(anchors, 3000, seed=60)
    reqs["mode"] = hv.HV_MODE_RGBA
    arrival = np.cumsum(np.random.default_rng(61).exponential(1e6 / 20000.0, size=len(reqs)))
    srv = hv.hv_server_start(ctx, Ls, hv.make_server_opts(max_batch=32, scratch_bytes=1 << 30))
    try:
        lat, parts, wall = hv.hv_server_replay_detail(srv, reqs, arrival)
        stats = hv.hv_server_stats(srv)
        short = hv.hv_server_shortcuts(srv)
    finally:
        hv.hv_server_stop(srv)
    assert (lat > 0).all() and np.isfinite(lat).all()
    assert wall >= arrival[-1]
    # the first three parts of each latency add up to it (clock reads apart);
    # the fourth is the time until the replay polled the result
    assert (parts >= -1.0).all() and np.allclose(parts[:, :3].sum(1), lat, atol=5.0)
    # tiles no object reaches complete at submission, without a launch
    assert stats["tiles"] + short["empty_tiles"] == len(reqs)
    assert stats["batches"] <= len(reqs)


def test_result_pool_and_unreachable_tiles(ctx, layers):
    """Parse Tasks (Sec. 4.1) drops tiles already in the Result Pool (Sec. 4.2)
    and tiles outside the data: requests served a second time come from the
    pool, under a capacity that forces evictions, and tiles no object can
    reach complete at submission as zeros; every tile equals the oracle's."""
    Ls, anchors, src = layers
    style = hv.make_style(*STYLE)
    reqs = mixed_requests(anchors, 90, seed=91)
    # room for about half of the tiles: the first round evicts, and the
    # second, submitted at once, finds the later half
    total = sum(hv.hv_tile_bytes(int(m)) for m in reqs["mode"])
    pool = hv.hv_result_pool_create(total // 2)
    srv = hv.hv_server_start(ctx, Ls, hv.make_server_opts(max_batch=8, scratch_bytes=8 * 262144 * 4,
                                                          style=style, pool=pool))
    try:
        ref = oracle_tiles(src, reqs)
        for rnd in range(2):
            for i in range(len(reqs)):
                assert hv.hv_server_submit(srv, reqs[i:i + 1], 100 * rnd + i) == hv.HV_OK
            got = poll_all(srv, len(reqs))
            for i in range(len(reqs)):
                assert got[100 * rnd + i] == ref[i], "round %d request %d" % (rnd, i)
        sc = hv.hv_server_shortcuts(srv)
        st = hv.hv_result_pool_stats(pool)
        assert sc["pool_hits"] > 0 and st["hits"] == sc["pool_hits"]
        assert st["inserts"] >= len(reqs) and st["evictions"] > 0 and st["bytes"] <= st["capacity"]
        # tiles of the polygon layer far from all of its polygons
        far = np.zeros(6, dtype=hv.REQ_DTYPE)
        far["z"], far["x"], far["y"] = 19, [0, 1, 5, (1 << 19) - 1, 0, 7], [0, 0, 9, (1 << 19) - 1, 3, 0]
        far["r16"], far["layer"], far["mode"] = 48, 2, [0, 1, 2, 2, 1, 0]
        before = sc["empty_tiles"]
        launched = hv.hv_server_stats(srv)["tiles"]
        for i in range(len(far)):
            assert hv.hv_server_submit(srv, far[i:i + 1], 1000 + i) == hv.HV_OK
        got = poll_all(srv, len(far))
        fref = oracle_tiles(src, far)
        for i in range(len(far)):
            assert got[1000 + i] == fref[i] and not any(got[1000 + i])
        assert hv.hv_server_shortcuts(srv)["empty_tiles"] == before + len(far)
        assert hv.hv_server_stats(srv)["tiles"] == launched          # no GPU work for them
    finally:
        hv.hv_server_stop(srv)
        hv.hv_result_pool_destroy(pool)
