"""Learned candidate lookup: exact positions and byte-equal tiles.

The learned model predicts an object's position in the Hilbert-sorted order
from its key; lookups confirm the bracket keys[p-1] < k <= keys[p] and fall
back to a full search outside the stored error window, so every answer is the
lower bound itself.  Tiles rendered through it equal the R-tree's and the
oracle's (HiVision Algorithms 1 and 2 are unchanged by how candidates are
found).
"""
import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE_T = (230, 40, 20, 0, 30, 90, 200, 0)
MODES = [hv.HV_MODE_MASK, hv.HV_MODE_COVERAGE, hv.HV_MODE_RGBA]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


def style():
    return hv.make_style(STYLE_T[:3], STYLE_T[4:7])


def render_dev(layer, reqs, mode, index):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((max(n, 1), hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    hv.hv_render_tiles(layer, d_req, n, mode, index, style(), out, out.numel(), s)
    s.synchronize()
    return out[:n].cpu().numpy()


def keys_of(layer, which, n):
    k = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    hv.hv_layer_keys(layer, which, k, n)
    return k[:n]


def lookup(layer, which, q):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    out = torch.empty(max(len(q), 1), dtype=torch.int64, device="cuda")
    fb = hv.hv_learned_lookup(layer, which, dq, len(q), out)
    return out[:len(q)].cpu().numpy().astype(np.uint64), fb


def check_lookups(layer, which, n, seed):
    keys = keys_of(layer, which, n).cpu().numpy().view(np.uint64)
    assert np.all(keys[1:] >= keys[:-1])
    rng = np.random.default_rng(seed)
    q = np.concatenate([
        rng.integers(0, 1 << 62, size=100_000, dtype=np.uint64),
        keys[rng.integers(0, n, size=50_000)],
        keys[rng.integers(0, n, size=20_000)] + np.uint64(1),
        keys[rng.integers(0, n, size=20_000)] - np.uint64(1),
        np.array([0, 1, keys[0], keys[-1], keys[-1] + np.uint64(1), (1 << 62) - 1, 1 << 62], dtype=np.uint64)])
    got, _ = lookup(layer, which, q)
    assert np.array_equal(got, np.searchsorted(keys, q, side="left"))
    # every stored key lies inside the model's error window: no fallback
    got, fb = lookup(layer, which, keys)
    assert np.array_equal(got, np.searchsorted(keys, keys, side="left"))
    assert fb == 0


def test_lookup_is_lower_bound_points(ctx):
    pts = gen.gmm_points(2_000_000, seed=31, k=32)
    pts = np.concatenate([pts, np.repeat(pts[:1000], 50, axis=0)])   # long runs of equal keys
    L = hv.hv_layer_load_points(ctx, pts)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        info = hv.info_dict(L)
        assert info["indexes"] == 3 and info["learned_error"] >= 0 and info["learned_pieces"] > 0
        # a piece keeps the MLP term only where it narrows its own bound
        assert info["learned_error"] <= info["learned_error_linear"]
        assert info["learned_mean_window"] <= info["learned_mean_window_linear"] + 1e-9
        check_lookups(L, 0, len(pts), 1)
    finally:
        hv.hv_layer_free(L)


def test_lookup_is_lower_bound_polygon_boxes(ctx):
    xy, ro, po = gen.star_polygons(50_000, seed=32, k=16, rho_median=5e-4)
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        info = hv.info_dict(L)
        assert info["n_objects"] == int(ro[-1]) and info["index_records"] >= info["n_objects"]
        check_lookups(L, 0, info["index_records"], 2)
        check_lookups(L, 1, len(po) - 1, 3)
    finally:
        hv.hv_layer_free(L)


@pytest.mark.parametrize("mlp", [True, False])
def test_learned_points_tiles(ctx, mlp):
    pts = gen.gmm_points(300_000, seed=33, k=16)
    reqs = gen.density_tiles(pts, 150, 0, 19, [1, 8, 32, 100, 600], seed=34)
    L = hv.hv_layer_load_points(ctx, pts)
    opts = hv.hv_build_opts()
    if mlp:
        opts.learned_steps = 200
    else:
        opts.learned_hidden = hv.HV_LEARNED_NO_MLP
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED, opts)
    try:
        info = hv.info_dict(L)
        if not mlp:
            assert info["learned_mlp"] == 0 and info["learned_error"] == info["learned_error_linear"]
        for mode in MODES:
            a = render_dev(L, reqs, mode, hv.HV_INDEX_LEARNED)
            b = render_dev(L, reqs, mode, hv.HV_INDEX_RTREE)
            assert np.array_equal(a, b)
            assert np.array_equal(a, oracle.render_points(pts, reqs, mode, STYLE_T))
    finally:
        hv.hv_layer_free(L)


def test_learned_lines_tiles(ctx):
    xy, off = gen.walk_lines(20_000, 120_000, seed=35, n_cities=30)
    # a few very long segments, which the halo does not cover (side tree)
    extra = np.array([[-(1 << 29), 0], [1 << 29, 1000], [5, -(1 << 28)], [7, 1 << 28]], dtype=np.int32)
    xy = np.concatenate([xy, extra])
    off = np.concatenate([off, [off[-1] + 2, off[-1] + 4]]).astype(np.uint64)
    mids = gen.segment_midpoints(xy, off, 3000, seed=36)
    reqs = np.concatenate([gen.density_tiles(mids, 100, 3, 17, [1, 8, 16, 40], seed=37),
                           [[12, 2048, 2048, 16], [14, 8192, 8200, 16], [10, 900, 512, 24]]]).astype(np.uint32)
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        info = hv.info_dict(L)
        # long segments are indexed as several bounded pieces
        assert info["piece_extent"] > 0 and info["index_records"] > info["n_objects"]
        for mode in MODES:
            a = render_dev(L, reqs, mode, hv.HV_INDEX_LEARNED)
            b = render_dev(L, reqs, mode, hv.HV_INDEX_RTREE)
            assert np.array_equal(a, b)
            assert np.array_equal(a, oracle.render_lines(xy, off, reqs, mode, STYLE_T))
    finally:
        hv.hv_layer_free(L)


def test_learned_polygon_tiles(ctx):
    xy, ro, po = gen.star_polygons(6_000, seed=38, k=16, rho_median=6e-4)
    cen = gen.polygon_centres(xy, ro, po)
    reqs = gen.density_tiles(cen, 50, 2, 10, [1, 8, 24], seed=39)
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for mode in MODES:
            a = render_dev(L, reqs, mode, hv.HV_INDEX_LEARNED)
            b = render_dev(L, reqs, mode, hv.HV_INDEX_RTREE)
            assert np.array_equal(a, b)
            assert np.array_equal(a, oracle.render_polygons(xy, ro, po, reqs, mode, STYLE_T))
    finally:
        hv.hv_layer_free(L)


def test_learned_polygon_outliers(ctx):
    """A few very large polygons among small ones: their boxes exceed the
    learned halo and live in the side tree, so strips deep inside them have
    an empty learned frontier in both stages and are filled through the side
    tree alone."""
    xy, ro, po = gen.star_polygons(3_000, seed=73, k=8, rho_median=6e-4)
    cen = gen.polygon_centres(xy, ro, po)[:12].astype(np.int64)
    h = 1 << 25
    sq = np.stack([np.stack([cen[:, 0] - h, cen[:, 1] - h], 1), np.stack([cen[:, 0] + h, cen[:, 1] - h], 1),
                   np.stack([cen[:, 0] + h, cen[:, 1] + h], 1), np.stack([cen[:, 0] - h, cen[:, 1] + h], 1)], 1)
    sq = np.clip(sq, -(1 << 30), (1 << 30) - 1).reshape(-1, 2).astype(np.int32)
    xy2 = np.concatenate([xy, sq])
    ro2 = np.concatenate([ro, ro[-1] + 4 * np.arange(1, 13, dtype=np.uint64)]).astype(np.uint64)
    po2 = np.concatenate([po, po[-1] + np.arange(1, 13, dtype=np.uint64)]).astype(np.uint64)
    # tiles inside the large squares, far from any of their edges, and tiles
    # over the small polygons
    reqs = np.concatenate([gen.density_tiles(cen + 12345, 12, 11, 14, [1, 8, 24], seed=75),
                           gen.density_tiles(gen.polygon_centres(xy, ro, po), 8, 3, 12, [8, 24], seed=76)])
    L = hv.hv_layer_load_polygons(ctx, xy2, ro2, po2)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        assert hv.info_dict(L)["learned_outliers"] > 0
        want = {mode: oracle.render_polygons(xy2, ro2, po2, reqs, mode, STYLE_T) for mode in MODES}
        for mode in MODES:
            for index in (hv.HV_INDEX_LEARNED, hv.HV_INDEX_RTREE):
                got = render_dev(L, reqs, mode, index)
                assert hv.hv_layer_take_status(L) == 0
                assert np.array_equal(got, want[mode])
    finally:
        hv.hv_layer_free(L)


def test_error_bound_gate(ctx):
    pts = gen.gmm_points(200_000, seed=40, k=8)
    L = hv.hv_layer_load_points(ctx, pts)
    opts = hv.hv_build_opts()
    opts.max_error = 1
    opts.learned_steps = 0
    opts.learned_segments = 16     # coarse pieces: a large error bound
    try:
        with pytest.raises(hv.HVError) as e:
            hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED, opts)
        assert e.value.status == hv.HV_ESTATE
        assert hv.info_dict(L)["indexes"] == hv.HV_INDEX_RTREE
        out = np.zeros((1, 8192), dtype=np.uint8)
        with pytest.raises(hv.HVError) as e:
            hv.hv_render_tiles(L, hv.make_requests([[3, 1, 1, 16]]), 1, hv.HV_MODE_MASK, hv.HV_INDEX_LEARNED,
                               None, out, out.nbytes)
        assert e.value.status == hv.HV_ESTATE
    finally:
        hv.hv_layer_free(L)


def test_empty_layer_learned(ctx):
    L = hv.hv_layer_load_points(ctx, np.zeros((0, 2), np.int32))
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        got = render_dev(L, np.array([[0, 0, 0, 16], [5, 3, 3, 40]], np.uint32), hv.HV_MODE_RGBA,
                         hv.HV_INDEX_LEARNED)
        assert not got.any()
    finally:
        hv.hv_layer_free(L)
