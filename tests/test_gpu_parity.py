"""GPU parity: CUDA tiles through the C ABI vs the CPU oracle, byte for byte.

Results are exact integer decisions, so the tolerance is zero everywhere
(HiVision Algorithm 1 and Algorithm 2 on the integer grid).
"""
import numpy as np
import pytest

import oracle
import oracle_par
from geom import (at, lines_to_arrays, polys_to_arrays, random_cluster_points,
                  random_star_polygons, random_walk_lines, ring_px)
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


@pytest.fixture(scope="module")
def lines50m(ctx):
    """The full-size linestring layer with both indexes, shared by its tests."""
    xy, off, reqs = gen.config3()
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    yield xy, off, reqs, L
    hv.hv_layer_free(L)


def style():
    return hv.make_style(STYLE_T[:3], STYLE_T[4:7])


def render_dev(layer, reqs, mode, index=hv.HV_INDEX_RTREE):
    """Device requests and device output (the benchmark's launch form)."""
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((max(n, 1), hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    hv.hv_render_tiles(layer, d_req, n, mode, index, style(), out, out.numel(), s)
    s.synchronize()
    return out[:n].cpu().numpy()


def points_layer(ctx, pts):
    L = hv.hv_layer_load_points(ctx, pts)
    hv.hv_layer_build_index(L)
    return L


def check_points(ctx, pts, reqs, modes=MODES):
    L = points_layer(ctx, pts)
    try:
        for mode in modes:
            got = render_dev(L, reqs, mode)
            ref = oracle.render_points(pts, reqs, mode, STYLE_T)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
    finally:
        hv.hv_layer_free(L)


def check_lines(ctx, xy, off, reqs, modes=MODES):
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L)
    try:
        for mode in modes:
            got = render_dev(L, reqs, mode)
            ref = oracle.render_lines(xy, off, reqs, mode, STYLE_T)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
    finally:
        hv.hv_layer_free(L)


def check_polygons(ctx, xy, ro, po, reqs, modes=MODES):
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L)
    try:
        for mode in modes:
            got = render_dev(L, reqs, mode)
            ref = oracle.render_polygons(xy, ro, po, reqs, mode, STYLE_T)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
    finally:
        hv.hv_layer_free(L)


# ---- the small workload: 100,000 uniform points, all 341 tiles of z 0-4 ----

def test_uniform_points_all_tiles_zoom_0_to_4(ctx):
    pts, reqs = gen.config1()
    check_points(ctx, pts, reqs)


# ---- random layers across zooms, radii and modes ---------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_clustered_points(ctx, seed):
    pts = gen.gmm_points(60_000, seed=seed, k=16)
    r16 = [1, 7, 16, 32, 100, 300]
    reqs = gen.density_tiles(pts, 120, 0, 19, r16, seed=seed + 50)
    check_points(ctx, pts, reqs)


@pytest.mark.parametrize("seed", [1, 2])
def test_lines(ctx, seed):
    xy, off = gen.walk_lines(10_000, 60_000, seed=seed, n_cities=40)
    mids = gen.segment_midpoints(xy, off, 5000, seed=seed)
    reqs = gen.density_tiles(mids, 100, 2, 18, [1, 8, 16, 24, 64], seed=seed + 60)
    check_lines(ctx, xy, off, reqs)


@pytest.mark.parametrize("seed", [1, 2])
def test_polygons(ctx, seed):
    xy, ro, po = gen.star_polygons(8_000, seed=seed, k=16, rho_median=6e-4)
    cen = gen.polygon_centres(xy, ro, po)
    reqs = gen.density_tiles(cen, 60, 2, 10, [1, 8, 20, 48], seed=seed + 70)
    check_polygons(ctx, xy, ro, po, reqs)


def test_tiles_inside_large_polygons(ctx):
    """Rays that leave the tile: a few huge star polygons (with holes) seen at
    high zoom, where whole tiles lie inside or straddle their edges."""
    rng = np.random.default_rng(17)
    polys = random_star_polygons(rng, 6, 6, 20, 30, 60, 128, 128, 30, holes=True)
    xy, ro, po = polys_to_arrays(polys)
    cen = gen.polygon_centres(xy, ro, po)
    reqs = gen.density_tiles(cen, 24, 9, 15, [1, 8, 40], seed=18)
    reqs2 = gen.density_tiles(xy, 24, 9, 15, [8], seed=19)        # tiles on the outlines
    check_polygons(ctx, xy, ro, po, np.concatenate([reqs, reqs2]))


def test_polygons_with_holes_and_lattice_vertices(ctx):
    rng = np.random.default_rng(5)
    z, tx, ty = 13, 3000, 5000
    polys = random_star_polygons(rng, 60, z, tx, ty, 30, 128, 128, 60, holes=True, snap=True)
    polys += [[ring_px(z, tx, ty, 100, 100, [(0, -7), (7, 0), (0, 7), (-7, 0)])],
              [ring_px(z, tx, ty, 40, 40, [(0, 0), (8, 0), (8, 8), (0, 8), (-4, 4)])]]
    xy, ro, po = polys_to_arrays(polys)
    reqs = np.array([[z, tx, ty, r] for r in (1, 8, 16, 40)] +
                    [[z + 1, 2 * tx + 1, 2 * ty, 8], [z - 1, tx // 2, ty // 2, 8]], dtype=np.uint32)
    check_polygons(ctx, xy, ro, po, reqs)


def test_lines_with_degenerate_segments(ctx):
    rng = np.random.default_rng(8)
    z, tx, ty = 12, 1000, 2000
    lines = random_walk_lines(rng, 40, 8, z, tx, ty, 4, 128, 128, 50)
    lines += [[at(z, tx, ty, 20, 20)] * 3,                 # zero-length segments
              [at(z, tx, ty, 5, 5)],                        # a single vertex draws nothing
              [at(z, tx, ty, 10, 200), at(z, tx, ty, 250, 200)]]  # level segment
    xy, off = lines_to_arrays(lines)
    reqs = np.array([[z, tx, ty, r] for r in (1, 8, 16, 33, 200)], dtype=np.uint32)
    check_lines(ctx, xy, off, reqs)


# ---- edge cases -----------------------------------------------------------

def test_dense_duplicates_and_tile_borders(ctx):
    z, tx, ty = 10, 300, 517
    rng = np.random.default_rng(4)
    p = random_cluster_points(rng, 5000, z, tx, ty, 0.3, 255, 0)   # a tight cluster on a corner
    p = np.concatenate([p, p[:1000], np.array([at(z, tx, ty, 0, 0, -0.5, -0.5)], np.int32)])
    reqs = np.array([[z, tx + a, ty + b, r] for a in (-1, 0, 1) for b in (-1, 0, 1) for r in (3, 40)],
                    dtype=np.uint32)
    check_points(ctx, p, reqs)


def test_grid_extremes(ctx):
    half = 1 << 30
    p = np.array([[-half, -half], [half - 1, half - 1], [-half, half - 1], [half - 1, -half], [0, 0],
                  [-1, -1]], dtype=np.int32)
    reqs = [[0, 0, 0, 1024], [0, 0, 0, 1], [1, 0, 0, 77], [1, 1, 1, 77], [19, 0, 0, 1024],
            [19, (1 << 19) - 1, (1 << 19) - 1, 1024], [19, 1 << 18, 1 << 18, 16],
            [19, (1 << 18) - 1, (1 << 18) - 1, 16], [5, 15, 16, 300]]
    check_points(ctx, p, np.array(reqs, dtype=np.uint32))


def _tiles_along(segs, zooms, per_seg, rng, r16s):
    """Tiles that contain sampled points of the given segments (x0, y0, x1, y1)."""
    half = 1 << 30
    out = []
    for (x0, y0, x1, y1) in segs:
        for t in rng.uniform(0.0, 1.0, per_seg):
            x = int(x0 + (x1 - x0) * t)
            y = int(y0 + (y1 - y0) * t)
            z = int(rng.choice(zooms))
            out.append([z, (x + half) >> (31 - z), (y + half) >> (31 - z), int(rng.choice(r16s))])
    return np.array(out, dtype=np.uint32)


def test_grid_spanning_segments(ctx):
    """Segments across the whole grid seen at high zoom: endpoints far from
    every pixel block (the absolute 64-bit test), pieces far larger than the
    pixels (the band filter), slopes near 0, 1 and infinity."""
    half = 1 << 30
    segs = [(-half, -half, half - 1, half - 1), (-half, 12345, half - 1, 12346),
            (777, -half, 778, half - 1), (-half + 5, half - 9, half - 3, -half + 1),
            (-(1 << 29), 3, (1 << 29) + 17, 1 << 20), (100, 200, 100 + (1 << 27), 200 + (1 << 13))]
    xy = np.array([[a, b] for s in segs for a, b in ((s[0], s[1]), (s[2], s[3]))], dtype=np.int32)
    off = np.arange(0, 2 * len(segs) + 1, 2, dtype=np.uint64)
    rng = np.random.default_rng(21)
    reqs = np.concatenate([_tiles_along(segs, [0, 3, 9, 14, 17, 19], 6, rng, [1, 8, 16, 100]),
                           np.array([[0, 0, 0, 1024], [2, 1, 2, 64]], dtype=np.uint32)])
    check_lines(ctx, xy, off, reqs)


def test_grid_spanning_polygon_edges(ctx):
    """A polygon over most of the grid, a thin sliver and a square hole: the
    fill's per-row crossing counts with edges far from the block, at high zoom
    along the edges and inside."""
    half = 1 << 30
    big = [(-half, -half), (half - 1, -half + 7), (3, half - 1)]
    sliver = [(-half + 10, 5), (half - 10, 7), (half - 10, 9), (-half + 10, 6)]
    hole = [(-1000000, -1000000), (-1000000, 1000000), (1000000, 1000000), (1000000, -1000000)]
    xy = np.array(big + hole + sliver, dtype=np.int32)
    ro = np.array([0, 3, 7, 11], dtype=np.uint64)
    po = np.array([0, 2, 3], dtype=np.uint64)
    edges = [big[i] + big[(i + 1) % 3] for i in range(3)] + [sliver[i] + sliver[(i + 1) % 4] for i in range(4)]
    rng = np.random.default_rng(22)
    reqs = np.concatenate([_tiles_along(edges, [1, 6, 12, 16, 19], 4, rng, [1, 8, 40]),
                           np.array([[19, 1 << 18, 1 << 18, 8], [12, 2047, 2047, 8], [0, 0, 0, 16]],
                                    dtype=np.uint32)])
    check_polygons(ctx, xy, ro, po, reqs)


def test_empty_and_single_object_layers(ctx):
    reqs = np.array([[0, 0, 0, 16], [7, 64, 64, 40]], dtype=np.uint32)
    check_points(ctx, np.zeros((0, 2), np.int32), reqs)
    check_points(ctx, np.array([[5, -7]], np.int32), reqs)
    xy, off = lines_to_arrays([[(0, 0)]])
    check_lines(ctx, xy, off, reqs)
    xy, ro, po = polys_to_arrays([])
    check_polygons(ctx, np.zeros((0, 2), np.int32), np.array([0], np.uint64), np.array([0], np.uint64), reqs)


def test_many_tiles_ragged_count(ctx):
    pts = gen.gmm_points(300_000, seed=9, k=32)
    reqs = gen.density_tiles(pts, 1237, 4, 15, 24, seed=19)
    check_points(ctx, pts, reqs, modes=[hv.HV_MODE_COVERAGE])


def test_host_and_device_buffers_agree(ctx):
    pts = gen.gmm_points(50_000, seed=21, k=8)
    reqs = gen.density_tiles(pts, 40, 5, 12, 20, seed=22)
    L = points_layer(ctx, pts)
    try:
        a = hv.render(L, reqs, hv.HV_MODE_RGBA, style())          # host requests, host output
        b = render_dev(L, reqs, hv.HV_MODE_RGBA)
        assert np.array_equal(a, b)
        # host requests, device output
        out = torch.zeros((len(reqs), hv.hv_tile_bytes(hv.HV_MODE_RGBA)), dtype=torch.uint8, device="cuda")
        hv.hv_render_tiles(L, hv.make_requests(reqs), len(reqs), hv.HV_MODE_RGBA, hv.HV_INDEX_RTREE,
                           style(), out, out.numel(), None)
        assert np.array_equal(out.cpu().numpy(), a)
    finally:
        hv.hv_layer_free(L)


def test_errors(ctx):
    pts = gen.uniform_points(1000, seed=1)
    L = points_layer(ctx, pts)
    try:
        out = np.zeros((2, 8192), dtype=np.uint8)
        for bad in ([20, 0, 0, 16], [3, 8, 0, 16], [3, 0, 0, 0], [3, 0, 0, 1025]):
            with pytest.raises(hv.HVError) as e:
                hv.hv_render_tiles(L, hv.make_requests([bad]), 1, hv.HV_MODE_MASK, hv.HV_INDEX_RTREE,
                                   None, out, out.nbytes)
            assert e.value.status == hv.HV_ERANGE
        with pytest.raises(hv.HVError) as e:
            hv.hv_render_tiles(L, hv.make_requests([[1, 0, 0, 16]] * 2), 2, hv.HV_MODE_MASK,
                               hv.HV_INDEX_RTREE, None, out, 8192)
        assert e.value.status == hv.HV_EINVAL
        with pytest.raises(hv.HVError) as e:
            hv.hv_render_tiles(L, hv.make_requests([[1, 0, 0, 16]]), 1, 7, hv.HV_INDEX_RTREE, None, out,
                               out.nbytes)
        assert e.value.status == hv.HV_EINVAL
        # invalid device requests: zero tiles and a sticky status bit
        reqs = [[2, 1, 1, 16], [2, 9, 0, 16], [30, 0, 0, 16]]
        got = render_dev(L, np.array(reqs, dtype=np.int64), hv.HV_MODE_MASK)
        assert not got[1].any() and not got[2].any() and got[0].any()
        assert hv.hv_layer_take_status(L) == 1
        assert hv.hv_layer_take_status(L) == 0
    finally:
        hv.hv_layer_free(L)
    with pytest.raises(hv.HVError) as e:
        hv.hv_layer_load_points(ctx, np.array([[1 << 30, 0]], dtype=np.int64).astype(np.int32))
    assert e.value.status == hv.HV_ERANGE
    with pytest.raises(hv.HVError) as e:
        hv.hv_layer_load_linestrings(ctx, np.zeros((3, 2), np.int32), np.array([0, 2, 1, 3], np.uint64))
    assert e.value.status == hv.HV_EINVAL


def test_memory_budget(ctx):
    small = hv.hv_create(0, 1 << 20)
    try:
        with pytest.raises(hv.HVError) as e:
            hv.hv_layer_load_points(small, gen.uniform_points(200_000, seed=3))
        assert e.value.status == hv.HV_ENOMEM
        assert hv.hv_ctx_device_bytes(small) == 0
    finally:
        hv.hv_destroy(small)


# ---- full-size workload in the benchmark's launch form, sampled ---------

@pytest.mark.slow
def test_clustered_100m_points_sampled_tiles(ctx):
    """100M clustered points, 10,000 density-weighted tiles (zoom 8-14,
    radius 2 px, RGBA) rendered in one call; 72 tiles (16 densest, 4
    emptiest, an even spread) against the oracle, and the learned index
    against the R-tree on all tiles."""
    pts, reqs = gen.config2()
    L = hv.hv_layer_load_points(ctx, pts)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        n = _sampled_check(L, lambda r, m: oracle.render_points(pts, r, m, STYLE_T), reqs, 52, 16)
        assert n >= 64
    finally:
        hv.hv_layer_free(L)


def _sampled_check(L, render_ref, reqs, n_even, n_dense, n_empty=4, mode=hv.HV_MODE_RGBA):
    """All tiles in one call through the R-tree and the learned index: the two
    must agree on every tile, and a sample (the densest and emptiest tiles and
    an even spread) must equal the oracle, evaluated on the host's cores."""
    got = render_dev(L, reqs, mode)
    learned = render_dev(L, reqs, mode, hv.HV_INDEX_LEARNED)
    diff = np.nonzero((got != learned).any(axis=1))[0]
    assert diff.size == 0, "learned index differs from the R-tree on %d tiles, first %s" % (diff.size, diff[:8])
    lit = (got.reshape(len(reqs), -1, 4)[:, :, 3] > 0).sum(1) if mode == hv.HV_MODE_RGBA else got.sum(1)
    order = np.argsort(lit, kind="stable")
    pick = set(order[-n_dense:].tolist()) | set(order[:n_empty].tolist())
    pick |= set(np.linspace(0, len(reqs) - 1, n_even).astype(int).tolist())
    pick = np.array(sorted(pick))
    ref = oracle_par.render(lambda r: render_ref(r, mode), reqs[pick])
    bad = [int(pick[k]) for k in range(len(pick)) if not np.array_equal(got[pick[k]], ref[k])]
    assert not bad, "tiles differ: %s" % bad
    return len(pick)


@pytest.mark.slow
@pytest.mark.parametrize("r16", [8, 16, 24])
def test_linestrings_50m_segments_sampled_tiles(ctx, lines50m, r16):
    """50M segments in 5M random-walk lines, 10,000 density-weighted tiles
    (zoom 6-16) at half-width 0.5, 1 and 1.5 px, RGBA, in one call; 72 tiles
    (16 densest, 4 emptiest, an even spread) against the oracle, and the
    learned index against the R-tree on all tiles."""
    xy, off, reqs, L = lines50m
    reqs = reqs.copy()
    reqs[:, 3] = r16
    n = _sampled_check(L, lambda r, m: oracle.render_lines(xy, off, r, m, STYLE_T), reqs, 52, 16)
    assert n >= 64


@pytest.mark.slow
def test_polygons_2m_sampled_tiles(ctx):
    """2M star polygons (72M edges), 10,000 density-weighted tiles (zoom 4-14,
    fill + 1 px outline, RGBA) in one call; 72 tiles (16 densest, 4
    emptiest, an even spread) against the oracle, and the learned index
    against the R-tree on all tiles."""
    xy, ro, po, reqs = gen.config4()
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        n = _sampled_check(L, lambda r, m: oracle.render_polygons(xy, ro, po, r, m, STYLE_T), reqs, 52, 16)
        assert n >= 64
    finally:
        hv.hv_layer_free(L)


def test_host_output_in_chunks(ctx):
    """More tiles than one host-output chunk (1024): the double-buffered,
    overlapped copies must assemble exactly the device result."""
    pts = gen.gmm_points(200_000, seed=23, k=8)
    reqs = gen.density_tiles(pts, 2500, 4, 14, 24, seed=24)
    L = points_layer(ctx, pts)
    try:
        for mode in (hv.HV_MODE_MASK, hv.HV_MODE_COVERAGE):
            host = hv.render(L, reqs, mode, style())
            dev = render_dev(L, reqs, mode)
            assert np.array_equal(host, dev)
        pinned = torch.empty((len(reqs), 8192), dtype=torch.uint8, pin_memory=True)
        hv.hv_render_tiles(L, hv.make_requests(reqs), len(reqs), hv.HV_MODE_MASK, hv.HV_INDEX_RTREE,
                           style(), pinned, pinned.numel(), None)
        assert np.array_equal(pinned.numpy(), render_dev(L, reqs, hv.HV_MODE_MASK))
    finally:
        hv.hv_layer_free(L)


@pytest.mark.parametrize("kind", ["points", "polygons"])
def test_pinned_host_output_written_by_the_kernels(ctx, kind):
    """Pinned host output is written by the kernels over the CPU-GPU link
    (the polygon layers' fill bits read back from it too): equal to the
    oracle in every mode, with host and with device requests."""
    if kind == "points":
        pts = gen.gmm_points(100_000, seed=25, k=8)
        L = points_layer(ctx, pts)
        reqs = gen.density_tiles(pts, 300, 4, 14, [8, 32], seed=26)
        ref = lambda m: oracle.render_points(pts, reqs, m, STYLE_T)
    else:
        xy, ro, po = gen.star_polygons(2_000, seed=27, k=8, rho_median=6e-4)
        L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
        hv.hv_layer_build_index(L)
        reqs = gen.density_tiles(gen.polygon_centres(xy, ro, po), 40, 3, 12, 8, seed=28)
        ref = lambda m: oracle.render_polygons(xy, ro, po, reqs, m, STYLE_T)
    try:
        d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
        for mode in MODES:
            want = ref(mode)
            for rq in (hv.make_requests(reqs), d_req):
                out = torch.full((len(reqs), hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, pin_memory=True)
                hv.hv_render_tiles(L, rq, len(reqs), mode, hv.HV_INDEX_RTREE, style(), out, out.numel(),
                                   torch.cuda.current_stream())
                assert np.array_equal(out.numpy(), want)
    finally:
        hv.hv_layer_free(L)


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_phase_profile_launch(ctx, kind):
    """The instrumented (phase-profile) launch renders the oracle's tiles, and
    its counters nest: the launch holds the block phase, busy warps are part
    of it, descents part of those, leaf visits part of the descents."""
    if kind == "points":
        pts = gen.gmm_points(80_000, seed=31, k=8)
        L = hv.hv_layer_load_points(ctx, pts)
        reqs = gen.density_tiles(pts, 30, 3, 14, [8, 32], seed=32)
        ref = lambda r, m: oracle.render_points(pts, r, m, STYLE_T)
    elif kind == "lines":
        xy, off = gen.walk_lines(4_000, 30_000, seed=33, n_cities=10)
        L = hv.hv_layer_load_linestrings(ctx, xy, off)
        reqs = gen.density_tiles(gen.segment_midpoints(xy, off, 2000), 30, 3, 15, [8, 24], seed=34)
        ref = lambda r, m: oracle.render_lines(xy, off, r, m, STYLE_T)
    else:
        xy, ro, po = gen.star_polygons(3_000, seed=35, k=8, rho_median=6e-4)
        L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
        reqs = gen.density_tiles(gen.polygon_centres(xy, ro, po), 20, 3, 12, 8, seed=36)
        ref = lambda r, m: oracle.render_polygons(xy, ro, po, r, m, STYLE_T)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
            n = len(reqs)
            d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
            out = torch.full((n, hv.hv_tile_bytes(hv.HV_MODE_RGBA)), 0xAB, dtype=torch.uint8, device="cuda")
            ph = torch.zeros(2 * hv.HV_PHASE_COUNT, dtype=torch.int64, device="cuda")
            hv.hv_render_tiles_phases(L, d_req, n, hv.HV_MODE_RGBA, index, style(), out, out.numel(), ph)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref(reqs, hv.HV_MODE_RGBA))
            v = ph.cpu().numpy()
            for part in range(2 if kind == "polygons" else 1):
                c = v[16 * part:16 * part + 16]
                assert c[9] in (n * 16, n * 32, n * 64)         # one CTA per strip of 16, 8 or 4 rows
                assert c[0] >= c[4] >= c[5] >= c[7] >= c[6] > 0
                assert c[0] >= c[1] + c[2] + c[3] + c[4] + c[8]
                assert 0 < c[10] <= n * 2048                    # 8 x 4 blocks of strips with work
            if kind != "polygons":
                assert not v[16:].any()
    finally:
        hv.hv_layer_free(L)
