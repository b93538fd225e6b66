"""GPU parity at the edge of the distance test: samples at exactly R, R +- 1
and R +- 2 grid units from long segments and polygon edges (Algorithm 1's
closed test `distance <= R`).

The segment kernels first decide a sample in single precision and fall back
to the exact integer test only inside an error margin; these layers put
samples on both sides of R by one or two units, with segments whose
endpoints lie up to 2^28 units away (large projection offsets) and on tiles
near the grid's edges (large coordinates), at zooms 4-19 and several radii.
Every tile is compared with the oracle byte for byte.
"""
import numpy as np
import pytest

import oracle
import oracle_par
from geom import centre, ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE_T = (230, 40, 20, 0, 30, 90, 200, 0)
MODES = [hv.HV_MODE_MASK, hv.HV_MODE_COVERAGE, hv.HV_MODE_RGBA]
HALF = 1 << 30
LONG = 1 << 28


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


def _clip(v):
    return int(min(max(v, -HALF), HALF - 1))


def _samples(z, tx, ty, i, j):
    """The pixel centre and one super-sample (+off, +off) of pixel (i, j)."""
    cx, cy = centre(z, tx, ty, i, j)
    off = ps(z) // 4
    return [(cx, cy), (cx + off, cy + off)]


def _segments_around(sx, sy, R):
    """Segments whose distance from (sx, sy) is R or just beyond, reached in
    the interior (axis-parallel and 3-4-5 slanted lines) and at an endpoint."""
    segs = []
    for d in (R, R + 1, R + 2, -R, -(R + 1)):
        segs.append((sx - LONG, sy + d, sx + LONG, sy + d))          # across: |d|
        segs.append((sx + d, sy - LONG, sx + d, sy + LONG))
    for d in (R - 1, R, R + 1):
        segs.append((sx + d, sy, sx + d + LONG, sy + 7))             # endpoint at (d, 0)
        segs.append((sx, sy - d, sx - 5, sy - d - LONG))             # endpoint at (0, -d)
    k0 = R // 5
    t = LONG // 5
    for k in (k0, k0 + 1):
        # the line through (sx - 3k, sy + 4k) along (4, 3): distance 5k
        px, py = sx - 3 * k, sy + 4 * k
        segs.append((px - 4 * t, py - 3 * t, px + 4 * t, py + 3 * t))
        # an endpoint at distance 5k along (3, 4), the segment leading away
        segs.append((sx + 3 * k, sy + 4 * k, sx + 3 * k + 3 * t, sy + 4 * k + 4 * t))
    return [tuple(_clip(v) for v in s) for s in segs]


def _cases():
    """(z, tile x, tile y, r16): tiles near the centre and near the grid's
    corners, where coordinates are largest."""
    out = []
    for z in (4, 8, 12, 16, 19):
        n = 1 << z
        for (tx, ty) in ((n // 2 - 1, n // 2), (n - 1, n - 1), (0, n - 1)):
            for r16 in (8, 16, 24, 40):
                out.append((z, tx, ty, r16))
    return out


def _layer_and_requests():
    segs, reqs = [], []
    rng = np.random.default_rng(5)
    for (z, tx, ty, r16) in _cases():
        R = r16 << (19 - z)
        for (i, j) in ((int(rng.integers(8, 248)), int(rng.integers(8, 248))), (0, 255)):
            for (sx, sy) in _samples(z, tx, ty, i, j):
                segs += _segments_around(sx, sy, R)
        reqs.append([z, tx, ty, r16])
    xy = np.array([[a, b] for s in segs for a, b in ((s[0], s[1]), (s[2], s[3]))], dtype=np.int32)
    off = np.arange(0, 2 * len(segs) + 1, 2, dtype=np.uint64)
    return xy, off, np.array(reqs, dtype=np.uint32)


def _render(layer, reqs, mode):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((n, hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    hv.hv_render_tiles(layer, d_req, n, mode, hv.HV_INDEX_RTREE, hv.make_style(STYLE_T[:3], STYLE_T[4:7]),
                       out, out.numel(), s)
    s.synchronize()
    return out.cpu().numpy()


def test_lines_at_the_radius(ctx):
    xy, off, reqs = _layer_and_requests()
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L)
    try:
        for mode in MODES:
            got = _render(L, reqs, mode)
            ref = oracle_par.render(lambda r: oracle.render_lines(xy, off, r, mode, STYLE_T), reqs)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
            # the layer does reach the tiles: some pixels are covered
            assert (ref != 0).any()
    finally:
        hv.hv_layer_free(L)


def test_polygon_outlines_at_the_radius(ctx):
    """Squares whose edges pass at R and R + 1 from a sample: the outline
    launch's distance test at its margins, composed over the fill."""
    rings = []
    rng = np.random.default_rng(6)
    reqs = []
    for (z, tx, ty, r16) in _cases():
        R = r16 << (19 - z)
        i, j = int(rng.integers(8, 248)), int(rng.integers(8, 248))
        for (sx, sy) in _samples(z, tx, ty, i, j):
            for d in (R, R + 1):
                # the square's left edge at x = sx + d, the square to the right
                x0, x1 = _clip(sx + d), _clip(sx + d + LONG)
                y0, y1 = _clip(sy - LONG), _clip(sy + LONG)
                if x1 > x0:
                    rings.append([(x0, y0), (x1, y0), (x1, y1), (x0, y1)])
        reqs.append([z, tx, ty, r16])
    xy = np.array([p for r in rings for p in r], dtype=np.int32)
    ro = np.arange(0, 4 * len(rings) + 1, 4, dtype=np.uint64)
    po = np.arange(0, len(rings) + 1, dtype=np.uint64)
    reqs = np.array(reqs, dtype=np.uint32)
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L)
    try:
        for mode in MODES:
            got = _render(L, reqs, mode)
            ref = oracle_par.render(lambda r: oracle.render_polygons(xy, ro, po, r, mode, STYLE_T), reqs)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
    finally:
        hv.hv_layer_free(L)


def test_leaves_with_more_pairs_than_one_round(ctx):
    """Hundreds of long segments through the same pixel blocks at a 64 px
    half-width: a leaf's 32 pieces each reach every pixel of a block, up to
    1,024 (piece, pixel) pairs, staged and tested in rounds of 128; every
    tile equals the oracle's."""
    z, tx, ty = 16, 30000, 25000
    rng = np.random.default_rng(7)
    segs = []
    for k in range(400):
        cx, cy = centre(z, tx, ty, int(rng.integers(0, 64)), int(rng.integers(0, 64)))
        ang = rng.uniform(0, np.pi)
        L_ = int(rng.integers(1 << 12, 1 << 22))
        dx, dy = int(L_ * np.cos(ang)), int(L_ * np.sin(ang))
        segs.append(tuple(_clip(v) for v in (cx - dx, cy - dy, cx + dx, cy + dy)))
    xy = np.array([[a, b] for s in segs for a, b in ((s[0], s[1]), (s[2], s[3]))], dtype=np.int32)
    off = np.arange(0, 2 * len(segs) + 1, 2, dtype=np.uint64)
    reqs = np.array([[z, tx, ty, 1024], [z, tx, ty, 512], [z, tx, ty, 96], [z - 1, tx // 2, ty // 2, 1024],
                     [z, tx + 1, ty, 1024]],
                    dtype=np.uint32)
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L)
    try:
        for mode in MODES:
            got = _render(L, reqs, mode)
            ref = oracle_par.render(lambda r: oracle.render_lines(xy, off, r, mode, STYLE_T), reqs)
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d: %d tiles differ, first %s" % (mode, bad.size, reqs[bad[0]])
    finally:
        hv.hv_layer_free(L)
