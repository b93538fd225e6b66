"""Small batches: the same tiles rendered one at a time (each 4-row strip
split into 4 column parts, one CTA each), three at a time (2 parts) and as
one batch (full-width strips), for every layer kind and output mode, plain,
anti-aliased and patterned polygon fills, R-tree and learned index; every
tile equal to the oracle's byte for byte (Algorithm 1, Algorithm 2)."""
import numpy as np
import pytest

import oracle
import oracle_par
from geom import (lines_to_arrays, polys_to_arrays, random_cluster_points, random_star_polygons,
                  random_walk_lines)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE_T = (230, 40, 20, 0, 30, 90, 200, 0)
MODES = [hv.HV_MODE_MASK, hv.HV_MODE_COVERAGE, hv.HV_MODE_RGBA]
Z, TX, TY = 12, 1400, 1800


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


def _requests():
    """The tile the objects sit in, its neighbours, its parent and children,
    at several radii (strips and column parts cross the objects everywhere)."""
    out = []
    for dx, dy in ((0, 0), (1, 0), (0, 1), (-1, -1)):
        out.append([Z, TX + dx, TY + dy, 16])
    out += [[Z - 1, TX // 2, TY // 2, 24], [Z + 1, 2 * TX + 1, 2 * TY, 8], [Z + 2, 4 * TX + 1, 4 * TY + 2, 40]]
    return np.array(out, dtype=np.uint32)


def _hatch():
    p = np.zeros((3, 5, 4), dtype=np.uint8)
    for j in range(3):
        p[j, (2 * j) % 5] = (250, 200, 10, 255)
        p[j, (2 * j + 1) % 5] = (10, 120, 250, 255)
    return p


def _render(L, reqs, mode, index, fill):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((n, hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    style = hv.make_style(STYLE_T[:3], STYLE_T[4:7])
    s = torch.cuda.current_stream()
    if fill is None:
        hv.hv_render_tiles(L, d_req, n, mode, index, style, out, out.numel(), s)
    else:
        hv.hv_render_tiles_styled(L, d_req, n, mode, index, style, fill, out, out.numel(), s)
    s.synchronize()
    return out.cpu().numpy()


def _check(L, reqs, mode, ref, fill=None):
    for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
        for size in (1, 3, len(reqs)):
            got = np.concatenate([_render(L, reqs[k:k + size], mode, index, fill)
                                  for k in range(0, len(reqs), size)])
            bad = np.nonzero((got != ref).any(axis=1))[0]
            assert bad.size == 0, "mode %d index %d batches of %d: tiles %s differ" % (mode, index, size, bad)


def test_points(ctx):
    rng = np.random.default_rng(91)
    pts = random_cluster_points(rng, 20000, Z, TX, TY, 60)
    reqs = _requests()
    L = hv.hv_layer_load_points(ctx, pts)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for mode in MODES:
            ref = oracle_par.render(lambda r: oracle.render_points(pts, r, mode, STYLE_T), reqs)
            assert (ref != 0).any()
            _check(L, reqs, mode, ref)
    finally:
        hv.hv_layer_free(L)


def test_lines(ctx):
    rng = np.random.default_rng(92)
    xy, off = lines_to_arrays(random_walk_lines(rng, 400, 12, Z, TX, TY, 6))
    reqs = _requests()
    L = hv.hv_layer_load_linestrings(ctx, xy, off)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for mode in MODES:
            ref = oracle_par.render(lambda r: oracle.render_lines(xy, off, r, mode, STYLE_T), reqs)
            assert (ref != 0).any()
            _check(L, reqs, mode, ref)
    finally:
        hv.hv_layer_free(L)


@pytest.mark.parametrize("aa,pattern", [(False, False), (True, False), (True, True)])
def test_polygons(ctx, aa, pattern):
    rng = np.random.default_rng(93)
    xy, ro, po = polys_to_arrays(random_star_polygons(rng, 300, Z, TX, TY, 9, holes=True))
    reqs = _requests()
    pat = _hatch() if pattern else None
    fill = hv.make_fill_style(aa, pat) if (aa or pattern) else None
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for mode in MODES:
            ref = oracle_par.render(lambda r: oracle.render_polygons(xy, ro, po, r, mode, STYLE_T, aa=aa,
                                                                     pattern=pat), reqs)
            assert (ref != 0).any()
            _check(L, reqs, mode, ref, fill)
    finally:
        hv.hv_layer_free(L)
