"""Fill styles of polygon layers (Sec. 3.2.2 fill styles, Sec. 4.1 Pattern
Library) against the oracle, byte for byte: the anti-aliased fill (decided at
the four super-samples, the outline composed over the partly covered fill)
and pattern fill anchored to the global pixel grid, alone and together, in
every output mode, through the R-tree and the learned index."""
import numpy as np
import pytest

import oracle
import oracle_par
from geom import polys_to_arrays, random_star_polygons
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


def hatch():
    """A 5 x 3 pattern: a diagonal hatch of two colours on transparency."""
    p = np.zeros((3, 5, 4), dtype=np.uint8)
    for j in range(3):
        p[j, (2 * j) % 5] = (250, 200, 10, 255)
        p[j, (2 * j + 1) % 5] = (10, 120, 250, 255)
    return p


def render(L, reqs, mode, fill, index):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((n, hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    hv.hv_render_tiles_styled(L, d_req, n, mode, index, hv.make_style(STYLE_T[:3], STYLE_T[4:7]), fill, out,
                              out.numel(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(ctx, xy, ro, po, reqs):
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    try:
        for aa, pat in ((True, None), (False, hatch()), (True, hatch())):
            fill = hv.make_fill_style(aa, pat)
            for mode in MODES:
                ref = oracle_par.render(lambda r: oracle.render_polygons(xy, ro, po, r, mode, STYLE_T, aa=aa,
                                                                         pattern=pat), reqs)
                for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
                    got = render(L, reqs, mode, fill, index)
                    bad = np.nonzero((got != ref).any(axis=1))[0]
                    assert bad.size == 0, "aa=%s pattern=%s mode %d index %d: tiles %s" % (
                        aa, pat is not None, mode, index, bad[:5])
    finally:
        hv.hv_layer_free(L)


def test_star_polygons(ctx):
    xy, ro, po = gen.star_polygons(2_000, seed=81, k=8, rho_median=6e-4)
    reqs = gen.density_tiles(gen.polygon_centres(xy, ro, po), 16, 4, 12, [1, 8, 24], seed=82)
    check(ctx, xy, ro, po, reqs)


def test_large_polygons_with_holes_and_lattice_vertices(ctx):
    rng = np.random.default_rng(83)
    polys = random_star_polygons(rng, 6, 6, 20, 30, 60, 128, 128, 30, holes=True)
    polys += random_star_polygons(rng, 40, 13, 3000, 5000, 30, 128, 128, 60, holes=True, snap=True)
    xy, ro, po = polys_to_arrays(polys)
    cen = gen.polygon_centres(xy, ro, po)
    reqs = np.concatenate([gen.density_tiles(cen, 20, 8, 15, [1, 8], seed=84),
                           gen.density_tiles(xy, 20, 9, 15, [8], seed=85),
                           np.array([[13, 3000, 5000, 4], [14, 6001, 10001, 8]], dtype=np.uint32)])
    check(ctx, xy, ro, po, reqs)


def test_host_output_and_bad_styles(ctx):
    xy, ro, po = gen.star_polygons(500, seed=86, k=4, rho_median=1e-3)
    reqs = gen.density_tiles(gen.polygon_centres(xy, ro, po), 6, 4, 10, 8, seed=87)
    L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L)
    try:
        fill = hv.make_fill_style(True, hatch())
        out = np.zeros((len(reqs), hv.hv_tile_bytes(hv.HV_MODE_RGBA)), np.uint8)
        hv.hv_render_tiles_styled(L, hv.make_requests(reqs), len(reqs), hv.HV_MODE_RGBA, hv.HV_INDEX_RTREE,
                                  hv.make_style(STYLE_T[:3], STYLE_T[4:7]), fill, out, out.nbytes)
        ref = oracle.render_polygons(xy, ro, po, reqs, hv.HV_MODE_RGBA, STYLE_T, aa=True, pattern=hatch())
        assert np.array_equal(out, ref)
        # no fill style: the plain rendering
        plain = np.zeros_like(out)
        hv.hv_render_tiles_styled(L, hv.make_requests(reqs), len(reqs), hv.HV_MODE_RGBA, hv.HV_INDEX_RTREE,
                                  hv.make_style(STYLE_T[:3], STYLE_T[4:7]), None, plain, plain.nbytes)
        assert np.array_equal(plain, oracle.render_polygons(xy, ro, po, reqs, hv.HV_MODE_RGBA, STYLE_T))
        for bad in (np.full((2, 2, 4), 128, np.uint8), np.zeros((17, 2, 4), np.uint8)):
            with pytest.raises(hv.HVError) as e:
                hv.hv_render_tiles_styled(L, hv.make_requests(reqs), len(reqs), hv.HV_MODE_RGBA, hv.HV_INDEX_RTREE,
                                          None, hv.make_fill_style(False, bad), out, out.nbytes)
            assert e.value.status == hv.HV_EINVAL
    finally:
        hv.hv_layer_free(L)
