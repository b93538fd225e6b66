"""Display-driven buffer and overlay analysis (HiBuffer and HiBO, Sec. 2.3;
SIBV extends HiBuffer's buffers, Sec. 3.2) against the oracle, byte for byte:
the buffer of a layer at a distance given in grid units (whatever the zoom),
and the bitwise overlay of two layers' buffers."""
import numpy as np
import pytest

import oracle
import oracle_par
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
def layers(ctx):
    pts = gen.gmm_points(100_000, seed=61, k=8)
    xy, off = gen.walk_lines(5_000, 40_000, seed=62, n_cities=10)
    pxy, ro, po = gen.star_polygons(3_000, seed=63, k=8, rho_median=6e-4)
    Ls = {"points": hv.hv_layer_load_points(ctx, pts), "lines": hv.hv_layer_load_linestrings(ctx, xy, off),
          "polygons": hv.hv_layer_load_polygons(ctx, pxy, ro, po)}
    for L in Ls.values():
        hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    src = {"points": (pts,), "lines": (xy, off), "polygons": (pxy, ro, po)}
    anchors = {"points": pts, "lines": gen.segment_midpoints(xy, off, 2000),
               "polygons": gen.polygon_centres(pxy, ro, po)}
    yield Ls, src, anchors
    for L in Ls.values():
        hv.hv_layer_free(L)


def ref_buffer(kind, src, reqs, mode, R):
    f = {"points": oracle.render_points, "lines": oracle.render_lines, "polygons": oracle.render_polygons}[kind]
    return f(*src[kind], reqs, mode, STYLE_T, R_units=R)


def gpu_buffer(L, reqs, mode, R, index=hv.HV_INDEX_RTREE):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((n, hv.hv_tile_bytes(mode)), 0xAB, dtype=torch.uint8, device="cuda")
    hv.hv_render_buffer(L, d_req, n, mode, index, R, hv.make_style(STYLE_T[:3], STYLE_T[4:7]), out, out.numel(),
                        torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_buffer_equals_oracle(layers, kind):
    """Radii of 0, a few, hundreds and thousands of pixels at the tiles'
    zooms, none a multiple of 1/16 px at all of them; R-tree and learned
    index.  (The oracle splats every object over every pixel in its reach, so
    the wide radii use fewer tiles and modes.)"""
    Ls, src, anchors = layers
    reqs = gen.density_tiles(anchors[kind], 24, 4, 16, 1, seed=64)
    reqs[:, 3] = 0                                     # r16 is ignored
    cases = [(0, MODES, reqs), (1234, MODES, reqs), (98765, [hv.HV_MODE_COVERAGE], reqs[reqs[:, 0] <= 14][:12]),
             (3_000_000, [hv.HV_MODE_MASK], reqs[reqs[:, 0] <= 8][:6])]
    for R, modes, rq in cases:
        for mode in modes:
            ref = oracle_par.render(lambda r: ref_buffer(kind, src, r, mode, R), rq)
            for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
                got = gpu_buffer(Ls[kind], rq, mode, R, index)
                bad = np.nonzero((got != ref).any(axis=1))[0]
                assert bad.size == 0, "R=%d mode %d index %d: tiles %s differ" % (R, mode, index, bad[:5])


def test_buffer_host_buffers_and_range(layers):
    Ls, src, anchors = layers
    reqs = gen.density_tiles(anchors["points"], 5, 6, 12, 1, seed=65)
    out = np.zeros((len(reqs), 8192), np.uint8)
    hv.hv_render_buffer(Ls["points"], hv.make_requests(reqs), len(reqs), hv.HV_MODE_MASK, hv.HV_INDEX_RTREE,
                        50_000, None, out, out.nbytes)
    assert np.array_equal(out, ref_buffer("points", src, reqs, hv.HV_MODE_MASK, 50_000))
    for bad in (-1, (1 << 29) + 1):
        with pytest.raises(hv.HVError) as e:
            hv.hv_render_buffer(Ls["points"], hv.make_requests(reqs), len(reqs), hv.HV_MODE_MASK,
                                hv.HV_INDEX_RTREE, bad, None, out, out.nbytes)
        assert e.value.status == hv.HV_ERANGE


@pytest.mark.parametrize("a,b", [("points", "lines"), ("polygons", "points"), ("lines", "polygons"),
                                 ("polygons", "polygons")])
def test_overlay_equals_oracle(layers, a, b):
    Ls, src, anchors = layers
    reqs = np.concatenate([gen.density_tiles(anchors[a], 10, 5, 14, 1, seed=66),
                           gen.density_tiles(anchors[b], 10, 5, 14, 1, seed=67)])
    ra, rb = 40_000, 250_000
    ma = np.array([oracle.mask_bits(t) for t in ref_buffer(a, src, reqs, hv.HV_MODE_MASK, ra)])
    mb = np.array([oracle.mask_bits(t) for t in ref_buffer(b, src, reqs, hv.HV_MODE_MASK, rb)])
    want = {hv.HV_OVERLAY_AND: ma & mb, hv.HV_OVERLAY_OR: ma | mb, hv.HV_OVERLAY_XOR: ma ^ mb,
            hv.HV_OVERLAY_DIFF: ma & ~mb}
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    for op, w in want.items():
        out = torch.full((n, 8192), 0xAB, dtype=torch.uint8, device="cuda")
        hv.hv_overlay_tiles(Ls[a], ra, Ls[b], rb, op, d_req, n, hv.HV_INDEX_RTREE, out, out.numel(),
                            torch.cuda.current_stream())
        got = np.array([oracle.mask_bits(t) for t in out.cpu().numpy()])
        assert np.array_equal(got, w), "op %d" % op
    with pytest.raises(hv.HVError):
        hv.hv_overlay_tiles(Ls[a], ra, Ls[b], rb, 7, d_req, n, hv.HV_INDEX_RTREE, out, out.numel())
