"""Index records in host memory (HV_PLACE_HOST: read by the kernels over the
CPU-GPU link, the role of the paper's memory-mapped index files, Sec. 4):
tiles equal the oracle's and the device-resident layer's, with both indexes,
and the layer holds its records in host memory instead of device memory."""
import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402

STYLE_T = (230, 40, 20, 0, 30, 90, 200, 0)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


def render(L, reqs, index):
    n = len(reqs)
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    out = torch.full((n, hv.hv_tile_bytes(hv.HV_MODE_RGBA)), 0xAB, dtype=torch.uint8, device="cuda")
    hv.hv_render_tiles(L, d_req, n, hv.HV_MODE_RGBA, index, hv.make_style(STYLE_T[:3], STYLE_T[4:7]), out,
                       out.numel(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_host_resident_records(ctx, kind, tmp_path):
    if kind == "points":
        pts = gen.gmm_points(200_000, seed=71, k=8)
        load = lambda: hv.hv_layer_load_points(ctx, pts)
        reqs = gen.density_tiles(pts, 40, 3, 15, [8, 40], seed=72)
        ref = oracle.render_points(pts, reqs, hv.HV_MODE_RGBA, STYLE_T)
    elif kind == "lines":
        xy, off = gen.walk_lines(8_000, 60_000, seed=73, n_cities=10)
        load = lambda: hv.hv_layer_load_linestrings(ctx, xy, off)
        reqs = gen.density_tiles(gen.segment_midpoints(xy, off, 3000), 40, 3, 16, [8, 24], seed=74)
        ref = oracle.render_lines(xy, off, reqs, hv.HV_MODE_RGBA, STYLE_T)
    else:
        xy, ro, po = gen.star_polygons(3_000, seed=75, k=8, rho_median=6e-4)
        load = lambda: hv.hv_layer_load_polygons(ctx, xy, ro, po)
        reqs = gen.density_tiles(gen.polygon_centres(xy, ro, po), 20, 3, 12, 8, seed=76)
        ref = oracle.render_polygons(xy, ro, po, reqs, hv.HV_MODE_RGBA, STYLE_T)
    dev, host = load(), load()
    opts = hv.hv_build_opts()
    opts.object_placement = hv.HV_PLACE_HOST
    hv.hv_layer_build_index(dev, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    hv.hv_layer_build_index(host, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED, opts)
    try:
        di, hi = hv.hv_layer_info_get(dev), hv.hv_layer_info_get(host)
        assert di.host_bytes == 0 and hi.host_bytes > 0
        assert hi.device_bytes + hi.host_bytes == di.device_bytes
        for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
            got = render(host, reqs, index)
            assert np.array_equal(got, ref), "index %d" % index
            assert np.array_equal(got, render(dev, reqs, index))
        # a saved host-resident layer loads back with device-resident records
        path = str(tmp_path / "layer.hvl")
        hv.hv_layer_save(host, path)
        back = hv.hv_layer_load_file(ctx, path)
        try:
            assert hv.hv_layer_info_get(back).host_bytes == 0
            assert np.array_equal(render(back, reqs, hv.HV_INDEX_RTREE), ref)
        finally:
            hv.hv_layer_free(back)
    finally:
        hv.hv_layer_free(dev)
        hv.hv_layer_free(host)
