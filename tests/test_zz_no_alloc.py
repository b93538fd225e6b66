"""The allocation-free entry point against the allocating one.

hv_render_tiles_static serves callers that may not allocate device memory
(when another allocator or pool owns the device's memory, or on paths that
cannot take the synchronisation an allocation may imply): it stages host
requests in a fixed device array of the library instead of cudaMalloc'd
scratch, and reads device requests in place.  Its tiles must equal
hv_render_tiles' exactly, call after call, although every call with host
requests reuses the same staging array.
"""
import numpy as np
import pytest

from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402


def test_static_entry_matches_allocating_entry():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = hv.hv_create(0)
    try:
        pts = gen.gmm_points(300_000, seed=91, k=16)
        L = hv.hv_layer_load_points(ctx, pts)
        hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE)
        style = hv.make_style((200, 30, 60), (20, 140, 250))
        stream = torch.cuda.current_stream()
        try:
            # two calls in a row with different requests: the second must not
            # see anything of the first in the shared staging array
            for seed, n, mode in ((92, 300, hv.HV_MODE_RGBA), (93, 17, hv.HV_MODE_COVERAGE)):
                reqs = hv.make_requests(gen.density_tiles(pts, n, 3, 15, [8, 32], seed=seed))
                tb = hv.hv_tile_bytes(mode)
                ref = torch.zeros((n, tb), dtype=torch.uint8, device="cuda")
                hv.hv_render_tiles(L, reqs, n, mode, hv.HV_INDEX_RTREE, style, ref, ref.numel(), stream)
                got = torch.full((n, tb), 0xAB, dtype=torch.uint8, device="cuda")
                hv.hv_render_tiles_static(L, reqs, n, mode, hv.HV_INDEX_RTREE, style, got, got.numel(), stream)
                stream.synchronize()
                assert torch.equal(got, ref)
            # the whole staging array (4096 requests), then device-resident
            # requests (read in place) twice in a row
            full = hv.make_requests(gen.density_tiles(pts, 4096, 2, 16, [4, 16, 40], seed=99))
            ref = torch.zeros((4096, 8192), dtype=torch.uint8, device="cuda")
            hv.hv_render_tiles(L, full, 4096, hv.HV_MODE_MASK, hv.HV_INDEX_RTREE, None, ref, ref.numel(), stream)
            got = torch.full((4096, 8192), 0xAB, dtype=torch.uint8, device="cuda")
            hv.hv_render_tiles_static(L, full, 4096, hv.HV_MODE_MASK, hv.HV_INDEX_RTREE, None, got,
                                      got.numel(), stream)
            stream.synchronize()
            assert torch.equal(got, ref)
            d_full = torch.from_numpy(full.view(np.uint8).copy()).cuda()
            for n in (4096, 123):
                got.fill_(0xCD)
                hv.hv_render_tiles_static(L, d_full, n, hv.HV_MODE_MASK, hv.HV_INDEX_RTREE, None, got,
                                          got.numel(), stream)
                stream.synchronize()
                assert torch.equal(got[:n], ref[:n])
            with pytest.raises(hv.HVError) as e:
                big = hv.make_requests(np.tile([[3, 1, 1, 16]], (4097, 1)))
                hv.hv_render_tiles_static(L, big, 4097, hv.HV_MODE_MASK, hv.HV_INDEX_RTREE, None, got,
                                          got.numel(), stream)
            assert e.value.status == hv.HV_EINVAL
        finally:
            hv.hv_layer_free(L)
    finally:
        hv.hv_destroy(ctx)


@pytest.mark.parametrize("kind", ["lines", "polygons"])
def test_static_entry_other_layer_kinds(kind):
    """Segments (one launch) and polygons (an outline and a fill launch, the
    second reading the first's output) through the staging array."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = hv.hv_create(0)
    try:
        if kind == "lines":
            xy, off = gen.walk_lines(3_000, 20_000, seed=94, n_cities=10)
            anchors = gen.segment_midpoints(xy, off, 2000, seed=95)
            L = hv.hv_layer_load_linestrings(ctx, xy, off)
        else:
            xy, ro, po = gen.star_polygons(3_000, seed=96, k=8, rho_median=6e-4)
            anchors = gen.polygon_centres(xy, ro, po)
            L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
        hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE)
        style = hv.make_style((200, 30, 60), (20, 140, 250))
        stream = torch.cuda.current_stream()
        try:
            for seed, n, mode in ((97, 40, hv.HV_MODE_RGBA), (98, 9, hv.HV_MODE_MASK)):
                reqs = hv.make_requests(gen.density_tiles(anchors, n, 3, 14, [8, 24], seed=seed))
                tb = hv.hv_tile_bytes(mode)
                ref = torch.zeros((n, tb), dtype=torch.uint8, device="cuda")
                hv.hv_render_tiles(L, reqs, n, mode, hv.HV_INDEX_RTREE, style, ref, ref.numel(), stream)
                got = torch.full((n, tb), 0xAB, dtype=torch.uint8, device="cuda")
                hv.hv_render_tiles_static(L, reqs, n, mode, hv.HV_INDEX_RTREE, style, got, got.numel(), stream)
                stream.synchronize()
                assert torch.equal(got, ref)
        finally:
            hv.hv_layer_free(L)
    finally:
        hv.hv_destroy(ctx)
