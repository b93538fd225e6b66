"""Layer files: a saved and reloaded layer renders byte-equal tiles with
both indexes, without a rebuild (the paper keeps its indexes as files, Sec. 4)."""
import numpy as np
import pytest

from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_12489_gb300 import hv  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hv.hv_create(0)
    yield c
    hv.hv_destroy(c)


def build(ctx, kind):
    if kind == "points":
        a = gen.gmm_points(200_000, seed=71, k=8)
        L = hv.hv_layer_load_points(ctx, a)
    elif kind == "lines":
        xy, off = gen.walk_lines(5_000, 40_000, seed=72, n_cities=10)
        a = gen.segment_midpoints(xy, off, 1000)
        L = hv.hv_layer_load_linestrings(ctx, xy, off)
    else:
        xy, ro, po = gen.star_polygons(3_000, seed=73, k=8, rho_median=6e-4)
        a = gen.polygon_centres(xy, ro, po)
        L = hv.hv_layer_load_polygons(ctx, xy, ro, po)
    hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    return L, gen.density_tiles(a, 30, 3, 12, [8, 24], seed=74)


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_save_load_roundtrip(ctx, kind, tmp_path):
    L, reqs = build(ctx, kind)
    path = str(tmp_path / ("%s.hvl" % kind))
    style = hv.make_style((200, 10, 10), (10, 10, 200))
    try:
        hv.hv_layer_save(L, path)
        L2 = hv.hv_layer_load_file(ctx, path)
        try:
            i1, i2 = hv.info_dict(L), hv.info_dict(L2)
            for k in ("kind", "indexes", "n_objects", "n_polygons", "mbr", "tree_levels", "tree_nodes",
                      "learned_error", "learned_outliers", "learned_pieces", "learned_halo"):
                assert i1[k] == i2[k], k
            for index in (hv.HV_INDEX_RTREE, hv.HV_INDEX_LEARNED):
                a = hv.render(L, reqs, hv.HV_MODE_RGBA, style, index)
                b = hv.render(L2, reqs, hv.HV_MODE_RGBA, style, index)
                assert np.array_equal(a, b)
        finally:
            hv.hv_layer_free(L2)
    finally:
        hv.hv_layer_free(L)


def test_bad_files(ctx, tmp_path):
    with pytest.raises(hv.HVError) as e:
        hv.hv_layer_load_file(ctx, str(tmp_path / "missing.hvl"))
    assert e.value.status == hv.HV_EINVAL
    p = tmp_path / "junk.hvl"
    p.write_bytes(b"not a layer file at all" * 10)
    with pytest.raises(hv.HVError) as e:
        hv.hv_layer_load_file(ctx, str(p))
    assert e.value.status == hv.HV_EINVAL
    L, _ = build(ctx, "points")
    try:
        good = tmp_path / "good.hvl"
        hv.hv_layer_save(L, str(good))
        data = good.read_bytes()
        (tmp_path / "cut.hvl").write_bytes(data[: len(data) // 2])
        with pytest.raises(hv.HVError) as e:
            hv.hv_layer_load_file(ctx, str(tmp_path / "cut.hvl"))
        assert e.value.status == hv.HV_EINVAL
        assert hv.hv_ctx_device_bytes(ctx) > 0
    finally:
        hv.hv_layer_free(L)
