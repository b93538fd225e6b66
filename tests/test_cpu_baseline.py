"""The multithreaded CPU R-tree baseline renders the oracle's tiles."""
import numpy as np

import oracle
from workloads import gen


def test_cpu_rtree_matches_oracle():
    import cpu_baseline
    pts = gen.gmm_points(150_000, seed=95, k=8)
    reqs = gen.density_tiles(pts, 12, 2, 16, [8, 32, 70], seed=96)
    t = cpu_baseline.PointTree(pts, threads=4)
    got, threads = t.render_rgba(reqs, (230, 40, 20))
    assert threads == 4
    ref = oracle.render_points(pts, reqs, oracle.MODE_RGBA, (230, 40, 20, 0, 0, 0, 0, 0))
    assert np.array_equal(got, ref)
    t.close()


def test_cpu_rtree_empty_layer():
    import cpu_baseline
    t = cpu_baseline.PointTree(np.zeros((0, 2), np.int32), threads=2)
    got, _ = t.render_rgba([[3, 1, 1, 16]], (1, 2, 3))
    assert not got.any()


STYLE = (230, 40, 20, 0, 30, 90, 200, 0)


def test_cpu_rtree_lines_match_oracle():
    import cpu_baseline
    xy, off = gen.walk_lines(2_000, 15_000, seed=97, n_cities=12)
    extra = np.array([[-(1 << 29), 5], [1 << 29, 900], [3, 3]], dtype=np.int32)   # a long and a 1-vertex line
    xy = np.concatenate([xy, extra])
    off = np.concatenate([off, [off[-1] + 2, off[-1] + 3]]).astype(np.uint64)
    mids = gen.segment_midpoints(xy, off, 2000, seed=98)
    reqs = np.concatenate([gen.density_tiles(mids, 10, 4, 16, [8, 16, 40], seed=99),
                           [[12, 2048, 2048, 16]]]).astype(np.uint32)
    t = cpu_baseline.LineTree(xy, off, threads=3)
    got, threads = t.render(reqs, STYLE)
    assert threads == 3
    assert np.array_equal(got, oracle.render_lines(xy, off, reqs, oracle.MODE_RGBA, STYLE))
    t.close()


def test_cpu_rtree_polygons_match_oracle():
    import cpu_baseline
    xy, ro, po = gen.star_polygons(1_500, seed=100, k=8, rho_median=6e-4)
    cen = gen.polygon_centres(xy, ro, po)
    reqs = gen.density_tiles(cen, 8, 3, 12, [8, 24], seed=101)
    t = cpu_baseline.PolygonTree(xy, ro, po, threads=4)
    got, _ = t.render(reqs, STYLE)
    assert np.array_equal(got, oracle.render_polygons(xy, ro, po, reqs, oracle.MODE_RGBA, STYLE))
    t.close()
