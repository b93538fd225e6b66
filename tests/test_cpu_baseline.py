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
