"""The synthetic inputs follow their stated recipes (shapes, counts, ranges,
simple polygons, valid tiles) and are reproducible from their seeds."""
import numpy as np

from workloads import gen

HALF = 1 << 30


def test_points_in_grid_and_seeded():
    a = gen.gmm_points(200_000, seed=7, k=16)
    b = gen.gmm_points(200_000, seed=7, k=16)
    assert a.dtype == np.int32 and a.shape == (200_000, 2)
    assert np.array_equal(a, b)
    assert a.min() >= -HALF and a.max() <= HALF - 1
    # the mixture is clustered: far fewer distinct 2^20-unit cells than a uniform draw would fill
    cells = np.unique((a.astype(np.int64) + HALF) >> 20, axis=0).shape[0]
    u = gen.uniform_points(200_000, seed=7)
    ucells = np.unique((u.astype(np.int64) + HALF) >> 20, axis=0).shape[0]
    assert cells < ucells / 2


def test_walk_lines_exact_segment_count():
    xy, off = gen.walk_lines(1_000, 9_000, seed=8, n_cities=20)
    nv = np.diff(off.astype(np.int64))
    assert off[0] == 0 and off[-1] == xy.shape[0]
    assert (nv >= 2).all() and int((nv - 1).sum()) == 9_000        # every line has >= 1 segment
    assert xy.min() >= -HALF and xy.max() <= HALF - 1


def _orient(a, b, c):
    v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (v > 0) - (v < 0)


def _on_segment(a, b, c):
    return min(a[0], b[0]) <= c[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= c[1] <= max(a[1], b[1])


def _segments_meet(a, b, c, d):
    o1, o2, o3, o4 = _orient(a, b, c), _orient(a, b, d), _orient(c, d, a), _orient(c, d, b)
    if o1 != o2 and o3 != o4:
        return True
    return ((o1 == 0 and _on_segment(a, b, c)) or (o2 == 0 and _on_segment(a, b, d)) or
            (o3 == 0 and _on_segment(c, d, a)) or (o4 == 0 and _on_segment(c, d, b)))


def test_star_polygons_are_simple():
    xy, ro, po = gen.star_polygons(300, seed=9, k=8, rho_median=6e-4)
    assert len(po) == 301 and np.array_equal(po, np.arange(301))       # one ring per polygon
    nv = np.diff(ro.astype(np.int64))
    assert nv.min() >= 8 and nv.max() <= 64
    assert xy.min() >= -HALF and xy.max() <= HALF - 1
    for p in range(0, 300, 10):
        v = [tuple(int(c) for c in q) for q in xy[int(ro[p]):int(ro[p + 1])]]
        n = len(v)
        edges = [(v[i], v[(i + 1) % n]) for i in range(n)]
        for i in range(n):
            for j in range(i + 2, n):
                if i == 0 and j == n - 1:
                    continue                     # adjacent through the closing vertex
                assert not _segments_meet(*edges[i], *edges[j]), (p, i, j)


def test_density_tiles_valid():
    pts = gen.gmm_points(50_000, seed=10, k=8)
    t = gen.density_tiles(pts, 5_000, 8, 14, [8, 32], seed=11)
    z, x, y, r = t[:, 0].astype(np.int64), t[:, 1].astype(np.int64), t[:, 2].astype(np.int64), t[:, 3]
    assert z.min() >= 8 and z.max() <= 14 and set(np.unique(r)) <= {8, 32}
    assert (x < (1 << z)).all() and (y < (1 << z)).all()
    # every tile contains an object of the layer (density weighted)
    k = np.random.default_rng(0).integers(0, len(t), 50)
    for i in k:
        span = 1 << (31 - int(z[i]))
        x0 = -HALF + int(x[i]) * span
        y0 = -HALF + int(y[i]) * span
        inside = ((pts[:, 0] >= x0) & (pts[:, 0] < x0 + span) & (pts[:, 1] >= y0) & (pts[:, 1] < y0 + span))
        assert inside.any()


def test_shards_partition_the_batch():
    rows = np.arange(103)
    parts = [gen.shard(rows, r, 4) for r in range(4)]
    assert np.array_equal(np.sort(np.concatenate(parts)), rows)
