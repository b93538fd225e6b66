"""The bucket grids used to pick a window's objects out of a huge layer
return exactly the objects a brute-force box test keeps, and their cell
counts bound the populations from above (no GPU)."""
import numpy as np

import cellgrid
from cellgrid import PointGrid, SegmentGrid, segments_of_lines
from workloads import gen


def test_segments_of_lines_brute():
    xy, off = gen.walk_lines(300, 2_000, seed=3, n_cities=5)
    xy = np.concatenate([xy, [[7, 8]]]).astype(np.int32)          # a one-vertex line
    off = np.concatenate([off, [off[-1] + 1]]).astype(np.uint64)
    want = [list(xy[v]) + list(xy[v + 1]) for l in range(len(off) - 1)
            for v in range(int(off[l]), int(off[l + 1]) - 1)]
    assert np.array_equal(segments_of_lines(xy, off), np.array(want, dtype=np.int32))


def test_grid_queries_equal_brute_force(monkeypatch):
    monkeypatch.setattr(cellgrid, "CHUNK", 1 << 16)                # several chunks
    rng = np.random.default_rng(1)
    pts = np.concatenate([gen.gmm_points(200_000, seed=4, k=8),
                          np.array([[-(1 << 30), -(1 << 30)], [(1 << 30) - 1, (1 << 30) - 1]], np.int32)])
    xy, off = gen.walk_lines(5_000, 60_000, seed=5, n_cities=10, step_mean=3e-3)
    segs = segments_of_lines(xy, off)
    pg, sg = PointGrid(pts), SegmentGrid(segs)
    assert len(sg.long) > 0
    p64, s64 = pts.astype(np.int64), segs.astype(np.int64)
    for k in range(40):
        c = (pts[rng.integers(len(pts))] if k % 2 else segs[rng.integers(len(segs)), :2]).astype(np.int64)
        w = int(2 ** rng.uniform(0, 28))
        box = (c[0] - w, c[1] - w, c[0] + w, c[1] + 3 * w)
        x0, y0, x1, y1 = box
        inside = (p64[:, 0] >= x0) & (p64[:, 0] <= x1) & (p64[:, 1] >= y0) & (p64[:, 1] <= y1)
        q = pg.query(*box)
        assert sorted(map(tuple, q)) == sorted(map(tuple, pts[inside]))
        assert pg.upper_count(*box) >= len(q)
        meets = ((np.minimum(s64[:, 0], s64[:, 2]) <= x1) & (np.maximum(s64[:, 0], s64[:, 2]) >= x0) &
                 (np.minimum(s64[:, 1], s64[:, 3]) <= y1) & (np.maximum(s64[:, 1], s64[:, 3]) >= y0))
        qs = sg.query(*box)
        assert sorted(map(tuple, qs)) == sorted(map(tuple, segs[meets]))
        assert sg.upper_count(*box) >= len(qs)
