"""Bucket grids that find the objects of a huge layer near a small box.

Test infrastructure for checking windows of tiles of billion-object layers
against the oracle: the oracle makes a pass over every object it is given,
so a window is checked by giving it only the objects whose bounding box meets
the window's box widened by the largest distance at which an object can still
cover one of the window's samples.  Every such object is returned (the
filter is an exact box-intersection test), so the oracle's values on the
window equal its values over the whole layer.

Objects are bucketed by the cell of a 1024 x 1024 grid (2^21 units) holding
their (box-centre) point, in chunks, each chunk sorted by cell with two
stable 16-bit radix passes.  Segments longer than a cell are kept aside and
searched in full.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HALF = 1 << 30
CELL_BITS = 21
NC = 1 << (31 - CELL_BITS)      # cells per axis (1024)
CHUNK = 1 << 26


def _cell(v):
    return ((np.asarray(v, dtype=np.int64) + HALF) >> CELL_BITS).clip(0, NC - 1)


def _sort_by_cell(key):
    """Stable permutation sorting 20-bit keys (two 16-bit radix passes)."""
    lo = (key & 0xFFFF).astype(np.uint16)
    o1 = np.argsort(lo, kind="stable")
    del lo
    hi = (key[o1] >> 16).astype(np.uint16)
    o2 = np.argsort(hi, kind="stable")
    return o1[o2]


class _Buckets:
    """Records grouped by cell, chunk by chunk."""

    def __init__(self, records, cx, cy, threads=16):
        n = records.shape[0]

        def one(s):
            e = min(n, s + CHUNK)
            key = (cx[s:e].astype(np.uint32) << 10) | cy[s:e].astype(np.uint32)
            order = _sort_by_cell(key)
            cnt = np.bincount(key, minlength=NC * NC)
            starts = np.zeros(NC * NC + 1, dtype=np.int64)
            np.cumsum(cnt, out=starts[1:])
            return records[s:e][order], starts, cnt

        # numpy's sorts and gathers release the GIL: chunks run side by side
        with ThreadPoolExecutor(max_workers=threads) as ex:
            done = list(ex.map(one, range(0, n, CHUNK)))
        self.chunks = [(r, st) for r, st, _ in done]
        self.counts = np.zeros((NC, NC), dtype=np.int64)
        for _, _, cnt in done:
            self.counts += cnt.reshape(NC, NC)
        # summed-area table for quick upper bounds of box populations
        self.sat = np.zeros((NC + 1, NC + 1), dtype=np.int64)
        self.sat[1:, 1:] = self.counts.cumsum(0).cumsum(1)

    def _cells(self, x0, y0, x1, y1):
        return int(_cell(x0)), int(_cell(y0)), int(_cell(x1)), int(_cell(y1))

    def upper_count(self, x0, y0, x1, y1):
        a, b, c, d = self._cells(x0, y0, x1, y1)
        s = self.sat
        return int(s[c + 1, d + 1] - s[a, d + 1] - s[c + 1, b] + s[a, b])

    def gather(self, x0, y0, x1, y1):
        a, b, c, d = self._cells(x0, y0, x1, y1)
        parts = []
        for recs, starts in self.chunks:
            for cx in range(a, c + 1):
                lo, hi = starts[cx * NC + b], starts[cx * NC + d + 1]
                if hi > lo:
                    parts.append(recs[lo:hi])
        if not parts:
            return None
        return np.concatenate(parts)


class PointGrid:
    """Points (n, 2) int32."""

    def __init__(self, xy):
        self.b = _Buckets(xy, _cell(xy[:, 0]), _cell(xy[:, 1]))

    def upper_count(self, x0, y0, x1, y1):
        return self.b.upper_count(x0, y0, x1, y1)

    def query(self, x0, y0, x1, y1):
        """Every point in [x0, x1] x [y0, y1] (inclusive)."""
        p = self.b.gather(x0, y0, x1, y1)
        if p is None:
            return np.zeros((0, 2), dtype=np.int32)
        x, y = p[:, 0], p[:, 1]
        return p[(x >= x0) & (x <= x1) & (y >= y0) & (y <= y1)]


class SegmentGrid:
    """Segments (n, 4) int32 rows (ax, ay, bx, by)."""

    def __init__(self, segs):
        a = segs.astype(np.int64)
        ext = np.maximum(np.abs(a[:, 2] - a[:, 0]), np.abs(a[:, 3] - a[:, 1]))
        short = ext <= (1 << CELL_BITS)
        self.long = segs[~short]
        s = segs[short]
        a = a[short]
        # a short segment meeting a box has its midpoint within half its
        # extent (at most 2^20 units) of the box
        self.reach = (1 << (CELL_BITS - 1)) + 1
        self.b = _Buckets(s, _cell((a[:, 0] + a[:, 2]) >> 1), _cell((a[:, 1] + a[:, 3]) >> 1))

    def upper_count(self, x0, y0, x1, y1):
        r = self.reach
        return self.b.upper_count(x0 - r, y0 - r, x1 + r, y1 + r) + len(self.long)

    @staticmethod
    def _meets(s, x0, y0, x1, y1):
        s = s.astype(np.int64)
        mnx, mxx = np.minimum(s[:, 0], s[:, 2]), np.maximum(s[:, 0], s[:, 2])
        mny, mxy = np.minimum(s[:, 1], s[:, 3]), np.maximum(s[:, 1], s[:, 3])
        return (mnx <= x1) & (mxx >= x0) & (mny <= y1) & (mxy >= y0)

    def query(self, x0, y0, x1, y1):
        """Every segment whose bounding box meets [x0, x1] x [y0, y1]."""
        r = self.reach
        near = self.b.gather(x0 - r, y0 - r, x1 + r, y1 + r)
        parts = [self.long[self._meets(self.long, x0, y0, x1, y1)]]
        if near is not None:
            parts.append(near[self._meets(near, x0, y0, x1, y1)])
        return np.concatenate(parts)


def segments_of_lines(xy, line_off):
    """The segments (n, 4) of polylines (a line with k vertices has k - 1)."""
    off = np.asarray(line_off, dtype=np.int64)
    nseg = np.maximum(off[1:] - off[:-1] - 1, 0)
    total = int(nseg.sum())
    first = np.zeros(len(nseg), dtype=np.int64)
    np.cumsum(nseg[:-1], out=first[1:])
    starts = np.repeat(off[:-1], nseg) + (np.arange(total, dtype=np.int64) - np.repeat(first, nseg))
    return np.concatenate([xy[starts], xy[starts + 1]], axis=1)
