"""The render kernel's integer shortcuts, modelled on the CPU against the
plain definitions they stand in for (Algorithm 1's closed distance test,
Algorithm 2's half-open ray crossing):

* the Chebyshev lane mask of a box is a necessary condition: every lane with
  a sample within R of some point of the box is in it;
* the certain cover of a box of points (Chebyshev distance q = floor(R/sqrt 2)
  from all of the box) marks only samples that every point of the box covers;
* squared distances of samples in a point's Chebyshev reach, and the
  box-to-sample gaps of the point kernel's node tests, are exact in unsigned
  32-bit arithmetic when R + 2 off <= 46,340;
* the crossed columns of an edge per pixel row, found by a three-step search
  over exact products, are the columns whose centre the edge crosses
  strictly to the right (half-open in y);
* a segment leaf's staging of (piece, pixel) pairs takes every pair exactly
  once over its rounds.

Each model follows the kernel's steps (shifts by the pixel size, clamps to
+-2^30, 32-bit wrap-around) in Python integers.  No GPU is needed.
"""
import math

import numpy as np

HALF = 1 << 30


def _sar(v, s):
    """Arithmetic right shift of a (signed 32-bit) int."""
    return v >> s


def rect_lanes(bx0, by0, L, ext, x0, y0, x1, y1):
    """Lanes (bit 8 r + c) whose pixel centre lies within Chebyshev distance
    ext of the box, as the kernel computes them."""
    if x0 > x1 or y0 > y1 or x0 < -HALF or y0 < -HALF:
        return 0
    ax = max(x0 - bx0, -HALF) - ext
    bx = min(x1 - bx0, HALF) + ext
    ay = max(y0 - by0, -HALF) - ext
    by = min(y1 - by0, HALF) + ext
    c0, c1 = max(-_sar(-ax, L), 0), min(_sar(bx, L), 7)
    r0, r1 = max(-_sar(-ay, L), 0), min(_sar(by, L), 3)
    if c0 > c1 or r0 > r1:
        return 0
    col = (0xFF << c0) & (0xFF >> (7 - c1))
    rows = (0x01010101 << (8 * r0)) & (0x01010101 >> (8 * (3 - r1)))
    return (col * rows) & 0xFFFFFFFF


def certain_lanes(bx0, by0, L, off, q, x0, y0, x1, y1):
    """Per sample k (bit 0: +x, bit 1: +y), the lanes whose sample k lies in
    [x1 - q, x0 + q] x [y1 - q, y0 + q]."""
    m = [0, 0, 0, 0]
    if x0 > x1 or y0 > y1 or x0 < -HALF or y0 < -HALF:
        return m
    lx, hx = max(x1 - bx0, -HALF) - q, min(x0 - bx0, HALF) + q
    ly, hy = max(y1 - by0, -HALF) - q, min(y0 - by0, HALF) + q
    if lx > hx or ly > hy:
        return m
    col, row = [0, 0], [0, 0]
    for k in range(2):
        o = -off if k else off
        c0, c1 = max(-_sar(-(lx + o), L), 0), min(_sar(hx + o, L), 7)
        r0, r1 = max(-_sar(-(ly + o), L), 0), min(_sar(hy + o, L), 3)
        col[k] = 0 if c0 > c1 else (0xFF << c0) & (0xFF >> (7 - c1))
        row[k] = 0 if r0 > r1 else (0x01010101 << (8 * r0)) & (0x01010101 >> (8 * (3 - r1)))
    for k in range(4):
        m[k] = (col[k & 1] * row[k >> 1]) & 0xFFFFFFFF
    return m


def _sample(bx0, by0, L, off, lane, k):
    c, r = lane & 7, lane >> 3
    return (bx0 + (c << L) + (off if k & 1 else -off), by0 + (r << L) + (off if k & 2 else -off))


def _box_dist2(x0, y0, x1, y1, sx, sy):
    gx = max(x0 - sx, sx - x1, 0)
    gy = max(y0 - sy, sy - y1, 0)
    return gx * gx + gy * gy


def _far_dist2(x0, y0, x1, y1, sx, sy):
    gx = max(abs(sx - x0), abs(sx - x1))
    gy = max(abs(sy - y0), abs(sy - y1))
    return gx * gx + gy * gy


def _block(rng):
    z = int(rng.integers(0, 20))
    L = 23 - z
    ps = 1 << L
    off = (ps >> 2) if rng.random() < 0.75 else 0
    R = (int(rng.choice([1, 8, 16, 24, 32, 40, 1024])) << (19 - z)) if rng.random() < 0.8 else int(rng.integers(0, 1 << 24))
    bx0 = int(rng.integers(-HALF, HALF - 8 * ps)) // ps * ps + ps // 2
    by0 = int(rng.integers(-HALF, HALF - 4 * ps)) // ps * ps + ps // 2
    return L, ps, off, R, bx0, by0


def _box_near(rng, bx0, by0, ps, R, off):
    span = R + 2 * off + 9 * ps
    cx = bx0 + int(rng.integers(-span, span + 1))
    cy = by0 + int(rng.integers(-span, span + 1))
    w = int(rng.choice([0, 1, ps // 3 + 1, ps, 4 * ps, 64 * ps]))
    h = int(rng.choice([0, 1, ps // 3 + 1, ps, 4 * ps]))
    x0 = min(max(cx - int(rng.integers(0, w + 1)), -HALF), HALF - 1)
    y0 = min(max(cy - int(rng.integers(0, h + 1)), -HALF), HALF - 1)
    return x0, y0, min(x0 + w, HALF - 1), min(y0 + h, HALF - 1)


def test_chebyshev_lanes_are_necessary():
    rng = np.random.default_rng(11)
    reached = 0
    for _ in range(4000):
        L, ps, off, R, bx0, by0 = _block(rng)
        x0, y0, x1, y1 = _box_near(rng, bx0, by0, ps, R, off)
        m = rect_lanes(bx0, by0, L, R + off, x0, y0, x1, y1)
        for lane in range(32):
            for k in range(4 if off else 1):
                sx, sy = _sample(bx0, by0, L, off, lane, k)
                if _box_dist2(x0, y0, x1, y1, sx, sy) <= R * R:
                    reached += 1
                    assert (m >> lane) & 1, (L, off, R, (x0, y0, x1, y1), lane, k)
    assert reached > 1000


def _certain_box(rng, bx0, by0, L, ps, off, R, q):
    """Half the boxes random near the block, half with their far corner at
    Chebyshev distance q - 1, q or q + 1 from a sample along each axis."""
    if rng.random() < 0.5:
        return _box_near(rng, bx0, by0, ps, max(R // 4, 1), off)
    lane, k = int(rng.integers(0, 32)), int(rng.integers(0, 4 if off else 1))
    sx, sy = _sample(bx0, by0, L, off, lane, k)
    d = max(q + int(rng.integers(-1, 2)), 0)
    w, h = int(rng.integers(0, d + 1)), int(rng.integers(0, d + 1))
    fx, fy = int(rng.choice([-1, 1])), int(rng.choice([-1, 1]))
    # far corner at (sx + fx d, sy + fy d), the box extending back towards s
    xa, xb = sorted((sx + fx * d, sx + fx * (d - w)))
    ya, yb = sorted((sy + fy * d, sy + fy * (d - h)))
    return tuple(min(max(v, -HALF), HALF - 1) for v in (xa, ya, xb, yb))


def test_certain_cover_marks_only_covered_samples():
    rng = np.random.default_rng(12)
    marked = 0
    for _ in range(6000):
        L, ps, off, R, bx0, by0 = _block(rng)
        q = math.isqrt(R * R // 2)
        assert 2 * q * q <= R * R < 2 * (q + 1) * (q + 1)
        x0, y0, x1, y1 = _certain_box(rng, bx0, by0, L, ps, off, R, q)
        m = certain_lanes(bx0, by0, L, off, q, x0, y0, x1, y1)
        for k in range(4 if off else 1):
            for lane in range(32):
                if (m[k] >> lane) & 1:
                    marked += 1
                    sx, sy = _sample(bx0, by0, L, off, lane, k)
                    # the farthest point of the box (a corner) is within R
                    assert _far_dist2(x0, y0, x1, y1, sx, sy) <= R * R, (L, off, R, (x0, y0, x1, y1), lane, k)
    assert marked > 1000


def test_narrow_squares_are_exact_in_32_bits():
    """Samples in a point's Chebyshev reach: |d -+ off| <= R + 2 off, so under
    R + 2 off <= 46,340 each square is below 2^31 and a sum of two below
    2^32; the 32-bit results equal the exact ones, also at the limit."""
    rng = np.random.default_rng(13)
    M = (1 << 32) - 1
    for _ in range(20000):
        z = int(rng.integers(9, 20))
        L = 23 - z
        ps = 1 << L
        off = ps >> 2
        R = int(rng.integers(0, 46340 - 2 * off + 1))
        ext = R + off
        # a point and a lane with the pixel centre within ext of it along each axis
        dx = int(rng.integers(-ext, ext + 1)) if rng.random() < 0.9 else int(rng.choice([-ext, ext]))
        dy = int(rng.integers(-ext, ext + 1)) if rng.random() < 0.9 else int(rng.choice([-ext, ext]))
        for sgn_x in (1, -1):
            for sgn_y in (1, -1):
                ex, ey = dx + sgn_x * off, dy + sgn_y * off
                assert abs(ex) <= R + 2 * off <= 46340 and abs(ey) <= 46340
                xs, ys = (ex * ex) & M, (ey * ey) & M
                assert xs < (1 << 31) and ys < (1 << 31)
                assert ((xs + ys) & M) == ex * ex + ey * ey
                assert (((xs + ys) & M) <= ((R * R) & M)) == (ex * ex + ey * ey <= R * R)
    # the bound is tight: 46,341 would overflow a signed square
    assert 46340 * 46340 < (1 << 31) <= 46341 * 46341


def crossing_columns(ex0, ey0, ex1, ey1, bx0, by0, L, ox=0, oy=0):
    """The kernel's per-row prefix of crossed columns (bit 8 r + c)."""
    lx, ly, hx, hy = ex0, ey0, ex1, ey1
    if ly > hy:
        lx, ly, hx, hy = ex1, ey1, ex0, ey0
    if ly == hy:
        return 0
    dx, dy = hx - lx, hy - ly
    m = 0
    for r in range(4):
        y = by0 + (r << L) + oy
        if y < ly or y >= hy:
            continue
        n0 = dx * (y - ly) - (bx0 + ox - lx) * dy
        t = 4 if n0 > (3 << L) * dy else 0
        if n0 > ((t + 1) << L) * dy:
            t += 2
        if n0 > (t << L) * dy:
            t += 1
        if t == 7 and n0 > (7 << L) * dy:
            t = 8
        m |= ((1 << t) - 1) << (8 * r)
    return m


def _crosses_right(ax, ay, bx, by, cx, cy):
    """Algorithm 2's test: the edge straddles y = cy half-open and crosses the
    horizontal ray from (cx, cy) strictly to the right."""
    if (ay > cy) == (by > cy):
        return False
    lx, ly, hx, hy = (ax, ay, bx, by) if ay < by else (bx, by, ax, ay)
    return (hx - lx) * (cy - ly) - (cx - lx) * (hy - ly) > 0


def test_crossing_columns_equal_the_ray_test():
    rng = np.random.default_rng(14)
    crossed = 0
    for _ in range(5000):
        z = int(rng.integers(0, 20))
        L = 23 - z
        ps = 1 << L
        bx0 = int(rng.integers(-HALF, HALF - 8 * ps)) // ps * ps + ps // 2
        by0 = int(rng.integers(-HALF, HALF - 4 * ps)) // ps * ps + ps // 2
        off = (ps >> 2) * int(rng.choice([0, 1]))
        ox, oy = int(rng.choice([-off, off])), int(rng.choice([-off, off]))
        # edges through the block at every slope, endpoints on sample rows, far away, or level
        far = int(rng.choice([ps, 16 * ps, 1 << 28]))
        pts = []
        for _e in range(2):
            px = bx0 + int(rng.integers(-2 * ps, 10 * ps))
            py = by0 + (int(rng.integers(-1, 5)) << L) + oy if rng.random() < 0.3 else by0 + int(rng.integers(-far, far))
            pts.append((min(max(px, -HALF), HALF - 1), min(max(py, -HALF), HALF - 1)))
        (ax, ay), (bx, by) = pts
        if rng.random() < 0.1:
            by = ay
        m = crossing_columns(ax, ay, bx, by, bx0, by0, L, ox, oy)
        for r in range(4):
            for c in range(8):
                want = _crosses_right(ax, ay, bx, by, bx0 + (c << L) + ox, by0 + (r << L) + oy)
                crossed += want
                assert bool((m >> (8 * r + c)) & 1) == want, ((ax, ay, bx, by), L, r, c, ox, oy)
    assert crossed > 1000


def test_planted_mistakes_are_caught():
    """Each check above fails for a plausible slip: a certain-cover half-side
    one unit too large, a Chebyshev reach without the super-sample offset,
    and a crossing search that also counts a crossing through the centre."""
    rng = np.random.default_rng(15)
    bad_q = bad_ext = 0
    for _ in range(6000):
        L, ps, off, R, bx0, by0 = _block(rng)
        q = math.isqrt(R * R // 2) + 1   # planted: 2 q^2 > R^2
        x0, y0, x1, y1 = _certain_box(rng, bx0, by0, L, ps, off, R, q)
        m = certain_lanes(bx0, by0, L, off, q, x0, y0, x1, y1)
        mr = rect_lanes(bx0, by0, L, R, x0, y0, x1, y1)   # planted: reach R, not R + off
        for k in range(4 if off else 1):
            for lane in range(32):
                sx, sy = _sample(bx0, by0, L, off, lane, k)
                if (m[k] >> lane) & 1 and _far_dist2(x0, y0, x1, y1, sx, sy) > R * R:
                    bad_q += 1
                if _box_dist2(x0, y0, x1, y1, sx, sy) <= R * R and not (mr >> lane) & 1:
                    bad_ext += 1
    assert bad_q > 0
    assert bad_ext > 0
    # a crossing through the sample itself (n0 == c ps dy) counted as crossed
    bad_tie = 0
    for _ in range(3000):
        L = int(rng.integers(0, 24))
        ps = 1 << L
        bx0, by0 = 0, 0
        c, r = int(rng.integers(0, 8)), int(rng.integers(0, 4))
        # an edge through the pixel centre (c, r): x = c ps exactly on row r
        dy = int(rng.integers(1, 50)) * ps
        dx = int(rng.integers(-50, 50)) * ps
        ax, ay = c * ps - dx, r * ps - dy
        bx, by = c * ps + dx, r * ps + dy
        m = crossing_columns(ax, ay, bx, by, bx0, by0, L)
        counted_with_ge = sum(1 for cc in range(8)
                              if (bx - ax) * (r * ps - ay) - (cc * ps - ax) * (by - ay) >= 0)
        if counted_with_ge != bin((m >> (8 * r)) & 0xFF).count("1"):
            bad_tie += 1
    assert bad_tie > 0


def test_narrow_box_reach_equals_the_exact_gap_test():
    """The node and frontier reach test of the point kernel in unsigned 32-bit
    arithmetic: for the lanes in a box's Chebyshev reach, gaps are at most
    R + 2 off, so under R + 2 off <= 46,340 the 32-bit test equals the exact
    box-to-sample test (Algorithm 1's distance <= R, to the nearest point of
    the box)."""
    rng = np.random.default_rng(16)
    M = (1 << 32) - 1
    checked = 0
    for _ in range(3000):
        z = int(rng.integers(9, 20))
        L = 23 - z
        ps = 1 << L
        off = (ps >> 2) if rng.random() < 0.75 else 0
        R = int(rng.integers(0, 46340 - 2 * off + 1))
        bx0 = int(rng.integers(-HALF, HALF - 8 * ps)) // ps * ps + ps // 2
        by0 = int(rng.integers(-HALF, HALF - 4 * ps)) // ps * ps + ps // 2
        x0, y0, x1, y1 = _box_near(rng, bx0, by0, ps, R, off)
        cand = rect_lanes(bx0, by0, L, R + off, x0, y0, x1, y1)
        ax = max(min(x0 - bx0, HALF), -HALF)
        bx = max(min(x1 - bx0, HALF), -HALF)
        ay = max(min(y0 - by0, HALF), -HALF)
        by = max(min(y1 - by0, HALF), -HALF)
        for lane in range(32):
            if not (cand >> lane) & 1:
                continue
            sx, sy = (lane & 7) << L, (lane >> 3) << L
            for k in range(4 if off else 1):
                px = sx + (off if k & 1 else -off)
                py = sy + (off if k & 2 else -off)
                gx = max(ax - px, px - bx, 0)
                gy = max(ay - py, py - by, 0)
                assert gx <= R + 2 * off and gy <= R + 2 * off
                narrow = ((gx * gx + gy * gy) & M) <= ((R * R) & M)
                exact = _box_dist2(x0, y0, x1, y1, bx0 + px, by0 + py) <= R * R
                assert narrow == exact, (L, off, R, (x0, y0, x1, y1), lane, k)
                checked += 1
    assert checked > 1000


def stage_pairs(pm, cap=128):
    """The segment leaf's staging of (piece, pixel) pairs: lane p's pairs are
    numbered from the exclusive prefix sum of the lanes' pixel counts; each
    round writes the pairs numbered [w0, w0 + cap) (unsigned wrap-around
    skips the earlier ones) and the warp then takes them in turn."""
    cnt = [bin(m).count("1") for m in pm]
    first = [sum(cnt[:p]) for p in range(32)]
    total = sum(cnt)
    rounds = []
    w0 = 0
    while w0 < total:
        slots = [None] * cap
        for p in range(32):
            m, g = pm[p], (first[p] - w0) & 0xFFFFFFFF
            while m:
                low = m & -m
                lane = low.bit_length() - 1
                m &= m - 1
                if g < cap:
                    assert slots[g] is None
                    slots[g] = (p << 5) | lane
                g = (g + 1) & 0xFFFFFFFF
        n = min(total - w0, cap)
        assert all(v is not None for v in slots[:n]) and all(v is None for v in slots[n:])
        rounds.append(slots[:n])
        w0 += cap
    return rounds


def test_pair_staging_takes_every_pair_once():
    """Up to 32 x 32 pairs per leaf, so up to 8 rounds of 128."""
    rng = np.random.default_rng(17)
    for _ in range(500):
        density = rng.choice([0.02, 0.2, 0.5, 1.0])
        pm = [int(sum(1 << b for b in range(32) if rng.random() < density)) for _ in range(32)]
        rounds = stage_pairs(pm)
        got = sorted(e for r in rounds for e in r)
        want = sorted((p << 5) | b for p in range(32) for b in range(32) if (pm[p] >> b) & 1)
        assert got == want
        assert len(rounds) == -(-len(want) // 128)
