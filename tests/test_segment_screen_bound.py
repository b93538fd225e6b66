"""The single-precision screen of the segment distance test, modelled on the
CPU: every decision it takes agrees with the exact integer predicate
(distance to the closed segment <= R, Algorithm 1), and it decides almost
every case, so the exact test runs only near R.

The model follows the render kernel's steps in float32 (int64 products
rounded once, a correctly rounded square root and division, fused
multiply-adds emulated in float64 and rounded once) on inputs chosen to be
hard for it: long segments with endpoints far from the block (large
projection offsets), coordinates near the grid's edges, samples at exactly
R, R +- 1 and R +- 2 grid units, and 3-4-5 slopes.  No GPU is needed.
"""
import numpy as np

F = np.float32


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _screen(ax, ay, bx, by, ps, off, R, margin=True):
    """Per-piece parameters: (mx, my, c0, e0, D, lo2, hi2).  margin=False
    plants a mistake: no margin at all."""
    dx, dy = bx - ax, by - ay
    Ls = dx * dx + dy * dy
    mx, my, c0, e0, D = F(1), F(0), F(np.int64(ay)), F(np.int64(ax)), F(0)
    if Ls > 0:
        D = np.sqrt(F(np.int64(Ls)))
        inv = F(1) / D
        mx = F(F(np.int64(dx)) * inv)
        my = F(F(np.int64(dy)) * inv)
        c0 = F(F(np.int64(dx * ay - dy * ax)) * inv)
        e0 = F(F(np.int64(dx * ax + dy * ay)) * inv)
    fR = F(R)
    s = F(F(F(F(F(32) * F(ps)) + abs(c0)) + abs(e0)) + D)
    s = F(s + fR)
    E1 = _fma(F(2.0 ** -18), s, F(2)) if margin else F(0)
    lo, hi = F(fR - E1), F(fR + E1)
    f = 2.0 ** -20 if margin else 0.0
    lo2 = F(F(lo * lo) * F(1 - f)) if lo > 0 else F(-1)
    hi2 = F(F(hi * hi) * F(1 + f))
    return mx, my, c0, e0, D, lo2, hi2


def _decide(par, sx, sy):
    """True / False where the screen decides, None inside its margin."""
    mx, my, c0, e0, D, lo2, hi2 = par
    sx, sy = F(sx), F(sy)
    across = _fma(mx, sy, -_fma(my, sx, c0))
    along = _fma(mx, sx, _fma(my, sy, -e0))
    u = F(along - min(max(along, F(0)), D))
    q = _fma(u, u, F(across * across))
    if q < lo2:
        return True
    if q > hi2:
        return False
    return None


def _exact(ax, ay, bx, by, sx, sy, R):
    dx, dy = bx - ax, by - ay
    wx, wy = sx - ax, sy - ay
    t = wx * dx + wy * dy
    L = dx * dx + dy * dy
    if t <= 0:
        return wx * wx + wy * wy <= R * R
    if t >= L:
        ex, ey = sx - bx, sy - by
        return ex * ex + ey * ey <= R * R
    cr = wx * dy - wy * dx
    return cr * cr <= R * R * L


def _cases(rng, n):
    """(segment relative to the block, sample relative to the block, ps, off, R)."""
    half = 1 << 30
    out = []
    for _ in range(n):
        z = int(rng.integers(0, 20))
        ps = 1 << (23 - z)
        off = ps >> 2
        R = int(rng.choice([1, 8, 16, 24, 40, 1024])) << (19 - z)
        if rng.random() < 0.2:
            R = int(rng.integers(0, 1 << 20))   # a ground radius (buffer analysis)
        sx = int(rng.integers(0, 8)) * ps + int(rng.choice([-off, off, 0]))
        sy = int(rng.integers(0, 4)) * ps + int(rng.choice([-off, off, 0]))
        kind = rng.integers(0, 5)
        far = int(rng.choice([1 << 10, 1 << 20, 1 << 28, half - 1]))
        if kind == 0:       # axis-parallel at distance R + d
            d = int(rng.integers(-2, 3))
            y = sy + (R + d) * int(rng.choice([-1, 1]))
            seg = (sx - int(rng.integers(0, far)), y, sx + int(rng.integers(1, far)), y)
        elif kind == 1:     # 3-4-5 slope at distance 5k near R
            k = R // 5 + int(rng.integers(-1, 2))
            px, py = sx - 3 * k, sy + 4 * k
            t = int(rng.integers(1, max(2, far // 5)))
            seg = (px - 4 * t, py - 3 * t, px + 4 * t, py + 3 * t)
        elif kind == 2:     # an endpoint at distance R + d, the segment leading away
            d = int(rng.integers(-2, 3))
            seg = (sx + R + d, sy, sx + R + d + int(rng.integers(0, far)), sy + int(rng.integers(-far, far)))
        elif kind == 3:     # random long segment passing near the sample
            ang = rng.uniform(0, 2 * np.pi)
            dist = R + rng.normal(0, 3)
            cx, cy = sx + dist * np.cos(ang), sy + dist * np.sin(ang)
            L = rng.uniform(0, far)
            seg = (int(cx - L * np.sin(ang)), int(cy + L * np.cos(ang)),
                   int(cx + rng.uniform(0, far) * np.sin(ang)), int(cy - rng.uniform(0, far) * np.cos(ang)))
        else:               # a point (zero-length segment) at distance about R
            d = R + int(rng.integers(-2, 3))
            seg = (sx + d, sy, sx + d, sy) if rng.random() < 0.5 else (sx + 3 * (d // 5), sy + 4 * (d // 5),) * 2
        # the kernel screens only segments whose endpoints lie within 2^30 of the block
        seg = tuple(int(min(max(v, -half), half)) for v in seg)
        out.append((seg, sx, sy, ps, off, R))
    return out


def test_screen_decisions_agree_with_the_exact_test():
    rng = np.random.default_rng(2005)
    decided = agree = 0
    cases = _cases(rng, 40000)
    for (ax, ay, bx, by), sx, sy, ps, off, R in cases:
        got = _decide(_screen(ax, ay, bx, by, ps, off, R), sx, sy)
        if got is None:
            continue
        decided += 1
        assert got == _exact(ax, ay, bx, by, sx, sy, R), ((ax, ay, bx, by), sx, sy, ps, R)
        agree += 1
    # the cases sit within a few units of R on purpose: most fall inside the
    # margin and go to the exact test, some are still decided
    assert decided == agree and decided > 0.1 * len(cases)


def test_screen_decides_away_from_the_boundary():
    """Samples at least 1% of R and 16 grid units from the boundary, segments
    up to 2^20 units long: the screen decides (nearly) all of them (its
    margin is 2 units plus 2^-18 of the magnitudes involved)."""
    rng = np.random.default_rng(12489)
    n = done = 0
    for _ in range(20000):
        z = int(rng.integers(2, 20))
        ps = 1 << (23 - z)
        R = int(rng.choice([8, 16, 24, 40])) << (19 - z)
        sx, sy = int(rng.integers(0, 8)) * ps, int(rng.integers(0, 4)) * ps
        ang = rng.uniform(0, 2 * np.pi)
        dist = R * rng.choice([rng.uniform(0, 0.99), rng.uniform(1.01, 3)])
        if abs(dist - R) < max(0.01 * R, 16):
            continue
        cx, cy = sx + dist * np.cos(ang), sy + dist * np.sin(ang)
        L = rng.uniform(ps, max(2 * ps, 1 << 20))
        seg = (int(round(cx - L * np.sin(ang))), int(round(cy + L * np.cos(ang))),
               int(round(cx + L * np.sin(ang))), int(round(cy - L * np.cos(ang))))
        got = _decide(_screen(*seg, ps, ps >> 2, R), sx, sy)
        n += 1
        if got is not None:
            done += 1
            assert got == _exact(*seg, sx, sy, R)
    assert done >= 0.999 * n


def test_a_screen_without_margin_is_caught():
    """The same boundary cases with the margin removed: the screen then takes
    wrong decisions, which the exact test exposes (the cases are hard
    enough to need the margin)."""
    rng = np.random.default_rng(2005)
    wrong = 0
    for (ax, ay, bx, by), sx, sy, ps, off, R in _cases(rng, 40000):
        got = _decide(_screen(ax, ay, bx, by, ps, off, R, margin=False), sx, sy)
        if got is not None and got != _exact(ax, ay, bx, by, sx, sy, R):
            wrong += 1
    assert wrong > 0
