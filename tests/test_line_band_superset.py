"""The band filter of long segment pieces, modelled on the CPU: the pixels of
an 8 x 4 block it keeps (those whose centre lies within R + 2 off + 2 of the
line through a point near the piece, found per pixel row in single precision
with every bound widened beyond its rounding) include every pixel that has a
sample within R of the segment (Algorithm 1's closed test), so narrowing a
piece's lanes to the band never drops a covered sample.

The model follows the render kernel's float32 steps (fused multiply-adds
emulated in float64 and rounded once) on lines at every slope, near-level
and near-vertical ones included, with the reference point up to 2 units off
the line, coordinates up to 2^30 from the block, and radii from 1 unit to
2^20.  No GPU is needed.
"""
import math

import numpy as np

F = np.float32


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _band(px, py, dx, dy, L, ext, off, widen=True):
    """The pixel mask (bit 8 r + c) the kernel's band filter keeps.
    widen=False plants a mistake: half-width R only, no rounding allowance."""
    fdx, fdy, fpx, fpy = F(np.int64(dx)), F(np.int64(dy)), F(np.int64(px)), F(np.int64(py))
    dn = np.sqrt(_fma(fdx, fdx, F(fdy * fdy)))
    E = F(F(np.int64(ext + off + 2)) + F(F(abs(fpx) + abs(fpy)) * F(2.0 ** -22)))
    if not widen:
        E = F(np.int64(ext - off))
    B = F(F(E * dn) * F(1 + 2.0 ** -20)) if widen else F(E * dn)
    ps = F(1 << L)
    A = F(ps * fdy)
    inv = F(1) / A if A != 0 else F(0)
    m = 0
    for r in range(4):
        t1 = F(-fpx * fdy)
        t2 = F(_fma(F(r), ps, -fpy) * fdx)
        K = F(t1 - t2)
        mag = F(F(abs(t1) + abs(t2)) + B)
        if A == 0:
            row = 0xFF if abs(K) <= F(B + F(mag * F(2.0 ** -20))) else 0
        else:
            lo, hi = F(F(-B - K) * inv), F(F(B - K) * inv)
            if inv < 0:
                lo, hi = hi, lo
            err = F(_fma(F(mag * abs(inv)), F(2.0 ** -20), F(1)) + F(F(abs(lo) + abs(hi)) * F(2.0 ** -20)))
            if not widen:
                err = F(0)
            lo, hi = max(F(lo - err), F(-1)), min(F(hi + err), F(8))
            c0, c1 = max(math.ceil(lo), 0), min(math.floor(hi), 7)
            row = ((0xFF << c0) & (0xFF >> (7 - c1))) & 0xFF if c0 <= c1 else 0
        m |= row << (8 * r)
    return m


def _within(ax, ay, bx, by, sx, sy, R):
    dx, dy = bx - ax, by - ay
    wx, wy = sx - ax, sy - ay
    t = wx * dx + wy * dy
    L = dx * dx + dy * dy
    if t <= 0:
        return wx * wx + wy * wy <= R * R
    if t >= L:
        return (sx - bx) ** 2 + (sy - by) ** 2 <= R * R
    cr = wx * dy - wy * dx
    return cr * cr <= R * R * L


def _cases(rng, n):
    half = 1 << 30
    for _ in range(n):
        z = int(rng.integers(0, 20))
        L = 23 - z
        ps = 1 << L
        off = (ps >> 2) if rng.random() < 0.75 else 0
        R = int(rng.choice([1, 8, 16, 24, 40])) << (19 - z) if rng.random() < 0.8 else int(rng.integers(1, 1 << 20))
        # a line through a point near the block at any slope (some near level
        # or vertical), the segment reaching far on both sides
        ang = rng.uniform(0, 2 * np.pi) if rng.random() < 0.7 else rng.choice([0, np.pi / 2]) + rng.normal(0, 1e-6)
        cx = rng.uniform(-2 * ps, 9 * ps) + rng.normal(0, R + 2 * off)
        cy = rng.uniform(-2 * ps, 5 * ps) + rng.normal(0, R + 2 * off)
        far = float(rng.choice([ps, 1 << 20, 1 << 28]))
        ta, tb = rng.uniform(0, far), rng.uniform(0, far)
        ax, ay = int(round(cx - ta * np.cos(ang))), int(round(cy - ta * np.sin(ang)))
        bx, by = int(round(cx + tb * np.cos(ang))), int(round(cy + tb * np.sin(ang)))
        ax, ay, bx, by = (int(min(max(v, -half + 1), half - 1)) for v in (ax, ay, bx, by))
        if (ax, ay) == (bx, by):
            continue
        # the reference point: a point of the segment, rounded, moved by up to 1 unit
        t = rng.uniform(0, 1)
        px = int(round(ax + t * (bx - ax))) + int(rng.integers(-1, 2))
        py = int(round(ay + t * (by - ay))) + int(rng.integers(-1, 2))
        yield (ax, ay, bx, by), (px, py), L, ps, off, R


def _covered_pixels(seg, ps, off, R):
    ax, ay, bx, by = seg
    for r in range(4):
        for c in range(8):
            samples = [(c * ps, r * ps)] if off == 0 else [
                (c * ps + ox, r * ps + oy) for ox in (-off, off) for oy in (-off, off)]
            if any(_within(ax, ay, bx, by, sx, sy, R) for sx, sy in samples):
                yield r, c


def test_band_keeps_every_covered_pixel():
    covered = 0
    for seg, (px, py), L, ps, off, R in _cases(np.random.default_rng(5012489), 3000):
        band = _band(px, py, seg[2] - seg[0], seg[3] - seg[1], L, R + off, off)
        for r, c in _covered_pixels(seg, ps, off, R):
            covered += 1
            assert (band >> (8 * r + c)) & 1, (R, off, seg, (px, py), r, c)
    assert covered > 1000


def test_a_band_without_widening_is_caught():
    """Half-width R and no rounding allowance drops covered pixels (samples
    off the pixel centre, the reference point off the line)."""
    dropped = 0
    for seg, (px, py), L, ps, off, R in _cases(np.random.default_rng(5012489), 3000):
        band = _band(px, py, seg[2] - seg[0], seg[3] - seg[1], L, R + off, off, widen=False)
        dropped += sum(1 for r, c in _covered_pixels(seg, ps, off, R) if not (band >> (8 * r + c)) & 1)
    assert dropped > 0
