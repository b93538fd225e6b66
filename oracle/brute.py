"""Pixel-driven brute force in pure Python (second, independent oracle).

TEST INFRASTRUCTURE ONLY.  For tiny layers and small pixel windows it
evaluates, for every sample of every pixel in the window, every object of the
layer with exact rational arithmetic (Python ``int`` and ``fractions``),
following HiVision Sec. 3.2 directly: a pixel is the computing unit and its
value is decided by the objects near it (Algorithm 1), and a pixel centre is
inside a polygon when that polygon's own edges cross the ray from it an odd
number of times (Algorithm 2).

It is written independently of ``hv_oracle.c`` (different formulas: the
nearest point of a segment is found by clamping the projection parameter as a
fraction, the fill crossing is located as a rational x coordinate) so that
agreement between the two pins both.
"""
from fractions import Fraction

TILE = 256
GRID_HALF = 1 << 30


def pixel_centre(z, tx, ty, i, j):
    """Centre of pixel (i, j) of tile (z, tx, ty) in grid units (y southward)."""
    ps = 1 << (23 - z)
    return (-GRID_HALF + tx * (1 << (31 - z)) + i * ps + ps // 2,
            -GRID_HALF + ty * (1 << (31 - z)) + j * ps + ps // 2)


def samples(z, tx, ty, i, j):
    """(centre, [NW, NE, SW, SE]) super-samples at +-ps/4 (Algorithm 1, P1..P4)."""
    cx, cy = pixel_centre(z, tx, ty, i, j)
    q = (1 << (23 - z)) // 4
    return (cx, cy), [(cx - q, cy - q), (cx + q, cy - q), (cx - q, cy + q), (cx + q, cy + q)]


def _dist2_point(p, s):
    return (p[0] - s[0]) ** 2 + (p[1] - s[1]) ** 2


def _dist2_segment(a, b, s):
    dx, dy = b[0] - a[0], b[1] - a[1]
    L = dx * dx + dy * dy
    if L == 0:
        return Fraction(_dist2_point(a, s))
    t = Fraction((s[0] - a[0]) * dx + (s[1] - a[1]) * dy, L)
    t = min(max(t, Fraction(0)), Fraction(1))
    px, py = a[0] + t * dx, a[1] + t * dy
    return (px - s[0]) ** 2 + (py - s[1]) ** 2


def _inside(rings, c):
    """Odd number of this polygon's edges cross the ray from c towards +x."""
    cnt = 0
    for ring in rings:
        n = len(ring)
        for k in range(n):
            a, b = ring[k], ring[(k + 1) % n]
            if (a[1] > c[1]) == (b[1] > c[1]):
                continue  # no half-open straddle (level edges never straddle)
            xc = a[0] + Fraction((b[0] - a[0]) * (c[1] - a[1]), b[1] - a[1])
            if xc > c[0]:
                cnt += 1
    return cnt % 2 == 1


def segments_of_lines(lines):
    segs = []
    for line in lines:
        for k in range(len(line) - 1):
            segs.append((tuple(line[k]), tuple(line[k + 1])))
    return segs


def edges_of_polygons(polys):
    segs = []
    for rings in polys:
        for ring in rings:
            n = len(ring)
            for k in range(n):
                segs.append((tuple(ring[k]), tuple(ring[(k + 1) % n])))
    return segs


def pixel_flags(kind, layer, z, tx, ty, r16, i, j, R=None):
    """Return (centre_hit, [4 sub-sample hits], fill) for one pixel.

    kind: 'points' (layer = [(x, y)]), 'lines' (layer = [[(x, y), ...]]),
    'polygons' (layer = [[ring, ...]] with ring = [(x, y), ...]).  The radius
    is r16 sixteenths of a pixel, or R grid units when R is given (a buffer
    distance on the ground)."""
    if R is None:
        R = r16 << (19 - z)
    R2 = R * R
    c, subs = samples(z, tx, ty, i, j)
    if kind == "points":
        def hit(s):
            return any(_dist2_point(p, s) <= R2 for p in layer)
    else:
        segs = segments_of_lines(layer) if kind == "lines" else edges_of_polygons(layer)

        def hit(s):
            return any(_dist2_segment(a, b, s) <= R2 for a, b in segs)
    fill = kind == "polygons" and any(_inside(rings, c) for rings in layer)
    return hit(c), [hit(s) for s in subs], fill


def fill_samples(layer, z, tx, ty, i, j):
    """The four super-samples of a pixel inside some polygon (anti-aliased fill)."""
    _, subs = samples(z, tx, ty, i, j)
    return [any(_inside(rings, s) for rings in layer) for s in subs]


def encode_pixel(mode, centre, subs, fill, style):
    """Bytes of one pixel in COVERAGE (1) or RGBA (2) mode; MASK bit for mode 0."""
    v = sum(1 for s in subs if s)
    if mode == 0:
        return int(centre or fill)
    if mode == 1:
        return v | (8 if fill else 0)
    alpha = (255 * v + 2) // 4
    if fill:
        return tuple((style[k] * alpha + style[4 + k] * (255 - alpha) + 127) // 255
                     for k in range(3)) + (255,)
    if v:
        return (style[0], style[1], style[2], alpha)
    return (0, 0, 0, 0)


def render_window(kind, layer, z, tx, ty, r16, i_range, j_range, mode, style=(0,) * 8, R=None):
    """Dict (i, j) -> encoded pixel for the pixels of a window of one tile."""
    out = {}
    for j in j_range:
        for i in i_range:
            centre, subs, fill = pixel_flags(kind, layer, z, tx, ty, r16, i, j, R)
            out[(i, j)] = encode_pixel(mode, centre, subs, fill, style)
    return out
