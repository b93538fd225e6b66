"""Small geometric fixtures for the tests (grid addressing written out once).

The grid: 2^31 units per axis, coordinates in [-2^30, 2^30), y southward;
at zoom z a pixel is 2^(23-z) units and pixel (i, j) of tile (z, tx, ty) has
its centre at -2^30 + tx*2^(31-z) + i*ps + ps/2 (and likewise for y).
"""
import json
import os

import numpy as np

HALF = 1 << 30
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def ps(z):
    return 1 << (23 - z)


def centre(z, tx, ty, i, j):
    p = ps(z)
    return (-HALF + tx * (1 << (31 - z)) + i * p + p // 2,
            -HALF + ty * (1 << (31 - z)) + j * p + p // 2)


def at(z, tx, ty, i, j, di=0.0, dj=0.0):
    """Grid point at pixel (i, j) of the tile, offset by (di, dj) px (exact
    when the offset is a multiple of 1/16 px)."""
    cx, cy = centre(z, tx, ty, i, j)
    p = ps(z)
    return (cx + int(round(di * p)), cy + int(round(dj * p)))


def ring_px(z, tx, ty, i, j, pts_px):
    """A ring given as pixel offsets from pixel (i, j)."""
    return [at(z, tx, ty, i, j, a, b) for a, b in pts_px]


def polys_to_arrays(polys):
    """[[ring, ...], ...] -> (xy, ring_off, poly_ring_off)."""
    xy, ring_off, poly_off = [], [0], [0]
    for rings in polys:
        for ring in rings:
            xy.extend(ring)
            ring_off.append(len(xy))
        poly_off.append(len(ring_off) - 1)
    return (np.array(xy, dtype=np.int32).reshape(-1, 2), np.array(ring_off, dtype=np.uint64),
            np.array(poly_off, dtype=np.uint64))


def lines_to_arrays(lines):
    xy, off = [], [0]
    for line in lines:
        xy.extend(line)
        off.append(len(xy))
    return np.array(xy, dtype=np.int32).reshape(-1, 2), np.array(off, dtype=np.uint64)


def coverage_fill(tile_cov):
    """(256, 256) bool of the fill bit of a COVERAGE tile."""
    return (np.asarray(tile_cov).reshape(256, 256) & 8) != 0


def coverage_value(tile_cov):
    return np.asarray(tile_cov).reshape(256, 256) & 7


def random_cluster_points(rng, n, z, tx, ty, spread_px, i0=128, j0=128):
    cx, cy = centre(z, tx, ty, i0, j0)
    p = ps(z)
    v = rng.normal(0, spread_px * p, size=(n, 2))
    return np.floor(np.stack([cx + v[:, 0], cy + v[:, 1]], 1)).astype(np.int64).clip(
        -HALF, HALF - 1).astype(np.int32)


def random_walk_lines(rng, n_lines, n_steps, z, tx, ty, step_px, i0=128, j0=128, spread_px=40):
    cx, cy = centre(z, tx, ty, i0, j0)
    p = ps(z)
    lines = []
    for _ in range(n_lines):
        x = cx + rng.normal(0, spread_px * p)
        y = cy + rng.normal(0, spread_px * p)
        h = rng.uniform(0, 2 * np.pi)
        line = [(int(np.floor(x)), int(np.floor(y)))]
        for _ in range(rng.integers(1, n_steps + 1)):
            h += rng.uniform(-0.6, 0.6)
            s = rng.exponential(step_px * p)
            x += s * np.cos(h)
            y += s * np.sin(h)
            line.append((int(np.clip(np.floor(x), -HALF, HALF - 1)),
                         int(np.clip(np.floor(y), -HALF, HALF - 1))))
        lines.append(line)
    return lines


def random_star_polygons(rng, n, z, tx, ty, radius_px, i0=128, j0=128, spread_px=40,
                         holes=False, snap=False):
    """Star polygons around random centres; optional square-ish holes and
    snapping of vertices to pixel centres (to put vertices on scanlines)."""
    p = ps(z)
    polys = []
    for _ in range(n):
        ci = i0 + rng.normal(0, spread_px)
        cj = j0 + rng.normal(0, spread_px)
        k = int(rng.integers(3, 12))
        ang = np.sort(rng.uniform(0, 2 * np.pi, size=k))
        rad = radius_px * rng.uniform(0.4, 1.0, size=k)
        ring = []
        for a, r in zip(ang, rad):
            fi, fj = ci + r * np.cos(a), cj + r * np.sin(a)
            if snap:
                fi, fj = round(fi), round(fj)
            x, y = centre(z, tx, ty, 0, 0)
            ring.append((int(np.clip(np.floor(x + fi * p), -HALF, HALF - 1)),
                         int(np.clip(np.floor(y + fj * p), -HALF, HALF - 1))))
        rings = [ring]
        if holes and rng.random() < 0.5:
            h = 0.25 * radius_px
            x, y = centre(z, tx, ty, 0, 0)
            rings.append([(int(np.floor(x + (ci + a) * p)), int(np.floor(y + (cj + b) * p)))
                          for a, b in ((-h, -h), (-h, h), (h, h), (h, -h))])
        polys.append(rings)
    return polys
