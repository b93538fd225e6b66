"""Seeded synthetic layers and tile-request streams.

This module only draws random inputs; it contains none of the rendering
arithmetic.  Both the CUDA path (tests, benchmark) and the CPU oracle consume
what it returns.  Every generator takes an explicit seed and uses numpy's
``Generator(PCG64(seed))``.

Coordinates are int32 units of a 2^31 x 2^31 Web-Mercator grid,
``[-2^30, 2^30)`` on each axis, y growing southward.  Continuous draws are
quantised with ``floor``; draws that land outside the grid are redrawn (points)
or reflected back into it (random walks), so nothing piles up on the border.

Stand-ins for the paper's datasets (Table 5-2: OSM / OpenCellID points,
linestrings and polygons, 40 M to 2.7 B items), which are not available:

* ``uniform_points``   -- uniformly scattered points.
* ``gmm_points``       -- clustered points (Gaussian mixture + uniform noise),
                          shaped like GPS / cell-tower point clouds.
* ``walk_lines``       -- polylines as random walks around city centres,
                          shaped like road networks.
* ``star_polygons``    -- simple star-shaped polygons around mixture centres,
                          shaped like building / land-use footprints.

Tile requests are ``(n, 4)`` uint32 arrays with columns ``z, x, y, r16``.

Large layers are drawn in chunks, each from its own stream spawned from the
seed (``SeedSequence(seed).spawn``), in a thread pool (numpy's random draws
and array arithmetic release the GIL): the result depends only on the seed and
the chunk size, not on the number of threads.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GRID = 1 << 31
HALF = 1 << 30
CHUNK = 1 << 22          # objects (points, lines, polygons) per drawing chunk


def rng_for(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _chunk_rngs(seed, n_chunks):
    """One independent generator per chunk, spawned from the seed."""
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(n_chunks)]


def _parallel(fn, jobs):
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        return list(ex.map(fn, jobs))


def _floor_i32(v):
    return np.floor(v).astype(np.int64)


def _in_grid(v):
    return (v >= -HALF) & (v < HALF)


def uniform_points(n, seed):
    """n points uniform over the whole grid, int32 (n, 2)."""
    rng = rng_for(seed)
    return rng.integers(-HALF, HALF, size=(n, 2), dtype=np.int64).astype(np.int32)


def _mixture(rng, k):
    """k isotropic Gaussian components: centres uniform in the inner 80% of the
    square, weights Dirichlet(1), sigma log-uniform in [1e-4, 1e-2] of the extent."""
    centres = rng.uniform(-0.8 * HALF, 0.8 * HALF, size=(k, 2))
    weights = rng.dirichlet(np.ones(k))
    sigma = np.exp(rng.uniform(np.log(1e-4), np.log(1e-2), size=k)) * GRID
    return centres, weights, sigma


def _draw_mixture(rng, centres, sigma, comp):
    out = np.empty((comp.shape[0], 2), dtype=np.int64)
    todo = np.arange(comp.shape[0])
    while todo.size:
        c = comp[todo]
        v = _floor_i32(centres[c] + sigma[c, None] * rng.standard_normal((todo.size, 2)))
        ok = _in_grid(v).all(axis=1)
        out[todo[ok]] = v[ok]
        todo = todo[~ok]
    return out


def gmm_points(n, seed, k=64, noise=0.05, chunk=CHUNK):
    """n points: (1 - noise) from a k-component Gaussian mixture, the rest
    uniform.  int32 (n, 2).  The component counts come from the seed's main
    stream; the coordinates are drawn in chunks of `chunk` points, each from
    its own spawned stream."""
    rng = rng_for(seed)
    centres, weights, sigma = _mixture(rng, k)
    n_noise = int(round(noise * n))
    counts = rng.multinomial(n - n_noise, weights)
    bounds = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(counts, out=bounds[1:])
    out = np.empty((n, 2), dtype=np.int32)
    starts = list(range(0, n, chunk))
    rngs = _chunk_rngs(seed, len(starts))

    def one(ci):
        s = starts[ci]
        e = min(n, s + chunk)
        r = rngs[ci]
        m = min(e, n - n_noise)           # [s, m): mixture, [m, e): noise
        if m > s:
            comp = (np.searchsorted(bounds, np.arange(s, m), side="right") - 1).astype(np.int32)
            out[s:m] = _draw_mixture(r, centres, sigma, comp)
        if e > max(s, m):
            q = max(s, m)
            out[q:e] = r.integers(-HALF, HALF, size=(e - q, 2), dtype=np.int64)

    _parallel(one, range(len(starts)))
    return out


def _reflect(v):
    """Fold coordinates back into [-2^30, 2^30) by mirroring at the border."""
    period = 2.0 * GRID
    w = np.mod(v + HALF, period)
    w = np.where(w >= GRID, period - w, w)
    return np.minimum(w - HALF, HALF - 1)


def walk_lines(n_lines, n_segments, seed, n_cities=1000, step_mean=1e-4, step_sigma_ln=1.0,
               turn_deg=30.0, chunk=CHUNK >> 4):
    """Random-walk polylines around city centres.

    Segments per line = 1 + multinomial(n_segments - n_lines, uniform), so the
    total is exactly n_segments.  Start points are Gaussian around uniformly
    placed city centres (sigma log-uniform in [1e-3, 1e-2] of the extent); step
    lengths are log-normal with the given mean (fraction of the extent) and
    sigma of the log; the heading turns by U(-turn, +turn) each step.  Walks
    that leave the grid are reflected back into it.  The per-line draws come
    from the seed's main stream, the walks from one spawned stream per chunk
    of `chunk` lines.
    Returns (xy int32 (V, 2), line_off uint64 (n_lines + 1))."""
    assert n_segments >= n_lines
    rng = rng_for(seed)
    segs = 1 + rng.multinomial(n_segments - n_lines, np.full(n_lines, 1.0 / n_lines))
    nv = segs + 1
    off = np.zeros(n_lines + 1, dtype=np.uint64)
    np.cumsum(nv, out=off[1:])
    V = int(off[-1])
    cc = rng.uniform(-0.8 * HALF, 0.8 * HALF, size=(n_cities, 2))
    cs = np.exp(rng.uniform(np.log(1e-3), np.log(1e-2), size=n_cities)) * GRID
    city = rng.integers(0, n_cities, size=n_lines)
    start = cc[city] + cs[city, None] * rng.standard_normal((n_lines, 2))
    mu = np.log(step_mean * GRID) - 0.5 * step_sigma_ln ** 2
    xy = np.empty((V, 2), dtype=np.int32)
    starts = list(range(0, n_lines, chunk))
    rngs = _chunk_rngs(seed, len(starts))

    def one(ci):
        l0 = starts[ci]
        l1 = min(n_lines, l0 + chunk)
        r = rngs[ci]
        v0, v1 = int(off[l0]), int(off[l1])
        cnv = nv[l0:l1]
        first = (off[l0:l1] - off[l0]).astype(np.int64)
        nl, nvx = l1 - l0, v1 - v0
        line_of_vertex = np.repeat(np.arange(nl), cnv)
        # per-vertex step (the first vertex of each line has a zero step)
        step = np.exp(mu + step_sigma_ln * r.standard_normal(nvx))
        dh = np.deg2rad(r.uniform(-turn_deg, turn_deg, size=nvx))
        dh[first] = r.uniform(0, 2 * np.pi, size=nl)
        step[first] = 0.0
        heading = np.cumsum(dh)
        heading -= np.repeat(heading[first] - dh[first], cnv)
        px = np.cumsum(step * np.cos(heading))
        py = np.cumsum(step * np.sin(heading))
        px -= np.repeat(px[first], cnv)
        py -= np.repeat(py[first], cnv)
        px += start[l0:l1][line_of_vertex, 0]
        py += start[l0:l1][line_of_vertex, 1]
        xy[v0:v1, 0] = _floor_i32(_reflect(px))
        xy[v0:v1, 1] = _floor_i32(_reflect(py))

    _parallel(one, range(len(starts)))
    return xy, off


def star_polygons(n, seed, k=256, nv_min=8, nv_max=64, rho_median=2e-4, rho_sigma_ln=0.75, chunk=CHUNK >> 6):
    """n simple star-shaped polygons (one ring each).

    Centres from a k-component mixture (as ``gmm_points``); vertex count
    uniform in [nv_min, nv_max]; vertex angles are sorted uniform draws
    (drawn as normalised partial sums of exponential spacings);
    vertex radius = rho * U(0.5, 1) with rho log-normal (median rho_median of
    the extent).  After quantisation a polygon is kept only if every pair of
    consecutive vertices turns strictly counter-clockwise about its integer
    centre and all vertices lie in the grid; a star polygon whose consecutive
    vertex pairs all turn the same way around one point is simple.  Rejected
    polygons are redrawn.  The per-polygon draws come from the seed's main
    stream, the vertices from one spawned stream per chunk of `chunk`
    polygons.  Returns (xy, ring_off, poly_ring_off)."""
    rng = rng_for(seed)
    centres, weights, sigma = _mixture(rng, k)
    comp = rng.choice(k, size=n, p=weights)
    pc = _draw_mixture(rng, centres, sigma, comp)
    nv = rng.integers(nv_min, nv_max + 1, size=n)
    rho = np.exp(np.log(rho_median * GRID) + rho_sigma_ln * rng.standard_normal(n))
    ring_off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(nv, out=ring_off[1:])
    xy = np.empty((int(ring_off[-1]), 2), dtype=np.int32)
    starts = list(range(0, n, chunk))
    rngs = _chunk_rngs(seed, len(starts))

    def one(ci):
        r = rngs[ci]
        todo = np.arange(starts[ci], min(n, starts[ci] + chunk))
        while todo.size:
            t_nv = nv[todo]
            tot = int(t_nv.sum())
            pid = np.repeat(np.arange(todo.size), t_nv)
            # sorted uniform angles per polygon without a sort: normalised
            # partial sums of nv + 1 exponential spacings (Renyi representation)
            e = r.standard_exponential(tot + todo.size)
            c = np.cumsum(e)
            ends = np.cumsum(t_nv + 1) - 1                # index of each polygon's last spacing
            base = np.concatenate([[0.0], c[ends[:-1]]])  # sum before each polygon
            total = c[ends] - base
            keep = np.ones(tot + todo.size, dtype=bool)
            keep[ends] = False
            ang = 2 * np.pi * (c[keep] - np.repeat(base, t_nv)) / np.repeat(total, t_nv)
            rad = np.repeat(rho[todo], t_nv) * r.uniform(0.5, 1.0, size=tot)
            cx = np.repeat(pc[todo, 0], t_nv).astype(np.float64)
            cy = np.repeat(pc[todo, 1], t_nv).astype(np.float64)
            vx = _floor_i32(cx + rad * np.cos(ang))
            vy = _floor_i32(cy + rad * np.sin(ang))
            st = np.zeros(todo.size + 1, dtype=np.int64)
            np.cumsum(t_nv, out=st[1:])
            nxt = np.arange(tot) + 1
            nxt[st[1:] - 1] = st[:-1]
            ex = vx - np.repeat(pc[todo, 0], t_nv)
            ey = vy - np.repeat(pc[todo, 1], t_nv)
            cross = ex * ey[nxt] - ey * ex[nxt]
            bad_v = (cross <= 0) | ~_in_grid(vx) | ~_in_grid(vy)
            # a polygon is bad when any of its vertices is
            bad = np.add.reduceat(bad_v.astype(np.int64), st[:-1]) > 0
            keep_v = ~bad[pid]
            # destination of each kept vertex: its polygon's final offset + rank in polygon
            rank = np.arange(tot) - st[pid]
            dest = ring_off[todo[pid[keep_v]]].astype(np.int64) + rank[keep_v]
            xy[dest, 0] = vx[keep_v]
            xy[dest, 1] = vy[keep_v]
            todo = todo[bad]

    _parallel(one, range(len(starts)))
    poly_ring_off = np.arange(n + 1, dtype=np.uint64)
    return xy, ring_off, poly_ring_off


# ---- tile requests --------------------------------------------------------

def tile_of(v, z):
    """Tile index of grid coordinate(s) v at zoom z (tile pyramid addressing)."""
    return ((np.asarray(v, dtype=np.int64) + HALF) >> (31 - z)).astype(np.int64)


def all_tiles(z_min, z_max, r16):
    """Every tile of zooms z_min..z_max (4^z tiles at zoom z)."""
    rows = []
    for z in range(z_min, z_max + 1):
        n = 1 << z
        xs, ys = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        rows.append(np.stack([np.full(n * n, z), xs.ravel(), ys.ravel(), np.full(n * n, r16)], 1))
    return np.concatenate(rows).astype(np.uint32)


def density_tiles(anchor_xy, n_tiles, z_min, z_max, r16, seed):
    """Density-weighted random tiles: pick a uniformly random object anchor
    (a point, a segment midpoint or a polygon centre), a zoom uniform in
    [z_min, z_max], and request the tile containing the anchor.  Duplicates
    are kept.  ``r16`` is a scalar or a sequence to draw uniformly from."""
    rng = rng_for(seed)
    idx = rng.integers(0, anchor_xy.shape[0], size=n_tiles)
    z = rng.integers(z_min, z_max + 1, size=n_tiles)
    a = np.asarray(anchor_xy)[idx].astype(np.int64)
    tx = (a[:, 0] + HALF) >> (31 - z)
    ty = (a[:, 1] + HALF) >> (31 - z)
    if np.isscalar(r16):
        r = np.full(n_tiles, r16)
    else:
        r = rng.choice(np.asarray(r16), size=n_tiles)
    return np.stack([z, tx, ty, r], 1).astype(np.uint32)


def segment_midpoints(xy, line_off, max_n=None, seed=0):
    """Midpoints (floor) of the segments of polylines, optionally subsampled."""
    off = np.asarray(line_off, dtype=np.int64)
    last = np.zeros(xy.shape[0], dtype=bool)
    last[off[1:] - 1] = True
    starts = np.nonzero(~last)[0]
    if max_n is not None and starts.size > max_n:
        starts = rng_for(seed).choice(starts, size=max_n, replace=False)
    a = xy[starts].astype(np.int64)
    b = xy[starts + 1].astype(np.int64)
    return ((a + b) // 2).astype(np.int32)


def polygon_centres(xy, ring_off, poly_ring_off):
    """Bounding-box centres (floor) of polygons' outer rings."""
    ro = np.asarray(ring_off, dtype=np.int64)
    po = np.asarray(poly_ring_off, dtype=np.int64)
    first = ro[po[:-1]]
    end = ro[po[:-1] + 1]
    x = xy[:, 0].astype(np.int64)
    y = xy[:, 1].astype(np.int64)
    mnx = np.minimum.reduceat(x, first)
    mxx = np.maximum.reduceat(x, first)
    mny = np.minimum.reduceat(y, first)
    mxy = np.maximum.reduceat(y, first)
    del end
    return np.stack([(mnx + mxx) // 2, (mny + mxy) // 2], 1).astype(np.int32)


# ---- the five benchmark workloads (shapes of the paper's experiments) ------

def config1():
    """100,000 uniform points; all 341 tiles of zoom 0-4; radius 1 px; MASK."""
    pts = uniform_points(100_000, seed=1)
    return pts, all_tiles(0, 4, 16)


def config2(n_points=100_000_000, n_tiles=10_000):
    """100M clustered points; 10,000 density-weighted tiles at zoom 8-14;
    radius 2 px; RGBA."""
    pts = gmm_points(n_points, seed=2, k=64)
    return pts, density_tiles(pts, n_tiles, 8, 14, 32, seed=102)


def config3(n_lines=5_000_000, n_segments=50_000_000, n_tiles=10_000, r16=16):
    """50M segments in 5M random-walk polylines; 10,000 density-weighted tiles
    at zoom 6-16; half-width r16 (8, 16 or 24 = 0.5, 1, 1.5 px)."""
    xy, off = walk_lines(n_lines, n_segments, seed=3)
    mids = segment_midpoints(xy, off, max_n=4 * n_tiles, seed=103)
    return xy, off, density_tiles(mids, n_tiles, 6, 16, r16, seed=203)


def config4(n_polys=2_000_000, n_tiles=10_000):
    """2M star polygons (8-64 vertices); 10,000 density-weighted tiles at
    zoom 4-14; fill + 1 px outline (half-width 0.5 px, r16 = 8)."""
    xy, ro, po = star_polygons(n_polys, seed=4)
    cen = polygon_centres(xy, ro, po)
    return xy, ro, po, density_tiles(cen, n_tiles, 4, 14, 8, seed=104)


def pan_zoom_trace(anchors, n, seed, n_sessions=256, z_start=10, z_min=2, z_max=18, zipf_s=1.1,
                   r16_range=(16, 48), p_pan=0.7):
    """Tile requests from seeded pan / zoom browsing sessions (the request
    stream of HiVision Exp. 3, shaped as interactive map use).

    ``anchors`` holds one (m, 2) anchor array per layer.  Each session picks a
    layer uniformly and a start tile at zoom ``z_start`` drawn Zipf(s) over the
    layer's tiles ranked by anchor count; each step pans to one of the 8
    neighbours (probability p_pan) or zooms in / out by one level (clamped to
    [z_min, z_max]).  Sessions are interleaved uniformly at random.  r16 is
    uniform in r16_range.  Returns an (n, 5) array [z, x, y, r16, layer]."""
    rng = rng_for(seed)
    starts = []
    for a in anchors:
        t = tile_of(a, z_start)
        key = (t[:, 0] << 32) | t[:, 1]
        uk, cnt = np.unique(key, return_counts=True)
        order = np.argsort(-cnt, kind="stable")
        ranked = uk[order]
        w = 1.0 / np.arange(1, len(ranked) + 1) ** zipf_s
        starts.append((ranked, w / w.sum()))
    state = np.zeros((n_sessions, 4), dtype=np.int64)   # layer, z, x, y
    for s in range(n_sessions):
        layer = int(rng.integers(0, len(anchors)))
        ranked, p = starts[layer]
        k = ranked[rng.choice(len(ranked), p=p)]
        state[s] = (layer, z_start, k >> 32, k & 0xFFFFFFFF)
    out = np.zeros((n, 5), dtype=np.int64)
    who = rng.integers(0, n_sessions, size=n)
    u = rng.random(n)
    nb = rng.integers(0, 8, size=n)
    kid = rng.integers(0, 4, size=n)
    r16 = rng.integers(r16_range[0], r16_range[1] + 1, size=n)
    moves = np.array([(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)])
    for i in range(n):
        layer, z, x, y = state[who[i]]
        if u[i] < p_pan:
            dx, dy = moves[nb[i]]
            m = (1 << z) - 1
            x, y = min(max(x + dx, 0), m), min(max(y + dy, 0), m)
        elif u[i] < p_pan + (1 - p_pan) / 2:
            if z < z_max:
                z, x, y = z + 1, 2 * x + (kid[i] & 1), 2 * y + (kid[i] >> 1)
        elif z > z_min:
            z, x, y = z - 1, x >> 1, y >> 1
        state[who[i]] = (layer, z, x, y)
        out[i] = (z, x, y, r16[i], layer)
    return out


def poisson_arrivals(n, rate, seed):
    """Arrival times (microseconds) of an open-loop Poisson stream."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1e6 / rate, size=n))


def shard(rows, rank, world):
    """Contiguous shard `rank` of `world` of a request array (replica serving:
    every rank holds the whole layer and renders its own share of tiles)."""
    n = len(rows)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return rows[lo:hi]
