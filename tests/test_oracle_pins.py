"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Closed forms from tests/golden/closed_forms.json, exact identities of the
sample construction, invariants, and byte-for-byte agreement with the
independent pure-Python brute force on tiny layers (HiVision Sec. 3.2,
Algorithms 1 and 2).
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from geom import (at, centre, coverage_fill, coverage_value, golden, lines_to_arrays, ps,
                  polys_to_arrays, random_cluster_points, random_star_polygons,
                  random_walk_lines, ring_px)

MASK, COV, RGBA = oracle.MODE_MASK, oracle.MODE_COVERAGE, oracle.MODE_RGBA
Z, TX, TY = 10, 300, 517          # a mid-zoom reference tile
GOLD = golden("closed_forms.json")
STYLE = (200, 30, 60, 0, 20, 140, 250, 0)


def req(z=Z, tx=TX, ty=TY, r16=16):
    return np.array([[z, tx, ty, r16]], dtype=np.uint32)


def mask_count(out):
    return int(oracle.mask_bits(out[0]).sum())


# ---- Algorithm 1: closed disc, pixel grid, tile addressing ----------------

@pytest.mark.parametrize("case", GOLD["gauss_circle"]["cases"], ids=lambda c: str(c["r16"]))
def test_gauss_circle(case):
    pts = np.array([at(Z, TX, TY, 100, 120)], dtype=np.int32)
    out = oracle.render_points(pts, req(r16=case["r16"]), MASK)
    assert mask_count(out) == case["count"]


def test_corner_point():
    case = GOLD["corner_point"]["cases"][0]
    pts = np.array([at(Z, TX, TY, 100, 120, -0.5, -0.5)], dtype=np.int32)
    out = oracle.render_points(pts, req(r16=case["r16"]), MASK)
    bits = oracle.mask_bits(out[0])
    assert bits.sum() == case["count"]
    assert bits[119:121, 99:101].all()


@pytest.mark.parametrize("z,tx,ty,i,j", [(0, 0, 0, 5, 7), (3, 2, 6, 250, 3), (10, 300, 517, 0, 255),
                                         (19, 262143, 1, 128, 64), (19, 0, 524287, 255, 0)])
def test_pixel_addressing(z, tx, ty, i, j):
    """A point on the centre of pixel (i, j) with a 1/16 px radius lights exactly
    that pixel (row j counted from the north edge), and none of its super-samples
    (they are sqrt(2)/4 px away)."""
    pts = np.array([centre(z, tx, ty, i, j)], dtype=np.int32)
    out = oracle.render_points(pts, req(z, tx, ty, 1), MASK)
    bits = oracle.mask_bits(out[0])
    assert bits.sum() == 1 and bits[j, i]
    cov = oracle.render_points(pts, req(z, tx, ty, 1), COV)
    assert cov.sum() == 0


def test_neighbour_tiles_see_across_border():
    """An object near a tile edge reaches into the next tile (east and south)."""
    pts = np.array([at(Z, TX, TY, 255, 255, 0.5, 0.5)], dtype=np.int32)
    reqs = np.array([[Z, TX, TY, 16], [Z, TX + 1, TY, 16], [Z, TX, TY + 1, 16],
                     [Z, TX + 1, TY + 1, 16]], dtype=np.uint32)
    out = oracle.render_points(pts, reqs, MASK)
    assert [oracle.mask_bits(o)[:, :].sum() for o in out] == [1, 1, 1, 1]
    assert oracle.mask_bits(out[3])[0, 0] and oracle.mask_bits(out[0])[255, 255]


@pytest.mark.parametrize("case", GOLD["segment_band"]["cases"],
                         ids=lambda c: "k%d_r%d" % (c["k"], c["r16"]))
def test_segment_band(case):
    k = case["k"]
    for vertical in (False, True):
        if vertical:
            line = [at(Z, TX, TY, 100, 100), at(Z, TX, TY, 100, 100 + k)]
        else:
            line = [at(Z, TX, TY, 100, 100), at(Z, TX, TY, 100 + k, 100)]
        xy, off = lines_to_arrays([line])
        out = oracle.render_lines(xy, off, req(r16=case["r16"]), MASK)
        assert mask_count(out) == case["count"]


def test_short_lines_draw_nothing():
    xy, off = lines_to_arrays([[at(Z, TX, TY, 50, 50)], []])
    out = oracle.render_lines(xy, off, req(r16=64), MASK)
    assert mask_count(out) == 0


def test_long_segment_needs_wide_products():
    """A segment spanning most of the grid at zoom 0 with a 64 px half-width:
    the cross product squared reaches ~2^120, past 64-bit range.  Compare
    with the exact rational distance of the brute force."""
    a = (-(1 << 30) + 12345, -(1 << 30) + 777)
    b = ((1 << 30) - 9876, (1 << 30) - 4321)
    xy, off = lines_to_arrays([[a, b]])
    for r16 in (1024, 333, 100, 7):
        cov = oracle.render_lines(xy, off, req(0, 0, 0, r16), COV)[0].reshape(256, 256)
        win = brute.render_window("lines", [[a, b]], 0, 0, 0, r16, range(100, 140),
                                  range(90, 150), COV)
        for (i, j), v in win.items():
            assert cov[j, i] == v, (i, j)


# ---- Algorithm 2: ray parity, level edges, vertices on the ray, holes ----

def _fill_count(polys, z=Z, tx=TX, ty=TY):
    xy, ro, po = polys_to_arrays(polys)
    out = oracle.render_polygons(xy, ro, po, req(z, tx, ty, 1), COV)
    return coverage_fill(out[0])


def _square(i, j, k):
    return ring_px(Z, TX, TY, i, j, [(0, 0), (k, 0), (k, k), (0, k)])


@pytest.mark.parametrize("case", GOLD["square_fill"]["cases"], ids=lambda c: str(c["k"]))
def test_square_fill_is_half_open(case):
    k = case["k"]
    f = _fill_count([[_square(60, 70, k)]])
    assert f.sum() == case["count"]
    assert f[70:70 + k, 60:60 + k].all()   # exactly [x0, x1) x [y0, y1)


@pytest.mark.parametrize("case", GOLD["square_with_hole"]["cases"], ids=lambda c: str(c["k"]))
def test_square_with_hole(case):
    k, h = case["k"], case["h"]
    o = (k - h) // 2
    f = _fill_count([[_square(60, 70, k), _square(60 + o, 70 + o, h)]])
    assert f.sum() == case["count"]
    assert not f[70 + o:70 + o + h, 60 + o:60 + o + h].any()


@pytest.mark.parametrize("case", GOLD["overlapping_squares"]["cases"], ids=lambda c: str(c["k"]))
def test_overlapping_squares(case):
    k, m = case["k"], case["m"]
    a, b = _square(60, 70, k), _square(60 + m, 70 + m, k)
    assert _fill_count([[a], [b]]).sum() == case["union"]
    assert _fill_count([[a, b]]).sum() == case["xor"]


@pytest.mark.parametrize("case", GOLD["diamond"]["cases"], ids=lambda c: str(c["k"]))
def test_diamond_turning_vertices(case):
    k = case["k"]
    ring = ring_px(Z, TX, TY, 100, 100, [(0, -k), (k, 0), (0, k), (-k, 0)])
    assert _fill_count([[ring]]).sum() == case["count"]


@pytest.mark.parametrize("case", GOLD["monotone_vertex"]["cases"], ids=lambda c: str(c["k"]))
def test_monotone_chain_through_vertex(case):
    k = case["k"]
    ring = ring_px(Z, TX, TY, 100, 100, [(0, 0), (k, 0), (k, k), (0, k), (-k // 2, k // 2)])
    assert _fill_count([[ring]]).sum() == case["count"]
    # the same polygon with its vertex order reversed
    assert _fill_count([[ring[::-1]]]).sum() == case["count"]


def test_polygon_mask_is_fill_or_outline():
    ring = _square(60, 70, 6)
    xy, ro, po = polys_to_arrays([[ring]])
    m = oracle.mask_bits(oracle.render_polygons(xy, ro, po, req(r16=8), MASK)[0])
    c = oracle.render_polygons(xy, ro, po, req(r16=8), COV)[0].reshape(256, 256)
    centre_on_outline = m & ((c & 8) == 0)
    # half-width 0.5 px: the outline reaches exactly the centres on the ring
    assert m.sum() == 36 + 6 + 6 + 1
    assert centre_on_outline.sum() == 13


# ---- identities of the sample construction --------------------------------

def _child_mask(render, z, tx, ty, r16):
    """The 512 x 512 array of MASK bits of the four child tiles at z+1."""
    reqs = np.array([[z + 1, 2 * tx + a, 2 * ty + b, 2 * r16] for b in (0, 1) for a in (0, 1)],
                    dtype=np.uint32)
    out = render(reqs, MASK)
    big = np.zeros((512, 512), dtype=np.uint8)
    for k, (a, b) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        big[256 * b:256 * b + 256, 256 * a:256 * a + 256] = oracle.mask_bits(out[k])
    return big


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_coverage_equals_children_masks(kind):
    """The four super-samples of a pixel are the centres of its four children
    at zoom z+1, so COVERAGE(z, r16) = sum of MASK(z+1, 2*r16) over them."""
    rng = np.random.default_rng(7)
    z, tx, ty = 9, 150, 258
    if kind == "points":
        pts = random_cluster_points(rng, 300, z, tx, ty, 40)

        def render(reqs, mode):
            return oracle.render_points(pts, reqs, mode)
    elif kind == "lines":
        xy, off = lines_to_arrays(random_walk_lines(rng, 20, 6, z, tx, ty, 8))

        def render(reqs, mode):
            return oracle.render_lines(xy, off, reqs, mode)
    else:
        xy, ro, po = polys_to_arrays(random_star_polygons(rng, 12, z, tx, ty, 20, holes=True))

        def render(reqs, mode):
            return oracle.render_polygons(xy, ro, po, reqs, mode)
    for r16 in (5, 16, 40):
        cov = render(np.array([[z, tx, ty, r16]], dtype=np.uint32), COV)[0].reshape(256, 256)
        big = _child_mask(render, z, tx, ty, r16)
        kids = big[0::2, 0::2] + big[1::2, 0::2] + big[0::2, 1::2] + big[1::2, 1::2]
        assert (cov & 7).sum() > 0
        if kind != "polygons":
            assert np.array_equal(cov & 7, kids)
            continue
        # a child MASK bit of a polygon layer is outline OR fill at the child
        # centre; where no child centre is filled it is the outline alone.
        reqs = np.array([[z + 1, 2 * tx + a, 2 * ty + b, 2 * r16] for b in (0, 1) for a in (0, 1)],
                        dtype=np.uint32)
        ccov = render(reqs, COV)
        fill = np.zeros((512, 512), dtype=bool)
        for k, (a, b) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
            fill[256 * b:256 * b + 256, 256 * a:256 * a + 256] = coverage_fill(ccov[k])
        any_fill = fill[0::2, 0::2] | fill[1::2, 0::2] | fill[0::2, 1::2] | fill[1::2, 1::2]
        assert (~any_fill).sum() > 1000 and any_fill.sum() > 100
        assert np.array_equal((cov & 7)[~any_fill], kids[~any_fill])


def test_radius_monotone_and_union_and_order():
    rng = np.random.default_rng(11)
    a = random_cluster_points(rng, 200, Z, TX, TY, 30)
    b = random_cluster_points(rng, 150, Z, TX, TY, 30, 90, 170)
    prev = None
    for r16 in (4, 9, 16, 31, 64):
        m = oracle.mask_bits(oracle.render_points(a, req(r16=r16), MASK)[0])
        if prev is not None:
            assert not (prev & ~m).any()
        prev = m
    ma = oracle.mask_bits(oracle.render_points(a, req(r16=20), MASK)[0])
    mb = oracle.mask_bits(oracle.render_points(b, req(r16=20), MASK)[0])
    ab = np.concatenate([b, a, a[:17]])[::-1]
    mab = oracle.mask_bits(oracle.render_points(ab, req(r16=20), MASK)[0])
    assert np.array_equal(mab, ma | mb)


def test_translation_by_whole_pixels():
    rng = np.random.default_rng(3)
    xy, off = lines_to_arrays(random_walk_lines(rng, 10, 5, Z, TX, TY, 6, 100, 100, 15))
    p = 1 << (23 - Z)
    sh = xy.astype(np.int64) + np.array([7 * p, -5 * p])
    o1 = oracle.render_lines(xy, off, req(r16=20), COV)[0].reshape(256, 256)
    o2 = oracle.render_lines(sh.astype(np.int32), off, req(r16=20), COV)[0].reshape(256, 256)
    assert np.array_equal(o1[20:230, 20:230], o2[15:225, 27:237])


def test_far_tiles_are_empty():
    rng = np.random.default_rng(5)
    pts = random_cluster_points(rng, 500, Z, TX, TY, 20)
    reqs = np.array([[Z, TX + 3, TY, 64], [Z, TX, TY - 2, 64], [Z + 2, 4 * TX + 9, 4 * TY, 64]],
                    dtype=np.uint32)
    assert not oracle.render_points(pts, reqs, RGBA).any()


def test_paper_r1_r2_claim():
    """Sec. 3.2: if the nearest object is within R1 = R - sqrt(2)/4 R_z of the
    centre, all four super-samples are covered; beyond R2 = R + sqrt(2)/4 R_z,
    none is."""
    rng = np.random.default_rng(9)
    pts = random_cluster_points(rng, 60, Z, TX, TY, 25)
    p = float(1 << (23 - Z))
    for r16 in (12, 32, 70):
        R = r16 * (1 << (19 - Z))
        cov = coverage_value(oracle.render_points(pts, req(r16=r16), COV)[0])
        for j in range(60, 200, 3):
            for i in range(60, 200, 3):
                cx, cy = centre(Z, TX, TY, i, j)
                d = np.sqrt(((pts.astype(np.float64) - [cx, cy]) ** 2).sum(1)).min()
                if d <= R - np.sqrt(2) / 4 * p - 1e-3 * p:
                    assert cov[j, i] == 4
                if d > R + np.sqrt(2) / 4 * p + 1e-3 * p:
                    assert cov[j, i] == 0


# ---- the C oracle against the pure-Python brute force ---------------------

def _compare_window(kind, layer, c_out, z, tx, ty, r16, mode, win):
    i_rng, j_rng = win
    ref = brute.render_window(kind, layer, z, tx, ty, r16, i_rng, j_rng, mode, STYLE)
    if mode == MASK:
        got = oracle.mask_bits(c_out)
        for (i, j), v in ref.items():
            assert int(got[j, i]) == v, (i, j)
    elif mode == COV:
        got = c_out.reshape(256, 256)
        for (i, j), v in ref.items():
            assert got[j, i] == v, (i, j)
    else:
        got = c_out.reshape(256, 256, 4)
        for (i, j), v in ref.items():
            assert tuple(int(x) for x in got[j, i]) == v, (i, j)


@pytest.mark.parametrize("mode", [MASK, COV, RGBA])
@pytest.mark.parametrize("seed", [1, 2])
def test_brute_points(mode, seed):
    rng = np.random.default_rng(seed)
    z, tx, ty = 12, 1000, 2000
    pts = random_cluster_points(rng, 12, z, tx, ty, 5, 30, 30)
    pts = np.concatenate([pts, pts[:2]])                    # duplicates
    r16 = int(rng.integers(8, 60))
    out = oracle.render_points(pts, [[z, tx, ty, r16]], mode, STYLE)[0]
    layer = [tuple(map(int, p)) for p in pts]
    _compare_window("points", layer, out, z, tx, ty, r16, mode, (range(14, 46), range(14, 46)))


@pytest.mark.parametrize("mode", [MASK, COV, RGBA])
@pytest.mark.parametrize("seed", [1, 2])
def test_brute_lines(mode, seed):
    rng = np.random.default_rng(seed + 10)
    z, tx, ty = 11, 700, 900
    lines = random_walk_lines(rng, 4, 4, z, tx, ty, 5, 30, 30, 6)
    lines.append([at(z, tx, ty, 25, 25), at(z, tx, ty, 25, 25)])   # zero-length segment
    lines.append([at(z, tx, ty, 20, 40, 0.3, 0.1), at(z, tx, ty, 40, 40, 0.3, 0.1)])  # level
    xy, off = lines_to_arrays(lines)
    r16 = int(rng.integers(4, 40))
    out = oracle.render_lines(xy, off, [[z, tx, ty, r16]], mode, STYLE)[0]
    layer = [[tuple(map(int, v)) for v in ln] for ln in lines]
    _compare_window("lines", layer, out, z, tx, ty, r16, mode, (range(14, 46), range(14, 46)))


@pytest.mark.parametrize("mode", [MASK, COV, RGBA])
@pytest.mark.parametrize("seed,snap", [(1, False), (2, True), (3, True)])
def test_brute_polygons(mode, seed, snap):
    rng = np.random.default_rng(seed + 20)
    z, tx, ty = 13, 3000, 5000
    polys = random_star_polygons(rng, 4, z, tx, ty, 8, 30, 30, 5, holes=True, snap=snap)
    xy, ro, po = polys_to_arrays(polys)
    r16 = int(rng.integers(2, 24))
    out = oracle.render_polygons(xy, ro, po, [[z, tx, ty, r16]], mode, STYLE)[0]
    layer = [[[tuple(map(int, v)) for v in ring] for ring in rings] for rings in polys]
    _compare_window("polygons", layer, out, z, tx, ty, r16, mode, (range(16, 44), range(16, 44)))


def test_brute_across_zoom_zero_and_nineteen():
    for z, tx, ty in ((0, 0, 0), (19, 4242, 77777)):
        rng = np.random.default_rng(z)
        pts = random_cluster_points(rng, 8, z, tx, ty, 3, 10, 10)
        out = oracle.render_points(pts, [[z, tx, ty, 23]], COV)[0]
        layer = [tuple(map(int, p)) for p in pts]
        _compare_window("points", layer, out, z, tx, ty, 23, COV, (range(0, 22), range(0, 22)))


# ---- buffer analysis: one radius in grid units for every tile ---------------

def _lattice_disc(r_num, r_den):
    """Pixel centres of a unit lattice within distance r = r_num / r_den of a
    lattice point: #{(i, j) : i^2 + j^2 <= r^2}, the Gauss circle count."""
    m = r_num // r_den + 1
    return sum(1 for i in range(-m, m + 1) for j in range(-m, m + 1) if (i * i + j * j) * r_den * r_den <= r_num * r_num)


@pytest.mark.parametrize("z,R", [(10, 10000), (10, 17000), (10, 8191), (10, 8192), (14, 100), (3, 123456789)])
def test_buffer_radius_gauss_circle(z, R):
    """A point at a pixel centre with a radius in grid units that r16 cannot
    express (R / pixel not a multiple of 1/16): the MASK covers the lattice
    points of the disc of radius R / pixel (R = 8191 and 8192 units at zoom 10
    straddle one pixel: 1 and 5 pixels)."""
    tx, ty = (1 << z) // 3, (1 << z) // 5
    p = np.array([centre(z, tx, ty, 128, 128)], dtype=np.int32)
    out = oracle.render_points(p, [[z, tx, ty, 1]], MASK, R_units=R)
    assert mask_count(out) == _lattice_disc(R, 1 << (23 - z))
    if (z, R) in ((10, 10000), (10, 8192)):
        assert mask_count(out) == 5
    if (z, R) == (10, 17000):
        assert mask_count(out) == 13
    if (z, R) == (10, 8191):
        assert mask_count(out) == 1


def test_buffer_radius_ignores_r16_and_matches_r16_radius():
    """The fixed radius replaces every request's own; expressed through r16
    (R = r16 * 2^(19 - z)) the two paths agree."""
    rng = np.random.default_rng(31)
    z, tx, ty = 12, 1000, 2000
    pts = random_cluster_points(rng, 40, z, tx, ty, 8)
    a = oracle.render_points(pts, [[z, tx, ty, 24], [z, tx, ty, 1000]], COV, R_units=24 << (19 - z))
    b = oracle.render_points(pts, [[z, tx, ty, 24]], COV)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[0])
    with pytest.raises(ValueError):
        oracle.render_points(pts, [[z, tx, ty, 16]], MASK, R_units=(1 << 29) + 1)


@pytest.mark.parametrize("kind", ["points", "lines", "polygons"])
def test_buffer_radius_brute(kind):
    """The C oracle with a ground radius against the brute force."""
    rng = np.random.default_rng(41)
    z, tx, ty = 13, 3000, 5000
    R = 3 * ps(z) + 777                           # 3.09 px, not a multiple of 1/16 px
    if kind == "points":
        layer = [tuple(map(int, p)) for p in random_cluster_points(rng, 10, z, tx, ty, 5, 30, 30)]
        out = oracle.render_points(np.array(layer, np.int32), [[z, tx, ty, 1]], COV, R_units=R)[0]
    elif kind == "lines":
        layer = random_walk_lines(rng, 3, 4, z, tx, ty, 5, 30, 30, 6)
        xy, off = lines_to_arrays(layer)
        out = oracle.render_lines(xy, off, [[z, tx, ty, 1]], COV, R_units=R)[0]
    else:
        layer = random_star_polygons(rng, 3, z, tx, ty, 8, 30, 30, 5, holes=True, snap=True)
        xy, ro, po = polys_to_arrays(layer)
        out = oracle.render_polygons(xy, ro, po, [[z, tx, ty, 1]], COV, R_units=R)[0]
    ref = brute.render_window(kind, layer, z, tx, ty, 1, range(16, 44), range(16, 44), COV, R=R)
    got = out.reshape(256, 256)
    assert all(got[j, i] == v for (i, j), v in ref.items())


# ---- fill styles: anti-aliased fill and pattern fill (Sec. 3.2.2, Sec. 4.1) --

def _centre_square(k, i0=60, j0=70, z=Z, tx=TX, ty=TY):
    return polys_to_arrays([[ring_px(z, tx, ty, i0, j0, [(0, 0), (k, 0), (k, k), (0, k)])]])


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_aa_fill_square_on_pixel_centres(k):
    """A k x k px square with its vertices on pixel centres, fill decided at
    the super-samples (+-1/4 px) with the half-open rule: the (k-1)^2 pixels
    strictly inside hold all four samples, the 4(k-1) edge pixels two, the
    four corner pixels one -- 4 k^2 samples, the square's area in quarter
    pixels."""
    xy, ro, po = _centre_square(k)
    f = oracle.render_polygons(xy, ro, po, req(r16=1), COV, aa=True)[0].reshape(256, 256) >> 4
    assert int(f.sum()) == 4 * k * k
    assert (f == 4).sum() == (k - 1) ** 2 and (f == 2).sum() == 4 * (k - 1) and (f == 1).sum() == 4
    assert f[70 + 1:70 + k, 60 + 1:60 + k].min(initial=4) == 4 and f[70, 60] == 1 and f[70 + k, 60 + k] == 1


def test_aa_fill_square_on_pixel_corners_is_exact():
    """Vertices on pixel corners: every pixel is wholly in or out, so the
    anti-aliased fill counts 4 or 0 and agrees with the centre fill."""
    k = 7
    xy, ro, po = polys_to_arrays([[[(x - ps(Z) // 2, y - ps(Z) // 2) for (x, y) in
                                    ring_px(Z, TX, TY, 60, 70, [(0, 0), (k, 0), (k, k), (0, k)])]]])
    cov = oracle.render_polygons(xy, ro, po, req(r16=1), COV, aa=True)[0].reshape(256, 256)
    plain = oracle.render_polygons(xy, ro, po, req(r16=1), COV)[0].reshape(256, 256)
    f = cov >> 4
    assert set(np.unique(f)) == {0, 4} and (f == 4).sum() == k * k
    assert np.array_equal(f == 4, (plain & 8) != 0)


def test_aa_fill_rgba_by_hand():
    """A square on pixel centres with a hairline outline (r16 = 1: no
    super-sample within reach of an edge, v = 0): interior pixels take the
    fill colour opaque, edge pixels (f = 2) the fill colour at alpha
    (255*2 + 2) >> 2 = 128, corners (f = 1) at alpha 64 -- worked out from
    A = (a_f * 255 + 127) / 255 = a_f and rgb = (fill * a_f * 255 + 127 a_f) /
    (255 a_f) = fill."""
    k = 4
    xy, ro, po = _centre_square(k)
    px = oracle.render_polygons(xy, ro, po, req(r16=1), RGBA, STYLE, aa=True)[0].reshape(256, 256, 4)
    fill = STYLE[4:7]
    assert tuple(px[72, 62]) == fill + (255,)
    assert tuple(px[70, 62]) == fill + (128,) and tuple(px[72, 60]) == fill + (128,)
    assert tuple(px[70, 60]) == fill + (64,) and tuple(px[70 + k, 60 + k]) == fill + (64,)
    assert tuple(px[69, 62]) == (0, 0, 0, 0)


def test_aa_rgba_compose_values_by_hand():
    """Outline over an anti-aliased fill, values worked out by hand for the
    line colour (200, 30, 60) over the fill colour (20, 140, 250):
    v = 2, f = 2: a_o = a_f = 128, A = (255*128 + 128*127 + 127) / 255 = 192,
      r = (200*128*255 + 20*128*127 + 127*192) / (255*192) = 140, g = 66, b = 123;
    v = 1, f = 3: a_o = 64, a_f = 191, A = 207, rgb = (76, 106, 191).
    The pixels are found by their COVERAGE bytes (v | f << 4) in a layer of
    random polygons with wide outlines."""
    rng = np.random.default_rng(3)
    z, tx, ty = 13, 3000, 5000
    polys = random_star_polygons(rng, 30, z, tx, ty, 20, 128, 128, 60)
    xy, ro, po = polys_to_arrays(polys)
    want = {(2, 2): (140, 66, 123, 192), (1, 3): (76, 106, 191, 207)}
    found = set()
    for r16 in (2, 4, 6):
        cov = oracle.render_polygons(xy, ro, po, [[z, tx, ty, r16]], COV, aa=True)[0].reshape(256, 256)
        px = oracle.render_polygons(xy, ro, po, [[z, tx, ty, r16]], RGBA, STYLE, aa=True)[0].reshape(256, 256, 4)
        for (v, f), rgba in want.items():
            jj, ii = np.nonzero(cov == (v | (f << 4)))
            for j, i in zip(jj[:20], ii[:20]):
                assert tuple(int(c) for c in px[j, i]) == rgba, (v, f, i, j)
                found.add((v, f))
    assert found == set(want)


def test_pattern_fill_checkerboard():
    """A 2 x 2 checkerboard pattern (opaque / transparent texels) over a
    k x k square with vertices on pixel corners: the filled pixels are those
    whose global column + row is even (256 is even, so the tile's pixel
    i + j decides), k^2 / 2 of them, each with its texel's colour."""
    k = 8
    red, blue = (250, 10, 10, 255), (10, 10, 250, 255)
    pat = np.array([[red, (0, 0, 0, 0)], [(0, 0, 0, 0), blue]], dtype=np.uint8)   # [row][column]
    xy, ro, po = polys_to_arrays([[[(x - ps(Z) // 2, y - ps(Z) // 2) for (x, y) in
                                    ring_px(Z, TX, TY, 60, 70, [(0, 0), (k, 0), (k, k), (0, k)])]]])
    m = oracle.mask_bits(oracle.render_polygons(xy, ro, po, req(r16=1), MASK, pattern=pat)[0])
    assert m.sum() == k * k // 2
    jj, ii = np.nonzero(m)
    assert ((ii + jj) % 2 == 0).all()
    px = oracle.render_polygons(xy, ro, po, req(r16=1), RGBA, STYLE, pattern=pat)[0].reshape(256, 256, 4)
    assert tuple(px[70, 60]) == red[:3] + (255,) and tuple(px[71, 61]) == blue[:3] + (255,)
    assert tuple(px[70, 61]) == (0, 0, 0, 0)


def test_pattern_is_anchored_to_the_global_pixel_grid():
    """A 4-wide, 2-high pattern: texel (row gy mod 2, column gx mod 4) of the
    global pixel (256 tx + i, 256 ty + j), so neighbouring tiles continue it."""
    k = 12
    pat = np.zeros((2, 4, 4), dtype=np.uint8)
    pat[0, 1] = (1, 2, 3, 255)
    pat[1, 3] = (4, 5, 6, 255)
    for tx, ty in ((TX, TY), (TX + 1, TY), (TX, TY + 3)):
        xy, ro, po = polys_to_arrays([[[(x - ps(Z) // 2, y - ps(Z) // 2) for (x, y) in
                                        ring_px(Z, tx, ty, 100, 100, [(0, 0), (k, 0), (k, k), (0, k)])]]])
        px = oracle.render_polygons(xy, ro, po, [[Z, tx, ty, 1]], RGBA, STYLE, pattern=pat)[0].reshape(256, 256, 4)
        for j in range(100, 100 + k):
            for i in range(100, 100 + k):
                gx, gy = 256 * tx + i, 256 * ty + j
                t = pat[gy % 2, gx % 4]
                want = tuple(int(c) for c in t[:3]) + (255,) if t[3] else (0, 0, 0, 0)
                assert tuple(int(c) for c in px[j, i]) == want


@pytest.mark.parametrize("seed", [1, 2])
def test_aa_fill_brute(seed):
    """The anti-aliased fill counts against the brute force's super-sample
    ray casting, holes and lattice vertices included."""
    rng = np.random.default_rng(seed + 40)
    z, tx, ty = 13, 3000, 5000
    polys = random_star_polygons(rng, 4, z, tx, ty, 8, 30, 30, 5, holes=True, snap=True)
    xy, ro, po = polys_to_arrays(polys)
    f = oracle.render_polygons(xy, ro, po, [[z, tx, ty, 4]], COV, aa=True)[0].reshape(256, 256) >> 4
    layer = [[[tuple(map(int, v)) for v in ring] for ring in rings] for rings in polys]
    for j in range(16, 44):
        for i in range(16, 44):
            assert f[j, i] == sum(brute.fill_samples(layer, z, tx, ty, i, j)), (i, j)


def test_rejects_out_of_range():
    pts = np.array([[0, 0]], dtype=np.int32)
    for bad in ([20, 0, 0, 16], [3, 8, 0, 16], [3, 0, 8, 16], [3, 0, 0, 0], [3, 0, 0, 1025]):
        with pytest.raises(ValueError):
            oracle.render_points(pts, [bad], MASK)
    with pytest.raises(ValueError):
        oracle.render_points(np.array([[1 << 30, 0]], dtype=np.int64).astype(np.int32), [[0, 0, 0, 16]], MASK)


def test_rgba_values_by_hand():
    """RGBA values worked out by hand.  Points placed exactly on 1..4 of a
    pixel's super-samples, with a radius (1/16 px) too small to reach any
    other sample, give v = 1..4 and alpha (255 v + 2) >> 2 = 64, 128, 191,
    255 in the line colour.  A square whose west edge passes through a
    pixel's two west super-samples covers exactly those two (v = 2) and fills
    the pixel (its centre lies inside), so the pixel is the composite
    ((line * 128 + fill * 127 + 127) // 255 per channel, 255); the pixel to
    its east is filled with v = 0, i.e. the fill colour itself."""
    z, tx, ty = 10, 300, 400
    q = ps(z) // 4
    line, fill = STYLE[:3], STYLE[4:7]
    for v, i in zip((1, 2, 3, 4), (40, 60, 80, 100)):
        cx, cy = centre(z, tx, ty, i, 50)
        samples = [(cx - q, cy - q), (cx + q, cy - q), (cx - q, cy + q), (cx + q, cy + q)][:v]
        pts = np.array(samples, dtype=np.int32)
        got = oracle.render_points(pts, [[z, tx, ty, 1]], RGBA, STYLE)[0].reshape(256, 256, 4)
        assert tuple(int(x) for x in got[50, i]) == line + ((255 * v + 2) >> 2,)
        assert int(np.count_nonzero(got[:, :, 3])) == 1          # no other pixel is reached
    i, j = 120, 130
    cx, cy = centre(z, tx, ty, i, j)
    x_edge = cx - q
    square = [(x_edge, cy - 5 * ps(z)), (x_edge + 40 * ps(z), cy - 5 * ps(z)),
              (x_edge + 40 * ps(z), cy + 5 * ps(z)), (x_edge, cy + 5 * ps(z))]
    xy, ro, po = polys_to_arrays([[square]])
    got = oracle.render_polygons(xy, ro, po, [[z, tx, ty, 1]], RGBA, STYLE)[0].reshape(256, 256, 4)
    comp = tuple((l * 128 + f * 127 + 127) // 255 for l, f in zip(line, fill)) + (255,)
    assert tuple(int(x) for x in got[j, i]) == comp
    assert tuple(int(x) for x in got[j, i + 1]) == fill + (255,)
    assert tuple(int(x) for x in got[j, i - 1]) == (0, 0, 0, 0)
