"""The pins have teeth: plant plausible mistakes in a copy of the C oracle
(on the CPU) and check that the pin battery rejects every one of them."""
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from geom import (at, centre, coverage_fill, golden, lines_to_arrays, polys_to_arrays,
                  random_cluster_points, random_star_polygons, random_walk_lines, ring_px)

SRC = os.path.join(os.path.dirname(oracle.__file__), "hv_oracle.c")
GOLD = golden("closed_forms.json")
Z, TX, TY = 10, 300, 517
MASK, COV, RGBA = oracle.MODE_MASK, oracle.MODE_COVERAGE, oracle.MODE_RGBA

MUTANTS = {
    "open_disc": ("return dx * dx + dy * dy <= R * R;", "return dx * dx + dy * dy < R * R;"),
    "straddle_closed_below": ("if ((ay > cy) == (by > cy)) return 0;",
                              "if ((ay >= cy) == (by >= cy)) return 0;"),
    "crossing_not_strict": ("return num > 0;", "return num >= 0;"),
    "ring_not_closed": ("uint64_t w = (v + 1 < v1) ? v + 1 : v0; /* rings close implicitly */",
                        "uint64_t w = (v + 1 < v1) ? v + 1 : v; /* rings close implicitly */"),
    "subsample_offset": ("int64_t ps = (int64_t)1 << (23 - z), q = ps / 4;\n    int64_t i0, i1, j0, j1;\n    pixel_window(o->x",
                         "int64_t ps = (int64_t)1 << (23 - z), q = ps / 8;\n    int64_t i0, i1, j0, j1;\n    pixel_window(o->x"),
    "far_cap_uses_a": ("int64_t ex = sx - bx, ey = sy - by;", "int64_t ex = sx - ax, ey = sy - ay;"),
    "narrow_products": ("unsigned __int128 lhs = c * c;",
                        "unsigned __int128 lhs = (uint64_t)(c * c);"),
    "tile_origin": ("f(obj, z, -GRID_HALF + tx * span, -GRID_HALF + ty * span, R,",
                    "f(obj, z, -GRID_HALF + ty * span, -GRID_HALF + tx * span, R,"),
    "radius_scale": ("return (int64_t)r16 << (19 - z); }", "return (int64_t)r16 << (18 - z); }"),
    "parity_and_not_xor": ("parity ^= 1;", "parity = 1;"),
    "aa_count_shifted": ("uint32_t f = (fo && fo->aa) ? popcount4(g >> 6) : 4u * centre_fill;",
                         "uint32_t f = (fo && fo->aa) ? popcount4(g >> 5) : 4u * centre_fill;"),
    "pattern_transposed": ("4 * ((gy % fo->ph) * fo->pw + gx % fo->pw)", "4 * ((gx % fo->ph) * fo->pw + gy % fo->pw)"),
    "buffer_radius_ignored": ("return t->R_fixed >= 0 ? t->R_fixed : radius_units(t->r16[i], t->z[i]);",
                              "return radius_units(t->r16[i], t->z[i]);"),
}


def _battery(lib):
    """Return the list of pins that fail for the oracle library `lib`."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    pts = np.array([at(Z, TX, TY, 100, 120)], dtype=np.int32)
    for c in GOLD["gauss_circle"]["cases"]:
        out = oracle.render_points(pts, [[Z, TX, TY, c["r16"]]], MASK, lib=lib)
        check("gauss", oracle.mask_bits(out[0]).sum() == c["count"])
    p = np.array([centre(3, 2, 6, 250, 3)], dtype=np.int32)
    b = oracle.mask_bits(oracle.render_points(p, [[3, 2, 6, 1]], MASK, lib=lib)[0])
    check("addressing", b.sum() == 1 and b[3, 250])
    for c in GOLD["segment_band"]["cases"]:
        xy, off = lines_to_arrays([[at(Z, TX, TY, 100, 100), at(Z, TX, TY, 100 + c["k"], 100)]])
        out = oracle.render_lines(xy, off, [[Z, TX, TY, c["r16"]]], MASK, lib=lib)
        check("band", oracle.mask_bits(out[0]).sum() == c["count"])

    def fill(polys):
        xy, ro, po = polys_to_arrays(polys)
        return coverage_fill(oracle.render_polygons(xy, ro, po, [[Z, TX, TY, 1]], COV, lib=lib)[0])

    for c in GOLD["square_fill"]["cases"]:
        k = c["k"]
        f = fill([[ring_px(Z, TX, TY, 60, 70, [(0, 0), (k, 0), (k, k), (0, k)])]])
        check("square", f.sum() == c["count"] and f[70:70 + k, 60:60 + k].all())
    for c in GOLD["diamond"]["cases"]:
        k = c["k"]
        f = fill([[ring_px(Z, TX, TY, 100, 100, [(0, -k), (k, 0), (0, k), (-k, 0)])]])
        check("diamond", f.sum() == c["count"])
    for c in GOLD["overlapping_squares"]["cases"]:
        k, m = c["k"], c["m"]
        a = ring_px(Z, TX, TY, 60, 70, [(0, 0), (k, 0), (k, k), (0, k)])
        bb = ring_px(Z, TX, TY, 60 + m, 70 + m, [(0, 0), (k, 0), (k, k), (0, k)])
        check("union", fill([[a], [bb]]).sum() == c["union"])
        check("xor", fill([[a, bb]]).sum() == c["xor"])
    # child identity on clustered points
    rng = np.random.default_rng(7)
    z, tx, ty = 9, 150, 258
    cp = random_cluster_points(rng, 200, z, tx, ty, 40)
    cov = oracle.render_points(cp, [[z, tx, ty, 16]], COV, lib=lib)[0].reshape(256, 256)
    kids = np.zeros((256, 256), dtype=np.int64)
    reqs = [[z + 1, 2 * tx + a, 2 * ty + bq, 32] for bq in (0, 1) for a in (0, 1)]
    out = oracle.render_points(cp, reqs, MASK, lib=lib)
    big = np.zeros((512, 512), dtype=np.int64)
    for k, (a, bq) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        big[256 * bq:256 * bq + 256, 256 * a:256 * a + 256] = oracle.mask_bits(out[k])
    kids = big[0::2, 0::2] + big[1::2, 0::2] + big[0::2, 1::2] + big[1::2, 1::2]
    check("children", np.array_equal(cov & 7, kids))
    # brute force on a tiny line layer and on a long zoom-0 segment
    rng = np.random.default_rng(12)
    z, tx, ty = 11, 700, 900
    lines = random_walk_lines(rng, 3, 4, z, tx, ty, 5, 30, 30, 6)
    xy, off = lines_to_arrays(lines)
    got = oracle.render_lines(xy, off, [[z, tx, ty, 20]], COV, lib=lib)[0].reshape(256, 256)
    ref = brute.render_window("lines", lines, z, tx, ty, 20, range(18, 42), range(18, 42), COV)
    check("brute_lines", all(got[j, i] == v for (i, j), v in ref.items()))
    a = (-(1 << 30) + 12345, -(1 << 30) + 777)
    bq = ((1 << 30) - 9876, (1 << 30) - 4321)
    xy, off = lines_to_arrays([[a, bq]])
    got = oracle.render_lines(xy, off, [[0, 0, 0, 100]], COV, lib=lib)[0].reshape(256, 256)
    ref = brute.render_window("lines", [[a, bq]], 0, 0, 0, 100, range(110, 130), range(100, 140), COV)
    check("brute_long", all(got[j, i] == v for (i, j), v in ref.items()))
    polys = random_star_polygons(np.random.default_rng(23), 3, 13, 3000, 5000, 8, 30, 30, 5,
                                 holes=True, snap=True)
    xy, ro, po = polys_to_arrays(polys)
    got = oracle.render_polygons(xy, ro, po, [[13, 3000, 5000, 6]], COV, lib=lib)[0].reshape(256, 256)
    ref = brute.render_window("polygons", polys, 13, 3000, 5000, 6, range(18, 42), range(18, 42), COV)
    check("brute_polygons", all(got[j, i] == v for (i, j), v in ref.items()))
    # buffer analysis: a ground radius that r16 cannot express
    bp = np.array([centre(10, 300, 517, 128, 128)], dtype=np.int32)
    out = oracle.render_points(bp, [[10, 300, 517, 1]], MASK, lib=lib, R_units=17000)
    check("buffer_radius", oracle.mask_bits(out[0]).sum() == 13)
    # fill styles: the anti-aliased square and a pattern that is not symmetric
    k = 5
    xy, ro, po = polys_to_arrays([[ring_px(Z, TX, TY, 60, 70, [(0, 0), (k, 0), (k, k), (0, k)])]])
    f = oracle.render_polygons(xy, ro, po, [[Z, TX, TY, 1]], COV, lib=lib, aa=True)[0].reshape(256, 256) >> 4
    check("aa_square", int(f.sum()) == 4 * k * k and (f == 1).sum() == 4)
    polys = random_star_polygons(np.random.default_rng(44), 3, 13, 3000, 5000, 8, 30, 30, 5, holes=True, snap=True)
    xy, ro, po = polys_to_arrays(polys)
    f = oracle.render_polygons(xy, ro, po, [[13, 3000, 5000, 4]], COV, lib=lib, aa=True)[0].reshape(256, 256) >> 4
    check("aa_brute", all(f[j, i] == sum(brute.fill_samples(polys, 13, 3000, 5000, i, j))
                          for j in range(18, 42) for i in range(18, 42)))
    pat = np.zeros((2, 4, 4), dtype=np.uint8)
    pat[0, 1] = (1, 2, 3, 255)
    pat[1, 3] = (4, 5, 6, 255)
    half = (1 << (22 - Z))
    xy, ro, po = polys_to_arrays([[[(x - half, y - half) for (x, y) in
                                    ring_px(Z, TX, TY, 100, 100, [(0, 0), (12, 0), (12, 12), (0, 12)])]]])
    px = oracle.render_polygons(xy, ro, po, [[Z, TX, TY, 1]], RGBA, lib=lib, pattern=pat)[0].reshape(256, 256, 4)
    ok = all((px[j, i, 3] == 255) == bool(pat[(256 * TY + j) % 2, (256 * TX + i) % 4, 3])
             for j in range(100, 112) for i in range(100, 112))
    check("pattern", ok)
    return failed


def test_unmutated_battery_passes():
    assert _battery(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    mut_src = tmp_path / ("mut_%s.c" % name)
    mut_src.write_text(src.replace(old, new))
    so = oracle.compile_source(str(mut_src), str(tmp_path / ("mut_%s.so" % name)))
    failed = _battery(oracle.bind(so))
    assert failed, "planted mistake %r passed every pin" % name
