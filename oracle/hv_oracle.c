/*
 * hv_oracle.c -- the parity oracle for the display-driven tile renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header
 * or constant with the CUDA library and must never be reached from the
 * product path.
 *
 * What it computes (HiVision, Sec. 3.2, Algorithm 1 and Algorithm 2), written
 * as the plain definition on an integer grid:
 *
 *   grid      : 2^31 units per axis, coordinates in [-2^30, 2^30), y grows
 *               southward, tile row 0 is north (Sec. 4: 256 x 256 px tiles
 *               in a tile pyramid, Sec. 2.2: 4^z tiles at level z).
 *   pixel     : at zoom z one pixel is ps = 2^(23-z) units wide (the paper's
 *               resolution R_z, Algorithm 1 step 1), pixel (i, j) of tile
 *               (z, tx, ty) has centre
 *                   cx = -2^30 + tx*2^(31-z) + i*ps + ps/2   (same for y).
 *   samples   : the centre and the four super-samples cx +- ps/4,
 *               cy +- ps/4 (Algorithm 1, the four points P1..P4).
 *   radius    : R = r16 * 2^(19-z) units, r16 = style radius in 1/16 px
 *               (Algorithm 1 step 2, R = N * R_z); or, for buffer analysis
 *               (Sec. 3.2: SIBV extends HiBuffer's buffers, whose distance is
 *               given on the ground), one R in grid units for every tile.
 *   covered   : C(s, R) = exists an object o with dist(o, s) <= R
 *               (closed comparison, Algorithm 1 "distance <= R").
 *   coverage  : v = number of the four super-samples with C (0..4, the
 *               output range of Algorithm 1).  The paper evaluates the
 *               super-samples against the single object nearest to the pixel
 *               centre; the oracle uses the exact per-sample definition.
 *   fill      : f(c) = exists a polygon Q whose own edges, over all of its
 *               rings, cross the ray from c towards +x an odd number of
 *               times (Algorithm 2, ray casting with per-polygon edge
 *               counts; level edges never count).  An edge (a, b) crosses
 *               when (a.y > c.y) != (b.y > c.y) and its crossing lies
 *               strictly right of c.  The half-open straddle rule stands in
 *               for the paper's IsLevel flag and its segment cutting (Sec. 3.1).
 *   fill styles (Sec. 3.2.2 fill styles, Sec. 4.1 Pattern Library):
 *               anti-aliased fill decides f at the four super-samples, as
 *               Algorithm 1 does for outlines (the fill count is the number
 *               inside, 0..4); without it the fill count is 4 when the centre
 *               is inside, else 0.  A pattern is a w x h grid of RGBA texels
 *               (alpha 0 or 255) laid over the global pixel grid: pixel
 *               (256 tx + i, 256 ty + j) takes texel ((256 ty + j) mod h,
 *               (256 tx + i) mod w); a transparent texel leaves the pixel
 *               unfilled, an opaque one gives the fill colour.
 *
 * The algorithm is deliberately data driven (the flow of Fig. 1-1): every
 * object is visited once, the requested tiles it can touch are looked up,
 * and the exact predicate is evaluated on every sample of a window that
 * contains all samples within reach.  A sample outside the window is farther
 * than R from the object, so the window only saves work; the result is the
 * definition above.  All arithmetic is exact integer arithmetic (int64, and
 * unsigned __int128 for the one product that needs 126 bits).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MODE_MASK 0
#define OR_MODE_COVERAGE 1
#define OR_MODE_RGBA 2

/* per-pixel flag bits kept while splatting */
#define F_SUB_NW 1u   /* (cx - q, cy - q) */
#define F_SUB_NE 2u   /* (cx + q, cy - q) */
#define F_SUB_SW 4u   /* (cx - q, cy + q) */
#define F_SUB_SE 8u   /* (cx + q, cy + q) */
#define F_CENTRE 16u
#define F_FILL 32u    /* the centre is inside */
#define F_FSUB_NW 64u /* the super-samples are inside (anti-aliased fill) */
#define F_FSUB_NE 128u
#define F_FSUB_SW 256u
#define F_FSUB_SE 512u

#define TILE_PX 256
#define GRID_HALF ((int64_t)1 << 30)

static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* ---- exact predicates ------------------------------------------------- */

/* |o - s|^2 <= R^2 for a point object. */
static int point_within(int64_t ox, int64_t oy, int64_t sx, int64_t sy, int64_t R) {
    int64_t dx = ox - sx, dy = oy - sy;
    return dx * dx + dy * dy <= R * R;
}

/* distance from s to the closed segment [a, b] is <= R.
 * With d = b - a, w = s - a, t = w.d, L = d.d:
 *   t <= 0  -> nearest point is a,
 *   t >= L  -> nearest point is b,
 *   else    -> squared distance is (w x d)^2 / L, so compare (w x d)^2 <= R^2 L.
 * A zero-length segment has t = 0 and falls into the first case. */
static int segment_within(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                          int64_t sx, int64_t sy, int64_t R) {
    int64_t dx = bx - ax, dy = by - ay;
    int64_t wx = sx - ax, wy = sy - ay;
    int64_t t = wx * dx + wy * dy;
    int64_t L = dx * dx + dy * dy;
    if (t <= 0) return wx * wx + wy * wy <= R * R;
    if (t >= L) {
        int64_t ex = sx - bx, ey = sy - by;
        return ex * ex + ey * ey <= R * R;
    }
    int64_t cross = wx * dy - wy * dx;
    unsigned __int128 c = (unsigned __int128)(cross < 0 ? -cross : cross);
    unsigned __int128 lhs = c * c;
    unsigned __int128 rhs = (unsigned __int128)(uint64_t)(R * R) * (unsigned __int128)(uint64_t)L;
    return lhs <= rhs;
}

/* Does edge (a, b) cross the ray from c towards +x?  Half-open in y, strict
 * in x.  With lo/hi the endpoints ordered by y, the crossing is right of c
 * iff (hi.x - lo.x)(c.y - lo.y) - (c.x - lo.x)(hi.y - lo.y) > 0. */
static int edge_crosses_right(int64_t ax, int64_t ay, int64_t bx, int64_t by,
                              int64_t cx, int64_t cy) {
    if ((ay > cy) == (by > cy)) return 0;
    int64_t lox = ax, loy = ay, hix = bx, hiy = by;
    if (ay > by) { lox = bx; loy = by; hix = ax; hiy = ay; }
    int64_t num = (hix - lox) * (cy - loy) - (cx - lox) * (hiy - loy);
    return num > 0;
}

/* ---- requested-tile lookup --------------------------------------------- */

typedef struct { uint64_t key; uint32_t req; } tile_ref;

static uint64_t tile_key(uint32_t z, uint32_t tx, uint32_t ty) {
    return ((uint64_t)z << 48) | ((uint64_t)tx << 24) | (uint64_t)ty;
}

static int cmp_ref(const void* a, const void* b) {
    const tile_ref* x = (const tile_ref*)a;
    const tile_ref* y = (const tile_ref*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->req < y->req ? -1 : (x->req > y->req);
}

typedef struct {
    const uint32_t *z, *x, *y, *r16;
    int64_t R_fixed;         /* >= 0: the radius of every request (grid units) */
    uint64_t n;
    tile_ref* refs;          /* sorted by key */
    int64_t rmax[32];        /* largest R requested at each zoom, -1 if none */
    uint16_t* flags;         /* n * 65536 per-pixel flags */
} req_table;

static int64_t radius_units(uint32_t r16, uint32_t z) { return (int64_t)r16 << (19 - z); }

/* The radius of request i. */
static int64_t request_radius(const req_table* t, uint64_t i) {
    return t->R_fixed >= 0 ? t->R_fixed : radius_units(t->r16[i], t->z[i]);
}

static int table_init(req_table* t, const uint32_t* z, const uint32_t* x,
                      const uint32_t* y, const uint32_t* r16, uint64_t n, int64_t R_fixed) {
    t->z = z; t->x = x; t->y = y; t->r16 = r16; t->n = n; t->R_fixed = R_fixed;
    for (int k = 0; k < 32; k++) t->rmax[k] = -1;
    t->refs = (tile_ref*)malloc(sizeof(tile_ref) * (n ? n : 1));
    t->flags = (uint16_t*)calloc(n ? n * TILE_PX * TILE_PX : 1, sizeof(uint16_t));
    if (!t->refs || !t->flags) return -1;
    for (uint64_t i = 0; i < n; i++) {
        t->refs[i].key = tile_key(z[i], x[i], y[i]);
        t->refs[i].req = (uint32_t)i;
        int64_t R = request_radius(t, i);
        if (R > t->rmax[z[i]]) t->rmax[z[i]] = R;
    }
    qsort(t->refs, n, sizeof(tile_ref), cmp_ref);
    return 0;
}

static void table_free(req_table* t) { free(t->refs); free(t->flags); }

/* first index in refs with key >= k */
static uint64_t table_lower(const req_table* t, uint64_t k) {
    uint64_t lo = 0, hi = t->n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (t->refs[mid].key < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Tile column containing grid coordinate v at zoom z, clamped to the pyramid. */
static int64_t tile_of(int64_t v, uint32_t z) {
    int64_t span = (int64_t)1 << (31 - z);
    return clamp64(floordiv(v + GRID_HALF, span), 0, ((int64_t)1 << z) - 1);
}

/* The object-kind specific work done on one requested tile. */
typedef void (*splat_fn)(const void* obj, uint32_t z, int64_t X0, int64_t Y0,
                         int64_t R, uint16_t* flags);

/* Visit every requested tile whose area lies within the largest requested
 * radius of the box [x0, x1] x [y0, y1] and call f on it. */
/* Call f on request i (tile (z, tx, ty)) with the tile's origin and radius. */
static void call_request(const req_table* t, uint64_t i, uint32_t z, int64_t tx, int64_t ty,
                         const void* obj, splat_fn f) {
    int64_t span = (int64_t)1 << (31 - z);
    uint32_t r = t->refs[i].req;
    int64_t R = request_radius(t, r);
    f(obj, z, -GRID_HALF + tx * span, -GRID_HALF + ty * span, R,
      t->flags + (uint64_t)r * TILE_PX * TILE_PX);
}

static void for_each_request(const req_table* t, int64_t x0, int64_t y0, int64_t x1,
                             int64_t y1, const void* obj, splat_fn f) {
    for (uint32_t z = 0; z < 32; z++) {
        int64_t E = t->rmax[z];
        if (E < 0) continue;
        if (x1 + E < -GRID_HALF || y1 + E < -GRID_HALF) continue;
        if (x0 - E >= GRID_HALF || y0 - E >= GRID_HALF) continue;
        int64_t tx0 = tile_of(x0 - E, z), tx1 = tile_of(x1 + E, z);
        int64_t ty0 = tile_of(y0 - E, z), ty1 = tile_of(y1 + E, z);
        uint64_t lo = table_lower(t, tile_key(z, 0, 0)), hi = table_lower(t, tile_key(z + 1, 0, 0));
        if ((uint64_t)(tx1 - tx0 + 1) * (uint64_t)(ty1 - ty0 + 1) > hi - lo) {
            /* the box spans more tiles than were requested at this zoom: the
               same calls, found by scanning this zoom's requests instead */
            for (uint64_t i = lo; i < hi; i++) {
                int64_t tx = (int64_t)((t->refs[i].key >> 24) & 0xFFFFFF), ty = (int64_t)(t->refs[i].key & 0xFFFFFF);
                if (tx < tx0 || tx > tx1 || ty < ty0 || ty > ty1) continue;
                call_request(t, i, z, tx, ty, obj, f);
            }
            continue;
        }
        for (int64_t tx = tx0; tx <= tx1; tx++) {
            for (int64_t ty = ty0; ty <= ty1; ty++) {
                uint64_t k = tile_key(z, (uint32_t)tx, (uint32_t)ty);
                for (uint64_t i = table_lower(t, k); i < t->n && t->refs[i].key == k; i++)
                    call_request(t, i, z, tx, ty, obj, f);
            }
        }
    }
}

/* Pixel index range [*lo, *hi] whose footprint comes within R of [v0, v1]. */
static void pixel_window(int64_t v0, int64_t v1, int64_t R, int64_t origin, int64_t ps,
                         int64_t* lo, int64_t* hi) {
    *lo = clamp64(floordiv(v0 - R - origin, ps) - 1, 0, TILE_PX - 1);
    *hi = clamp64(floordiv(v1 + R - origin, ps) + 1, 0, TILE_PX - 1);
}

/* ---- points ----------------------------------------------------------- */

typedef struct { int64_t x, y; } pt_obj;

static void splat_point(const void* obj, uint32_t z, int64_t X0, int64_t Y0, int64_t R,
                        uint16_t* flags) {
    const pt_obj* o = (const pt_obj*)obj;
    int64_t ps = (int64_t)1 << (23 - z), q = ps / 4;
    int64_t i0, i1, j0, j1;
    pixel_window(o->x, o->x, R, X0, ps, &i0, &i1);
    pixel_window(o->y, o->y, R, Y0, ps, &j0, &j1);
    for (int64_t j = j0; j <= j1; j++) {
        int64_t cy = Y0 + j * ps + ps / 2;
        for (int64_t i = i0; i <= i1; i++) {
            int64_t cx = X0 + i * ps + ps / 2;
            uint16_t f = 0;
            if (point_within(o->x, o->y, cx - q, cy - q, R)) f |= F_SUB_NW;
            if (point_within(o->x, o->y, cx + q, cy - q, R)) f |= F_SUB_NE;
            if (point_within(o->x, o->y, cx - q, cy + q, R)) f |= F_SUB_SW;
            if (point_within(o->x, o->y, cx + q, cy + q, R)) f |= F_SUB_SE;
            if (point_within(o->x, o->y, cx, cy, R)) f |= F_CENTRE;
            flags[j * TILE_PX + i] |= f;
        }
    }
}

/* ---- segments (linestring pieces and polygon edges) ------------------- */

typedef struct { int64_t ax, ay, bx, by; } seg_obj;

static void splat_segment(const void* obj, uint32_t z, int64_t X0, int64_t Y0, int64_t R,
                          uint16_t* flags) {
    const seg_obj* s = (const seg_obj*)obj;
    int64_t ps = (int64_t)1 << (23 - z), q = ps / 4;
    int64_t x0 = s->ax < s->bx ? s->ax : s->bx, x1 = s->ax < s->bx ? s->bx : s->ax;
    int64_t y0 = s->ay < s->by ? s->ay : s->by, y1 = s->ay < s->by ? s->by : s->ay;
    int64_t i0, i1, j0, j1;
    pixel_window(x0, x1, R, X0, ps, &i0, &i1);
    pixel_window(y0, y1, R, Y0, ps, &j0, &j1);
    for (int64_t j = j0; j <= j1; j++) {
        int64_t cy = Y0 + j * ps + ps / 2;
        for (int64_t i = i0; i <= i1; i++) {
            int64_t cx = X0 + i * ps + ps / 2;
            uint16_t f = 0;
            if (segment_within(s->ax, s->ay, s->bx, s->by, cx - q, cy - q, R)) f |= F_SUB_NW;
            if (segment_within(s->ax, s->ay, s->bx, s->by, cx + q, cy - q, R)) f |= F_SUB_NE;
            if (segment_within(s->ax, s->ay, s->bx, s->by, cx - q, cy + q, R)) f |= F_SUB_SW;
            if (segment_within(s->ax, s->ay, s->bx, s->by, cx + q, cy + q, R)) f |= F_SUB_SE;
            if (segment_within(s->ax, s->ay, s->bx, s->by, cx, cy, R)) f |= F_CENTRE;
            flags[j * TILE_PX + i] |= f;
        }
    }
}

/* ---- polygon fill ----------------------------------------------------- */

typedef struct {
    const int32_t* xy;        /* all vertices, interleaved x, y */
    const uint64_t* ring_off; /* ring r = vertices [ring_off[r], ring_off[r+1]) */
    uint64_t r0, r1;          /* this polygon's rings [r0, r1) */
    int64_t x0, y0, x1, y1;   /* its bounding box */
    int aa;                   /* also decide the four super-samples */
} poly_obj;

static int polygon_parity(const poly_obj* p, int64_t cx, int64_t cy) {
    int parity = 0;
    for (uint64_t r = p->r0; r < p->r1; r++) {
        uint64_t v0 = p->ring_off[r], v1 = p->ring_off[r + 1];
        for (uint64_t v = v0; v < v1; v++) {
            uint64_t w = (v + 1 < v1) ? v + 1 : v0; /* rings close implicitly */
            if (edge_crosses_right(p->xy[2 * v], p->xy[2 * v + 1], p->xy[2 * w],
                                   p->xy[2 * w + 1], cx, cy))
                parity ^= 1;
        }
    }
    return parity;
}

static void splat_fill(const void* obj, uint32_t z, int64_t X0, int64_t Y0, int64_t R,
                       uint16_t* flags) {
    (void)R;
    const poly_obj* p = (const poly_obj*)obj;
    int64_t ps = (int64_t)1 << (23 - z), q = ps / 4;
    int64_t i0, i1, j0, j1;
    /* a sample outside the polygon's box has even parity; the window reaches
       one pixel past the box, beyond every super-sample inside it */
    pixel_window(p->x0, p->x1, 0, X0, ps, &i0, &i1);
    pixel_window(p->y0, p->y1, 0, Y0, ps, &j0, &j1);
    for (int64_t j = j0; j <= j1; j++) {
        int64_t cy = Y0 + j * ps + ps / 2;
        for (int64_t i = i0; i <= i1; i++) {
            int64_t cx = X0 + i * ps + ps / 2;
            uint16_t f = 0;
            if (polygon_parity(p, cx, cy)) f |= F_FILL;
            if (p->aa) {
                if (polygon_parity(p, cx - q, cy - q)) f |= F_FSUB_NW;
                if (polygon_parity(p, cx + q, cy - q)) f |= F_FSUB_NE;
                if (polygon_parity(p, cx - q, cy + q)) f |= F_FSUB_SW;
                if (polygon_parity(p, cx + q, cy + q)) f |= F_FSUB_SE;
            }
            flags[j * TILE_PX + i] |= f;
        }
    }
}

/* ---- output encoding (Sec. 4.1 Render Tiles; zone array -> image) ----- */

static uint32_t popcount4(uint32_t f) {
    return (f & 1u) + ((f >> 1) & 1u) + ((f >> 2) & 1u) + ((f >> 3) & 1u);
}

uint64_t oracle_tile_bytes(int mode) {
    if (mode == OR_MODE_MASK) return TILE_PX * TILE_PX / 8;
    if (mode == OR_MODE_COVERAGE) return TILE_PX * TILE_PX;
    return TILE_PX * TILE_PX * 4;
}

/* Fill options of polygon layers: anti-aliased fill and a pattern (NULL
 * texels: the style's fill colour everywhere). */
typedef struct {
    int aa;
    const uint8_t* pattern;   /* pw * ph RGBA texels, row-major */
    uint32_t pw, ph;
} fill_opts;

/* style: line colour r,g,b,(unused) then fill colour r,g,b,(unused).
 * Per pixel: v = covered outline super-samples, f = fill count (super-samples
 * inside with anti-aliasing, else 4 when the centre is inside); a pattern
 * texel that is transparent makes f = 0, an opaque one gives the fill colour.
 * RGBA composes the outline over the fill: a_o = (255 v + 2) >> 2,
 * a_f = (255 f + 2) >> 2, A = (255 a_o + a_f (255 - a_o) + 127) / 255 and each
 * colour channel (line a_o 255 + fill a_f (255 - a_o) + 127 A) / (255 A); with
 * f = 4 this is (line a_o + fill (255 - a_o) + 127) / 255 with A = 255, with
 * f = 0 it is the line colour with alpha a_o. */
static void encode(const uint16_t* flags, const req_table* t, int mode, const uint8_t* style,
                   const fill_opts* fo, uint8_t* out) {
    uint64_t tb = oracle_tile_bytes(mode);
    for (uint64_t k = 0; k < t->n; k++) {
        const uint16_t* fl = flags + k * TILE_PX * TILE_PX;
        uint8_t* o = out + k * tb;
        memset(o, 0, tb);
        for (int j = 0; j < TILE_PX; j++) {
            for (int i = 0; i < TILE_PX; i++) {
                uint32_t g = fl[j * TILE_PX + i];
                uint32_t v = popcount4(g);
                uint32_t centre_fill = (g & F_FILL) ? 1u : 0u;
                uint32_t f = (fo && fo->aa) ? popcount4(g >> 6) : 4u * centre_fill;
                const uint8_t* fill = style + 4;
                if (fo && fo->pattern) {
                    uint64_t gx = (uint64_t)t->x[k] * TILE_PX + (uint64_t)i;
                    uint64_t gy = (uint64_t)t->y[k] * TILE_PX + (uint64_t)j;
                    const uint8_t* tx = fo->pattern + 4 * ((gy % fo->ph) * fo->pw + gx % fo->pw);
                    if (tx[3] == 0) { f = 0; centre_fill = 0; }
                    fill = tx;
                }
                if (mode == OR_MODE_MASK) {
                    if ((g & F_CENTRE) || centre_fill) {
                        /* bit b of little-endian word w of row j is pixel 32w+b */
                        int w = i / 32, b = i % 32;
                        o[(j * 8 + w) * 4 + b / 8] |= (uint8_t)(1u << (b % 8));
                    }
                } else if (mode == OR_MODE_COVERAGE) {
                    if (fo && fo->aa)
                        o[j * TILE_PX + i] = (uint8_t)(v | (f << 4));
                    else
                        o[j * TILE_PX + i] = (uint8_t)(v | ((f ? 1u : 0u) << 3));
                } else {
                    uint8_t* px = o + 4 * (j * TILE_PX + i);
                    uint32_t ao = (255u * v + 2u) >> 2, af = (255u * f + 2u) >> 2;
                    if (af) {
                        uint32_t A = (255u * ao + af * (255u - ao) + 127u) / 255u;
                        for (int c = 0; c < 3; c++)
                            px[c] = (uint8_t)((style[c] * ao * 255u + fill[c] * af * (255u - ao) + 127u * A) /
                                              (255u * A));
                        px[3] = (uint8_t)A;
                    } else if (v) {
                        px[0] = style[0]; px[1] = style[1]; px[2] = style[2];
                        px[3] = (uint8_t)ao;
                    }
                }
            }
        }
    }
}

/* ---- entry points ----------------------------------------------------- */

static int check_requests(const uint32_t* z, const uint32_t* x, const uint32_t* y,
                          const uint32_t* r16, uint64_t n, int64_t R_fixed) {
    if (R_fixed > ((int64_t)1 << 29)) return -2;
    for (uint64_t i = 0; i < n; i++) {
        if (z[i] > 19) return -2;
        if (x[i] >= (1u << z[i]) || y[i] >= (1u << z[i])) return -2;
        if (R_fixed < 0 && (r16[i] < 1 || r16[i] > 1024)) return -2;
    }
    return 0;
}

static int check_coords(const int32_t* xy, uint64_t n) {
    for (uint64_t i = 0; i < 2 * n; i++)
        if (xy[i] < -(int32_t)(1 << 30) || xy[i] > (int32_t)((1u << 30) - 1)) return -2;
    return 0;
}

/* Points: xy = n interleaved (x, y).  Returns 0, -1 (no memory) or -2 (range). */
int oracle_render_points_r(const int32_t* xy, uint64_t n, const uint32_t* z, const uint32_t* x,
                           const uint32_t* y, const uint32_t* r16, uint64_t n_req, int64_t R_fixed, int mode,
                           const uint8_t* style, uint8_t* out) {
    if (check_requests(z, x, y, r16, n_req, R_fixed) || check_coords(xy, n)) return -2;
    req_table t;
    if (table_init(&t, z, x, y, r16, n_req, R_fixed)) { table_free(&t); return -1; }
    for (uint64_t k = 0; k < n; k++) {
        pt_obj o = {xy[2 * k], xy[2 * k + 1]};
        for_each_request(&t, o.x, o.y, o.x, o.y, &o, splat_point);
    }
    encode(t.flags, &t, mode, style, NULL, out);
    table_free(&t);
    return 0;
}

/* Linestrings: line l has vertices [line_off[l], line_off[l+1]) and is drawn as
 * its consecutive segments; a line with fewer than two vertices draws nothing. */
int oracle_render_lines_r(const int32_t* xy, uint64_t n_vert, const uint64_t* line_off,
                          uint64_t n_lines, const uint32_t* z, const uint32_t* x,
                          const uint32_t* y, const uint32_t* r16, uint64_t n_req, int64_t R_fixed, int mode,
                          const uint8_t* style, uint8_t* out) {
    if (check_requests(z, x, y, r16, n_req, R_fixed) || check_coords(xy, n_vert)) return -2;
    req_table t;
    if (table_init(&t, z, x, y, r16, n_req, R_fixed)) { table_free(&t); return -1; }
    for (uint64_t l = 0; l < n_lines; l++) {
        for (uint64_t v = line_off[l]; v + 1 < line_off[l + 1]; v++) {
            seg_obj s = {xy[2 * v], xy[2 * v + 1], xy[2 * v + 2], xy[2 * v + 3]};
            int64_t x0 = s.ax < s.bx ? s.ax : s.bx, x1 = s.ax < s.bx ? s.bx : s.ax;
            int64_t y0 = s.ay < s.by ? s.ay : s.by, y1 = s.ay < s.by ? s.by : s.ay;
            for_each_request(&t, x0, y0, x1, y1, &s, splat_segment);
        }
    }
    encode(t.flags, &t, mode, style, NULL, out);
    table_free(&t);
    return 0;
}

/* Polygons: ring r has vertices [ring_off[r], ring_off[r+1]) and closes
 * implicitly; polygon p owns rings [poly_ring_off[p], poly_ring_off[p+1])
 * (outer ring and holes alike).  The outline uses the request's radius on
 * every edge; the fill is decided at the pixel centre. */
int oracle_render_polygons_styled(const int32_t* xy, uint64_t n_vert, const uint64_t* ring_off,
                                  uint64_t n_rings, const uint64_t* poly_ring_off, uint64_t n_polys,
                                  const uint32_t* z, const uint32_t* x, const uint32_t* y,
                                  const uint32_t* r16, uint64_t n_req, int64_t R_fixed, int mode,
                                  const uint8_t* style, int aa, const uint8_t* pattern, uint32_t pw,
                                  uint32_t ph, uint8_t* out) {
    (void)n_rings;
    if (check_requests(z, x, y, r16, n_req, R_fixed) || check_coords(xy, n_vert)) return -2;
    if (pattern) {
        if (pw < 1 || ph < 1 || pw > 16 || ph > 16) return -2;
        for (uint32_t k = 0; k < pw * ph; k++)
            if (pattern[4 * k + 3] != 0 && pattern[4 * k + 3] != 255) return -2;
    }
    fill_opts fo = {aa, pattern, pw, ph};
    req_table t;
    if (table_init(&t, z, x, y, r16, n_req, R_fixed)) { table_free(&t); return -1; }
    for (uint64_t p = 0; p < n_polys; p++) {
        poly_obj P = {xy, ring_off, poly_ring_off[p], poly_ring_off[p + 1], 0, 0, 0, 0, aa};
        int first = 1;
        for (uint64_t r = P.r0; r < P.r1; r++) {
            uint64_t v0 = ring_off[r], v1 = ring_off[r + 1];
            for (uint64_t v = v0; v < v1; v++) {
                uint64_t w = (v + 1 < v1) ? v + 1 : v0;
                seg_obj s = {xy[2 * v], xy[2 * v + 1], xy[2 * w], xy[2 * w + 1]};
                int64_t x0 = s.ax < s.bx ? s.ax : s.bx, x1 = s.ax < s.bx ? s.bx : s.ax;
                int64_t y0 = s.ay < s.by ? s.ay : s.by, y1 = s.ay < s.by ? s.by : s.ay;
                for_each_request(&t, x0, y0, x1, y1, &s, splat_segment);
                if (first) { P.x0 = x0; P.y0 = y0; P.x1 = x1; P.y1 = y1; first = 0; }
                if (x0 < P.x0) P.x0 = x0;
                if (y0 < P.y0) P.y0 = y0;
                if (x1 > P.x1) P.x1 = x1;
                if (y1 > P.y1) P.y1 = y1;
            }
        }
        if (!first) for_each_request(&t, P.x0, P.y0, P.x1, P.y1, &P, splat_fill);
    }
    encode(t.flags, &t, mode, style, &fo, out);
    table_free(&t);
    return 0;
}

int oracle_render_polygons_r(const int32_t* xy, uint64_t n_vert, const uint64_t* ring_off,
                             uint64_t n_rings, const uint64_t* poly_ring_off, uint64_t n_polys,
                             const uint32_t* z, const uint32_t* x, const uint32_t* y,
                             const uint32_t* r16, uint64_t n_req, int64_t R_fixed, int mode,
                             const uint8_t* style, uint8_t* out) {
    return oracle_render_polygons_styled(xy, n_vert, ring_off, n_rings, poly_ring_off, n_polys, z, x, y, r16,
                                         n_req, R_fixed, mode, style, 0, NULL, 0, 0, out);
}

/* The same with each request's own radius (R = r16 * 2^(19 - z)). */
int oracle_render_points(const int32_t* xy, uint64_t n, const uint32_t* z, const uint32_t* x,
                         const uint32_t* y, const uint32_t* r16, uint64_t n_req, int mode,
                         const uint8_t* style, uint8_t* out) {
    return oracle_render_points_r(xy, n, z, x, y, r16, n_req, -1, mode, style, out);
}

int oracle_render_lines(const int32_t* xy, uint64_t n_vert, const uint64_t* line_off,
                        uint64_t n_lines, const uint32_t* z, const uint32_t* x,
                        const uint32_t* y, const uint32_t* r16, uint64_t n_req, int mode,
                        const uint8_t* style, uint8_t* out) {
    return oracle_render_lines_r(xy, n_vert, line_off, n_lines, z, x, y, r16, n_req, -1, mode, style, out);
}

int oracle_render_polygons(const int32_t* xy, uint64_t n_vert, const uint64_t* ring_off,
                           uint64_t n_rings, const uint64_t* poly_ring_off, uint64_t n_polys,
                           const uint32_t* z, const uint32_t* x, const uint32_t* y,
                           const uint32_t* r16, uint64_t n_req, int mode, const uint8_t* style,
                           uint8_t* out) {
    return oracle_render_polygons_r(xy, n_vert, ring_off, n_rings, poly_ring_off, n_polys, z, x, y, r16,
                                    n_req, -1, mode, style, out);
}
