// Multithreaded CPU R-tree renderer: the paper's own pixel-driven method on
// the host cores, kept as a reported baseline for the GPU library (not used by
// it).  HiVision Sec. 3.2: every pixel asks the spatial index, per
// super-sample, whether an object lies within R (Algorithm 1, with the exact
// per-sample rule, stopping at the first hit), and for polygon layers whether
// its centre is inside some polygon (Algorithm 2: the polygon boxes that
// contain the centre, then the parity of that polygon's own edges crossing
// the ray towards +x).  Tile rows are processed by a pool of threads that take
// (tile, row) items in turn (the row split of the paper's hybrid engine,
// Sec. 4.3).
//
// Index: records (points, segments, polygon edges, polygon boxes) sorted by
// the 62-bit Hilbert key of their box centre, leaves of 32 records, inner
// nodes of 32 child boxes.  Output: RGBA tiles in the library's byte layout.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace {

constexpr int64_t kHalf = 1ll << 30;

uint64_t hilbert(int32_t gx, int32_t gy) {
    uint32_t x = (uint32_t)(gx + (int32_t)kHalf), y = (uint32_t)(gy + (int32_t)kHalf);
    uint64_t d = 0;
    for (uint32_t s = 1u << 30; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += (uint64_t)s * s * ((3 * rx) ^ ry);
        if (!ry) {
            if (rx) { x = ~x; y = ~y; }
            std::swap(x, y);
        }
    }
    return d;
}

struct Box { int32_t x0, y0, x1, y1; };
struct Seg { int32_t ax, ay, bx, by; };

Box unite(const Box& a, const Box& b) {
    return {std::min(a.x0, b.x0), std::min(a.y0, b.y0), std::max(a.x1, b.x1), std::max(a.y1, b.y1)};
}

template <class F>
void parallel_for(int nthreads, uint64_t n, F f) {
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; t++)
        th.emplace_back([&, t] {
            uint64_t lo = n * t / nthreads, hi = n * (t + 1) / nthreads;
            f(lo, hi, t);
        });
    for (auto& x : th) x.join();
}

void radix_sort(std::vector<uint64_t>& key, std::vector<uint32_t>& idx, int nthreads) {
    uint64_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> i2(n);
    for (int pass = 0; pass < 8; pass++) {
        int sh = pass * 8;
        std::vector<std::vector<uint64_t>> hist(nthreads, std::vector<uint64_t>(256, 0));
        parallel_for(nthreads, n, [&](uint64_t lo, uint64_t hi, int t) {
            for (uint64_t i = lo; i < hi; i++) hist[t][(key[i] >> sh) & 255]++;
        });
        uint64_t sum = 0;
        for (int b = 0; b < 256; b++)
            for (int t = 0; t < nthreads; t++) {
                uint64_t c = hist[t][b];
                hist[t][b] = sum;
                sum += c;
            }
        parallel_for(nthreads, n, [&](uint64_t lo, uint64_t hi, int t) {
            for (uint64_t i = lo; i < hi; i++) {
                uint64_t p = hist[t][(key[i] >> sh) & 255]++;
                k2[p] = key[i];
                i2[p] = idx[i];
            }
        });
        key.swap(k2);
        idx.swap(i2);
    }
}

// Packed Hilbert R-tree over record boxes.  levels[0] holds the boxes of the
// leaves (32 consecutive sorted records each); levels[l] the boxes of groups
// of 32 entries of levels[l - 1]; the last level is the root alone.
struct Index {
    std::vector<Box> rec;        // record boxes, sorted
    std::vector<uint32_t> id;    // original index of each sorted record
    std::vector<std::vector<Box>> levels;
};

void build_index(const std::vector<Box>& boxes, int nthreads, Index* I) {
    const uint64_t n = boxes.size();
    std::vector<uint64_t> key(n);
    std::vector<uint32_t> idx(n);
    parallel_for(nthreads, n, [&](uint64_t lo, uint64_t hi, int) {
        for (uint64_t i = lo; i < hi; i++) {
            const Box& b = boxes[i];
            key[i] = hilbert((int32_t)(((int64_t)b.x0 + b.x1) >> 1), (int32_t)(((int64_t)b.y0 + b.y1) >> 1));
            idx[i] = (uint32_t)i;
        }
    });
    radix_sort(key, idx, nthreads);
    I->rec.resize(n);
    I->id = idx;
    parallel_for(nthreads, n, [&](uint64_t lo, uint64_t hi, int) {
        for (uint64_t i = lo; i < hi; i++) I->rec[i] = boxes[idx[i]];
    });
    I->levels.clear();
    if (n == 0) return;
    std::vector<Box> cur((n + 31) / 32, Box{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN});
    for (uint64_t i = 0; i < n; i++) cur[i / 32] = unite(cur[i / 32], I->rec[i]);
    I->levels.push_back(cur);
    while (I->levels.back().size() > 1) {
        const std::vector<Box>& c = I->levels.back();
        std::vector<Box> up((c.size() + 31) / 32, Box{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN});
        for (uint64_t i = 0; i < c.size(); i++) up[i / 32] = unite(up[i / 32], c[i]);
        I->levels.push_back(up);
    }
}

// Is there a record, under entry `node` of levels[level], whose box passes
// `prune` and which passes `test`?  Depth first, first hit wins.
template <class Prune, class Test>
bool any_record(const Index& I, int level, uint64_t node, const Prune& prune, const Test& test) {
    if (level == 0) {
        uint64_t c0 = node * 32, c1 = std::min<uint64_t>(c0 + 32, I.rec.size());
        for (uint64_t c = c0; c < c1; c++)
            if (prune(I.rec[c]) && test(c)) return true;
        return false;
    }
    const std::vector<Box>& below = I.levels[level - 1];
    uint64_t c0 = node * 32, c1 = std::min<uint64_t>(c0 + 32, below.size());
    for (uint64_t c = c0; c < c1; c++)
        if (prune(below[c]) && any_record(I, level - 1, c, prune, test)) return true;
    return false;
}

template <class Prune, class Test>
bool query(const Index& I, const Prune& prune, const Test& test) {
    if (I.rec.empty()) return false;
    return any_record(I, (int)I.levels.size() - 1, 0, prune, test);
}

// ---- exact predicates (Sec. 3.2: closed distance; Algorithm 2 ray test) ----

bool seg_within(const Seg& s, int64_t px, int64_t py, int64_t R2) {
    const int64_t dx = (int64_t)s.bx - s.ax, dy = (int64_t)s.by - s.ay;
    const int64_t wx = px - s.ax, wy = py - s.ay;
    const int64_t t = wx * dx + wy * dy;
    if (t <= 0) return wx * wx + wy * wy <= R2;
    const int64_t L = dx * dx + dy * dy;
    if (t >= L) {
        const int64_t ex = px - s.bx, ey = py - s.by;
        return ex * ex + ey * ey <= R2;
    }
    const __int128 cr = (__int128)wx * dy - (__int128)wy * dx;
    return cr * cr <= (__int128)R2 * L;
}

bool crosses_right(const Seg& e, int64_t cx, int64_t cy) {
    if ((e.ay > cy) == (e.by > cy)) return false;
    int64_t lx = e.ax, ly = e.ay, hx = e.bx, hy = e.by;
    if (e.ay > e.by) { lx = e.bx; ly = e.by; hx = e.ax; hy = e.ay; }
    return (hx - lx) * (cy - ly) - (cx - lx) * (hy - ly) > 0;
}

int64_t box_dist2(const Box& b, int64_t px, int64_t py) {
    const int64_t gx = std::max<int64_t>({0, (int64_t)b.x0 - px, px - (int64_t)b.x1});
    const int64_t gy = std::max<int64_t>({0, (int64_t)b.y0 - py, py - (int64_t)b.y1});
    return gx * gx + gy * gy;
}

enum { kPoints = 0, kLines = 1, kPolygons = 2 };

struct Tree {
    int kind = kPoints;
    int nthreads = 1;
    Index obj;                    // points (degenerate boxes) or segments / edges
    std::vector<Seg> seg;         // segments / edges in the sorted order of obj
    Index poly;                   // polygon boxes (id = polygon)
    std::vector<Seg> edges;       // polygon edges in polygon order
    std::vector<uint64_t> edge_off;
};

Box seg_box(const Seg& s) {
    return {std::min(s.ax, s.bx), std::min(s.ay, s.by), std::max(s.ax, s.bx), std::max(s.ay, s.by)};
}

void index_segments(Tree* T, const std::vector<Seg>& segs) {
    std::vector<Box> boxes(segs.size());
    for (uint64_t i = 0; i < segs.size(); i++) boxes[i] = seg_box(segs[i]);
    build_index(boxes, T->nthreads, &T->obj);
    T->seg.resize(segs.size());
    for (uint64_t i = 0; i < segs.size(); i++) T->seg[i] = segs[T->obj.id[i]];
}

int pick_threads(int n) { return n > 0 ? n : (int)std::max(1u, std::thread::hardware_concurrency()); }

}  // namespace

extern "C" {

// Points: xy is n (x, y) int32 pairs.
void* cpu_rtree_build(const int32_t* xy, uint64_t n, int nthreads) {
    Tree* T = new Tree();
    T->kind = kPoints;
    T->nthreads = pick_threads(nthreads);
    std::vector<Box> boxes(n);
    for (uint64_t i = 0; i < n; i++) boxes[i] = {xy[2 * i], xy[2 * i + 1], xy[2 * i], xy[2 * i + 1]};
    build_index(boxes, T->nthreads, &T->obj);
    return T;
}

// Linestrings: line l has vertices [line_off[l], line_off[l + 1]) and draws
// its n - 1 segments.
void* cpu_rtree_build_lines(const int32_t* xy, const uint64_t* line_off, uint64_t n_lines, int nthreads) {
    Tree* T = new Tree();
    T->kind = kLines;
    T->nthreads = pick_threads(nthreads);
    std::vector<Seg> segs;
    for (uint64_t l = 0; l < n_lines; l++)
        for (uint64_t v = line_off[l]; v + 1 < line_off[l + 1]; v++)
            segs.push_back({xy[2 * v], xy[2 * v + 1], xy[2 * v + 2], xy[2 * v + 3]});
    index_segments(T, segs);
    return T;
}

// Polygons: ring r has vertices [ring_off[r], ring_off[r + 1]) and closes
// implicitly; polygon p owns rings [poly_ring_off[p], poly_ring_off[p + 1]).
void* cpu_rtree_build_polygons(const int32_t* xy, const uint64_t* ring_off, const uint64_t* poly_ring_off,
                               uint64_t n_polys, int nthreads) {
    Tree* T = new Tree();
    T->kind = kPolygons;
    T->nthreads = pick_threads(nthreads);
    std::vector<Box> pboxes;
    std::vector<uint32_t> pid;
    T->edge_off.assign(n_polys + 1, 0);
    for (uint64_t p = 0; p < n_polys; p++) {
        Box b{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
        for (uint64_t r = poly_ring_off[p]; r < poly_ring_off[p + 1]; r++) {
            const uint64_t v0 = ring_off[r], v1 = ring_off[r + 1];
            for (uint64_t v = v0; v < v1; v++) {
                const uint64_t w = v + 1 < v1 ? v + 1 : v0;
                const Seg e{xy[2 * v], xy[2 * v + 1], xy[2 * w], xy[2 * w + 1]};
                T->edges.push_back(e);
                b = unite(b, seg_box(e));
            }
        }
        T->edge_off[p + 1] = T->edges.size();
        pboxes.push_back(b);   // a polygon without vertices keeps an empty box
    }
    index_segments(T, T->edges);
    build_index(pboxes, T->nthreads, &T->poly);
    return T;
}

void cpu_rtree_free(void* t) { delete (Tree*)t; }

// RGBA tiles for requests (z, x, y, r16) as (n, 4) uint32.  style: line rgba,
// fill rgba (8 bytes; the alphas are unused).  Returns the threads used.
int cpu_rtree_render(void* tree, const uint32_t* reqs, uint64_t n_req, const uint8_t* style, uint8_t* out) {
    const Tree& T = *(const Tree*)tree;
    std::atomic<uint64_t> next{0};
    const uint64_t items = n_req * 256;
    std::vector<std::thread> th;
    for (int t = 0; t < T.nthreads; t++)
        th.emplace_back([&] {
            for (uint64_t it = next++; it < items; it = next++) {
                const uint64_t k = it / 256;
                const int j = (int)(it % 256);
                const uint32_t z = reqs[4 * k], tx = reqs[4 * k + 1], ty = reqs[4 * k + 2], r16 = reqs[4 * k + 3];
                const int64_t ps = 1ll << (23 - z), q = ps / 4, R = (int64_t)r16 << (19 - z), R2 = R * R;
                const int64_t X0 = -kHalf + (int64_t)tx * (1ll << (31 - z)), Y0 = -kHalf + (int64_t)ty * (1ll << (31 - z));
                const int64_t cy = Y0 + j * ps + ps / 2;
                uint8_t* row = out + k * 262144 + (uint64_t)j * 1024;
                for (int i = 0; i < 256; i++) {
                    const int64_t cx = X0 + i * ps + ps / 2;
                    int v = 0;
                    for (int s = 0; s < 4; s++) {
                        const int64_t sx = cx + ((s & 1) ? q : -q), sy = cy + ((s & 2) ? q : -q);
                        auto near = [&](const Box& b) { return box_dist2(b, sx, sy) <= R2; };
                        bool hit;
                        if (T.kind == kPoints) {
                            hit = query(T.obj, near, [](uint64_t) { return true; });   // a point is its own box
                        } else {
                            hit = query(T.obj, near, [&](uint64_t c) { return seg_within(T.seg[c], sx, sy, R2); });
                        }
                        v += hit;
                    }
                    bool filled = false;
                    if (T.kind == kPolygons) {
                        auto contains = [&](const Box& b) { return b.x0 <= cx && cx <= b.x1 && b.y0 <= cy && cy <= b.y1; };
                        filled = query(T.poly, contains, [&](uint64_t c) {
                            const uint32_t p = T.poly.id[c];
                            uint32_t parity = 0;
                            for (uint64_t e = T.edge_off[p]; e < T.edge_off[p + 1]; e++)
                                parity ^= crosses_right(T.edges[e], cx, cy) ? 1u : 0u;
                            return parity != 0;
                        });
                    }
                    uint8_t* px = row + 4 * i;
                    const uint32_t alpha = (255u * (uint32_t)v + 2u) >> 2;
                    if (filled) {
                        for (int c = 0; c < 3; c++)
                            px[c] = (uint8_t)((style[c] * alpha + style[4 + c] * (255u - alpha) + 127u) / 255u);
                        px[3] = 255;
                    } else if (v) {
                        px[0] = style[0]; px[1] = style[1]; px[2] = style[2];
                        px[3] = (uint8_t)alpha;
                    } else {
                        px[0] = px[1] = px[2] = px[3] = 0;
                    }
                }
            }
        });
    for (auto& x : th) x.join();
    return T.nthreads;
}

// Points, line colour only (kept for existing callers).
int cpu_rtree_render_rgba(void* tree, const uint32_t* reqs, uint64_t n_req, const uint8_t* rgb, uint8_t* out) {
    const uint8_t style[8] = {rgb[0], rgb[1], rgb[2], 0, 0, 0, 0, 0};
    return cpu_rtree_render(tree, reqs, n_req, style, out);
}

}  // extern "C"
