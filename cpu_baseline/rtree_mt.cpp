// Multithreaded CPU R-tree renderer: the paper's own pixel-driven method on
// the host cores, kept as a reported baseline for the GPU library (not used by
// it).  HiVision Sec. 3.2 / Algorithm 1 with the exact per-sample rule: each
// of a pixel's four super-samples asks the R-tree whether a point lies within
// R, stopping at the first hit; the tile rows are processed by a pool of
// threads that take (tile, row) items in turn (the row split of the paper's
// hybrid engine, Sec. 4.3).
//
// Points only (the headline workload).  Build: 62-bit Hilbert keys of the
// points, a parallel LSD radix sort, leaves of 32 points, inner nodes of 32
// child boxes.
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

struct Tree {
    std::vector<int32_t> px, py;            // sorted points
    std::vector<std::vector<Box>> levels;   // levels[0]: leaf boxes, levels[l]: boxes of level-l nodes
    int nthreads = 1;
};

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

Box unite(const Box& a, const Box& b) {
    return {std::min(a.x0, b.x0), std::min(a.y0, b.y0), std::max(a.x1, b.x1), std::max(a.y1, b.y1)};
}

// Is some point under entry `node` of levels[level] within R of (sx, sy)?
// Entries of levels[0] are leaves of 32 points; entries of levels[l] cover 32
// entries of levels[l - 1].
bool any_within(const Tree& T, int level, uint64_t node, int64_t sx, int64_t sy, int64_t R2) {
    const std::vector<Box>& below = level == 0 ? T.levels[0] : T.levels[level - 1];
    uint64_t c0 = node * 32, c1 = std::min<uint64_t>(c0 + 32, level == 0 ? T.px.size() : below.size());
    for (uint64_t c = c0; c < c1; c++) {
        if (level == 0) {
            int64_t dx = T.px[c] - sx, dy = T.py[c] - sy;
            if (dx * dx + dy * dy <= R2) return true;
            continue;
        }
        const Box& b = below[c];
        int64_t gx = std::max<int64_t>({0, (int64_t)b.x0 - sx, sx - (int64_t)b.x1});
        int64_t gy = std::max<int64_t>({0, (int64_t)b.y0 - sy, sy - (int64_t)b.y1});
        if (gx * gx + gy * gy <= R2 && any_within(T, level - 1, c, sx, sy, R2)) return true;
    }
    return false;
}

}  // namespace

extern "C" {

void* cpu_rtree_build(const int32_t* xy, uint64_t n, int nthreads) {
    Tree* T = new Tree();
    T->nthreads = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
    std::vector<uint64_t> key(n);
    std::vector<uint32_t> idx(n);
    parallel_for(T->nthreads, n, [&](uint64_t lo, uint64_t hi, int) {
        for (uint64_t i = lo; i < hi; i++) {
            key[i] = hilbert(xy[2 * i], xy[2 * i + 1]);
            idx[i] = (uint32_t)i;
        }
    });
    radix_sort(key, idx, T->nthreads);
    T->px.resize(n);
    T->py.resize(n);
    parallel_for(T->nthreads, n, [&](uint64_t lo, uint64_t hi, int) {
        for (uint64_t i = lo; i < hi; i++) {
            T->px[i] = xy[2 * idx[i]];
            T->py[i] = xy[2 * idx[i] + 1];
        }
    });
    // leaf boxes, then levels until a single root
    uint64_t nl = (n + 31) / 32;
    std::vector<Box> cur(nl);
    for (uint64_t l = 0; l < nl; l++) {
        Box b{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
        for (uint64_t i = l * 32; i < std::min<uint64_t>(n, l * 32 + 32); i++)
            b = unite(b, {T->px[i], T->py[i], T->px[i], T->py[i]});
        cur[l] = b;
    }
    T->levels.push_back(cur);
    while (T->levels.back().size() > 1) {
        const std::vector<Box>& c = T->levels.back();
        std::vector<Box> up((c.size() + 31) / 32, Box{INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN});
        for (uint64_t i = 0; i < c.size(); i++) up[i / 32] = unite(up[i / 32], c[i]);
        T->levels.push_back(up);
    }
    return T;
}

void cpu_rtree_free(void* t) { delete (Tree*)t; }

// RGBA tiles (the library's byte layout) for requests (z, x, y, r16) as
// (n, 4) uint32; line colour rgb.  Returns the threads used.
int cpu_rtree_render_rgba(void* tree, const uint32_t* reqs, uint64_t n_req, const uint8_t* rgb, uint8_t* out) {
    const Tree& T = *(const Tree*)tree;
    std::atomic<uint64_t> next{0};
    const uint64_t items = n_req * 256;
    const int top = (int)T.levels.size() - 1;
    std::vector<std::thread> th;
    for (int t = 0; t < T.nthreads; t++)
        th.emplace_back([&] {
            for (uint64_t it = next++; it < items; it = next++) {
                uint64_t k = it / 256;
                int j = (int)(it % 256);
                uint32_t z = reqs[4 * k], tx = reqs[4 * k + 1], ty = reqs[4 * k + 2], r16 = reqs[4 * k + 3];
                int64_t ps = 1ll << (23 - z), q = ps / 4, R = (int64_t)r16 << (19 - z), R2 = R * R;
                int64_t X0 = -kHalf + (int64_t)tx * (1ll << (31 - z)), Y0 = -kHalf + (int64_t)ty * (1ll << (31 - z));
                int64_t cy = Y0 + j * ps + ps / 2;
                uint8_t* row = out + k * 262144 + (uint64_t)j * 1024;
                for (int i = 0; i < 256; i++) {
                    int64_t cx = X0 + i * ps + ps / 2;
                    int v = 0;
                    if (!T.px.empty())
                        for (int s = 0; s < 4; s++)
                            v += any_within(T, top, 0, cx + ((s & 1) ? q : -q), cy + ((s & 2) ? q : -q), R2);
                    uint8_t* px = row + 4 * i;
                    if (v) {
                        px[0] = rgb[0]; px[1] = rgb[1]; px[2] = rgb[2];
                        px[3] = (uint8_t)((255 * v + 2) >> 2);
                    } else {
                        px[0] = px[1] = px[2] = px[3] = 0;
                    }
                }
            }
        });
    for (auto& x : th) x.join();
    return T.nthreads;
}

}  // extern "C"
