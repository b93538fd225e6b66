// Tile rendering: tile cull, warp-cooperative traversal with early exit,
// exact predicates and the output encode, fused in one kernel (one
// instantiation per layer kind).
//
//   HiVision Algorithm 1 (SIBV): a pixel's value is the number of its four
//   super-samples within distance R of some object (points, segments,
//   polygon edges); MASK mode decides the pixel centre only.
//   HiVision Algorithm 2 (SIBF): a pixel centre is filled when, for some
//   polygon whose box contains it, that polygon's edges cross the ray from
//   the centre an odd number of times.
//
// Work decomposition.  One CTA (8 warps) renders a strip of 256 x rows pixels
// of one tile (rows = 16 for large batches, 8 or 4 for small ones; batches
// too small to fill the GPU even then split each 4-row strip into 2 or 4
// column parts, one CTA each).  The CTA
// first culls the R-tree (or, with the learned index, the subtrees of the
// key ranges the model finds) against the strip's box expanded by R, breadth
// first, into a frontier of at most kFCap nodes in shared memory (the deepest
// level that fits), binned by 8-pixel block column.  Each warp then takes
// 8 x 4 pixel blocks (one pixel per lane, up to four samples per lane): it
// tests its column's frontier entries against its still-undecided samples,
// descends the intersecting subtrees depth first (a ballot over the 32 child
// boxes decides which children to visit; for points, children that certainly
// cover samples decide them on the spot), evaluates the exact predicate on
// the records of each visited leaf, and stops as soon as every sample of the
// block is decided.  Results go to a per-pixel byte array in shared memory;
// the epilogue encodes the strip (MASK bits, COVERAGE bytes or RGBA) with
// coalesced 16-byte stores.
#include "hv_device.cuh"
#include "hv_internal.h"
#include "hv_learned.cuh"

namespace hv {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kStripRows = 16;   // the largest strip; a launch picks 4, 8 or 16 rows
constexpr int kBW = 8, kBH = 4;
constexpr int kBlocksX = kTile / kBW;
constexpr int kFCap = 512;
constexpr int kBucketCap = 2048;   // keeps the static shared memory under 48 KiB
constexpr int kCullCells = 64;     // learned cull: at most this many Hilbert cells per strip
constexpr int kCullSub = kThreads / kCullCells;   // threads per cell
static_assert(kCullSub >= 2 && kCullSub <= 32 && (kCullSub & (kCullSub - 1)) == 0, "cell threads within a warp");
constexpr int kMaxPattern = 16;    // fill patterns: at most 16 x 16 texels

// result bits per pixel: bits 0-3 the outline's super-samples, bit 4 the
// centre, bits 5-7 the fill field (0: not filled; centre fill: 1; the
// anti-aliased fill: the number of super-samples inside, 0..4)
constexpr uint32_t kResCentre = 16u, kResFill = 32u;
constexpr int kResFillShift = 5;

struct TreeArg {
    const int32_t* nodes;
    uint64_t level_off[kMaxLevels + 1];
    uint64_t level_n[kMaxLevels + 1];
    int top;
    uint64_t n_obj;
    int4 root_box;
};

struct Params {
    const hv_tile_req* reqs;
    uint32_t n;
    int rows;                   // pixel rows per CTA strip: 4, 8 or 16
    int strips;                 // strips per tile (256 / rows)
    int cols;                   // pixel columns per CTA: 256, or 128 / 64 for batches too small to fill the GPU
    int parts;                  // CTAs per strip (256 / cols)
    int col_shift;              // log2(cols / 8): block columns per CTA as a shift
    const uint32_t* n_dev;      // if set, the batch size is min(*n_dev, n) (graph launches)
    int mode;
    int kind;
    uchar4 line;
    uchar4 fill;
    uint8_t* out;
    uint32_t tile_bytes;
    TreeArg tree;               // points, segments or polygon edges
    const void* obj;
    TreeArg mtree;              // polygon boxes (polygon layers)
    const int4* mbr_obj;
    const uint32_t* mbr_ids;
    const int4* poly_edges;
    const uint64_t* poly_edge_off;
    uint32_t* status;                 // bit 0: invalid request; bit 1: internal check failed
    unsigned long long* fault;        // first failed check: code << 56 | value
    uint64_t n_poly, n_edges;
    // learned candidate lookup (use_learned): models over the sorted keys of
    // the objects and of the polygon boxes, their halos and side trees
    int use_learned;
    int32_t R_units;            // >= 0: the radius of every tile (buffer analysis), else from r16
    // polygon fill style: anti-aliased fill, and a pattern of pat_w x pat_h
    // RGBA texels (0: none) laid over the global pixel grid
    int fill_aa;
    int pat_w, pat_h;
    const uchar4* pattern;      // device memory, pat_w * pat_h texels
    LModel lm, mlm;
    int32_t halo, mhalo;
    TreeArg side, mside;
    const void* side_obj;
    const uint32_t* side_ids;
    const int4* mside_obj;
    const uint32_t* mside_ids;
    // instrumentation (NULL in normal use): every node, leaf and polygon read
    // is appended as (tile << 38 | kind << 35 | id)
    unsigned long long* log;
    unsigned long long log_cap;
    unsigned long long* log_n;
    // phase profile (instrumented instantiation only): HV_PHASE_* counters
    unsigned long long* phases;
};

// Phase profile.  The instrumented instantiation (kProf) times the phases of
// every CTA with clock64() and adds them up over the launch, in warp-cycles:
// CTA-wide phases (one thread times them, every warp takes part) count their
// cycles times the warps of the CTA; block work counts each warp's own
// cycles.  The indices are the HV_PHASE_* values of the C header.
enum {
    kPTotal = 0, kPPrologue, kPCull, kPBin, kPBlocksCta, kPBlocksWarp, kPLeaf, kPDescend, kPEncode,
    kPCtas, kPBlocks, kPLeafVisits, kPNodeVisits, kPFrontierEntries, kPLeafEmpty, kPLeafDecided, kPN = 16
};

template <bool kProf>
__device__ __forceinline__ long long tick() {
    if constexpr (kProf) return clock64();
    return 0;
}

// outcome of a leaf visit (counted by the phase profile): no record in reach
// of an undecided sample, records tested without deciding one, a sample decided
constexpr uint32_t kVisitEmpty = 0, kVisitTested = 1, kVisitDecided = 2;

// kinds of logged reads
constexpr uint32_t kLogNode = 0, kLogLeaf = 1, kLogPolyNode = 2, kLogPolyLeaf = 3, kLogPoly = 4;

__device__ __forceinline__ void log_read(const Params& p, uint32_t kind, uint64_t id, int lane) {
    if (p.log != nullptr && lane == 0) {
        unsigned long long k = atomicAdd(p.log_n, 1ull);
        if (k < p.log_cap)
            p.log[k] = ((unsigned long long)(blockIdx.x / (p.strips * p.parts)) << 38) |
                       ((unsigned long long)kind << 35) | id;
    }
}

// Bounds checks on every index the traversal follows: a failure records the
// first offending value and the access is skipped (the tile is then wrong,
// never the memory).
__device__ __noinline__ void check_failed(const Params& p, uint32_t code, uint64_t v) {
    atomicCAS(p.fault, 0ull, ((unsigned long long)code << 56) | (v & ((1ull << 56) - 1)));
    atomicOr(p.status, 2u);
}

// The frontier is built in two buffers that the cull alternates; the pass
// over the blocks reads only the final one (f_buf), and the other serves the
// warps as scratch for segment leaves (Src::seg_scratch, pair_scratch) until
// the barrier that ends the pass.
struct Smem {
    uint8_t res[kStripRows * kTile];
    int4 fbox[2][kFCap];
    uint32_t fid[2][kFCap];
    const int32_t* lvl_base[2][kMaxLevels + 1];   // [0]: tree being traversed, [1]: its side tree
    uint32_t lvl_n[2][kMaxLevels + 1];            // nodes per level
    uint32_t stk_node[kWarps][kMaxLevels + 1];
    uint32_t stk_mask[kWarps][kMaxLevels + 1];
    uint32_t lanemask[kWarps][kMaxLevels + 1][32];
    // the frontier binned by 8-pixel block column: bucket c lists the entries
    // that can reach blocks of column c
    uint16_t bucket[kBucketCap];
    int bucket_off[kBlocksX + 1];
    int bucket_cur[kBlocksX];
    int binned;
    int f_count, f_level, f_buf, next_count, next_block;
    unsigned long long prof[kPN];   // phase profile of the CTA (kProf only)
};

// Add the cycles since t0 (or a count) to a phase counter of the CTA (one
// lane per warp).
template <bool kProf>
__device__ __forceinline__ void prof_add(Smem& sm, int k, unsigned long long v, int lane) {
    if constexpr (kProf) {
        if (lane == 0) atomicAdd(&sm.prof[k], v);
    }
}
template <bool kProf>
__device__ __forceinline__ void prof_since(Smem& sm, int k, long long t0, int lane) {
    if constexpr (kProf) prof_add<kProf>(sm, k, (unsigned long long)(clock64() - t0), lane);
}

// Where a traversal reads its objects: a tree's sorted objects (with polygon
// ids for polygon boxes) and the per-level node bases in shared memory.
struct Src {
    const void* obj;
    const uint32_t* ids;
    uint64_t n;
    const int32_t* nodes;        // node array (for the read log)
    const int32_t* const* lvl;   // lvl[l] = first node of level l
    const uint32_t* lvl_n;       // lvl_n[l] = nodes of level l
    int4* seg_scratch;           // per warp kSegScratch int4 (segment leaves)
    uint16_t* pair_scratch;      // per warp kPairCap pairs (segment leaves)
};

// Per-lane state of one 8 x 4 pixel block (lane l = pixel (l & 7, l >> 3)).
// Sample k of a lane sits at (cx -+ off, cy -+ off): bit 0 of k picks +x,
// bit 1 picks +y.  MASK mode and the fill use one sample, the centre.
struct Lane {
    int32_t cx, cy;        // pixel centre
    int32_t off;           // super-sample offset (0 in MASK mode and for fill)
    int32_t ext;           // reach of a lane's samples: R + off (Chebyshev)
    int64_t R2;
    uint32_t und;          // this lane's undecided samples (bit k: sample k)
    uint32_t Uk[4];        // warp-uniform: lanes whose sample k is undecided
    uint32_t U;            // warp-uniform: lanes with an undecided sample
    int nk;                // samples per lane (1 or 4)
    int32_t bx0, by0;      // warp-uniform: centre of the block's first pixel
    int32_t q;             // certain-cover half-side floor(R / sqrt 2) (points), else -1
    int L;                 // warp-uniform: log2 of the pixel size
    bool narrow;           // warp-uniform: R + 2 off <= kNarrow (32-bit distance tests)
};

// A sample that a box reaches in Chebyshev distance lies within ext + off =
// R + 2 off of it along each axis; with that at most kNarrow each squared
// gap is below 2^31 and the sum of two below 2^32, so squared distances of
// reachable samples are exact in unsigned 32-bit arithmetic.
constexpr int32_t kNarrow = 46340;   // floor(sqrt(2^31))


// Fold per-sample coverage masks (bit l: lane l's sample k was covered) into
// the warp's undecided state.
__device__ __forceinline__ void apply_cover(Lane& s, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            int lane) {
    s.Uk[0] &= ~c0;
    s.Uk[1] &= ~c1;
    s.Uk[2] &= ~c2;
    s.Uk[3] &= ~c3;
    s.U = s.Uk[0] | s.Uk[1] | s.Uk[2] | s.Uk[3];
    s.und = ((s.Uk[0] >> lane) & 1u) | (((s.Uk[1] >> lane) & 1u) << 1) | (((s.Uk[2] >> lane) & 1u) << 2) |
            (((s.Uk[3] >> lane) & 1u) << 3);
}

// Lanes of the block that have a sample within Chebyshev distance `ext` of
// the box [x0, x1] x [y0, y1]: a pixel column c qualifies when its centre
// lies in [x0 - ext, x1 + ext], i.e. ceil((x0-ext-bx0)/ps) <= c <=
// floor((x1+ext-bx0)/ps), and likewise for rows.  A necessary condition for
// any object inside the box to cover any of that lane's samples.
__device__ __forceinline__ uint32_t rect_lanes(const Lane& s, int32_t x0, int32_t y0, int32_t x1,
                                               int32_t y1) {
    // empty boxes and padding records lie outside the grid
    if (x0 > x1 || y0 > y1 || x0 < -kGridHalf || y0 < -kGridHalf) return 0u;
    // differences from the block origin fit 32 bits once clamped to +-2^30
    // (the reach is below 2^30, so farther boxes stay out of range)
    const int32_t ax = max(x0 - s.bx0, -kGridHalf) - s.ext, bx = min(x1 - s.bx0, kGridHalf) + s.ext;
    const int32_t ay = max(y0 - s.by0, -kGridHalf) - s.ext, by = min(y1 - s.by0, kGridHalf) + s.ext;
    const int32_t c0 = max(-((-ax) >> s.L), 0), c1 = min(bx >> s.L, 7);
    const int32_t r0 = max(-((-ay) >> s.L), 0), r1 = min(by >> s.L, 3);
    if (c0 > c1 || r0 > r1) return 0u;
    uint32_t col = (0xFFu << c0) & (0xFFu >> (7 - c1));
    uint32_t rows = (0x01010101u << (8 * r0)) & (0x01010101u >> (8 * (3 - r1)));
    return col * rows;
}

// Does the box [x0, x1] x [y0, y1] come within Euclidean distance R of an
// undecided sample of one of the lanes in `cand`?  Exact for every sample;
// stops at the first that qualifies.
template <bool kNarrowOk>
__device__ __forceinline__ bool round_reach(const Lane& s, int32_t x0, int32_t y0, int32_t x1,
                                            int32_t y1, uint32_t cand) {
    // box edges relative to the block's first pixel centre, clamped to
    // +-2^30 (32-bit arithmetic below): a clamped edge lies more than
    // 2^30 - 2^26 > R from every sample, so it never decides a gap within R
    const int32_t ax = max(min(x0 - s.bx0, kGridHalf), -kGridHalf), bx = max(min(x1 - s.bx0, kGridHalf), -kGridHalf);
    const int32_t ay = max(min(y0 - s.by0, kGridHalf), -kGridHalf), by = max(min(y1 - s.by0, kGridHalf), -kGridHalf);
    if (kNarrowOk && s.narrow) {
        // lanes in cand reach the box in Chebyshev distance: every gap below
        // is at most R + 2 off
        const uint32_t R2 = (uint32_t)s.R2;
        while (cand) {
            int l = __ffs(cand) - 1;
            cand &= cand - 1;
            const int32_t sx = (l & 7) << s.L, sy = (l >> 3) << s.L;
            const uint32_t gxm = (uint32_t)max(max(ax - (sx - s.off), (sx - s.off) - bx), 0);
            const uint32_t gxp = (uint32_t)max(max(ax - (sx + s.off), (sx + s.off) - bx), 0);
            const uint32_t gym = (uint32_t)max(max(ay - (sy - s.off), (sy - s.off) - by), 0);
            const uint32_t gyp = (uint32_t)max(max(ay - (sy + s.off), (sy + s.off) - by), 0);
            const uint32_t xm = gxm * gxm, xp = gxp * gxp, ym = gym * gym, yp = gyp * gyp;
            const bool h0 = (s.Uk[0] >> l) & 1u && xm + ym <= R2;
            const bool h1 = (s.Uk[1] >> l) & 1u && xp + ym <= R2;
            const bool h2 = (s.Uk[2] >> l) & 1u && xm + yp <= R2;
            const bool h3 = (s.Uk[3] >> l) & 1u && xp + yp <= R2;
            if (h0 | h1 | h2 | h3) return true;
        }
        return false;
    }
    while (cand) {
        int l = __ffs(cand) - 1;
        cand &= cand - 1;
        const int32_t sx = (l & 7) << s.L, sy = (l >> 3) << s.L;
        const uint32_t gxm = (uint32_t)max(max(ax - (sx - s.off), (sx - s.off) - bx), 0);
        const uint32_t gxp = (uint32_t)max(max(ax - (sx + s.off), (sx + s.off) - bx), 0);
        const uint32_t gym = (uint32_t)max(max(ay - (sy - s.off), (sy - s.off) - by), 0);
        const uint32_t gyp = (uint32_t)max(max(ay - (sy + s.off), (sy + s.off) - by), 0);
        const uint64_t xm = (uint64_t)gxm * gxm, xp = (uint64_t)gxp * gxp;
        const uint64_t ym = (uint64_t)gym * gym, yp = (uint64_t)gyp * gyp;
        const uint64_t R2 = (uint64_t)s.R2;
        const bool h0 = (s.Uk[0] >> l) & 1u && xm + ym <= R2;
        const bool h1 = (s.Uk[1] >> l) & 1u && xp + ym <= R2;
        const bool h2 = (s.Uk[2] >> l) & 1u && xm + yp <= R2;
        const bool h3 = (s.Uk[3] >> l) & 1u && xp + yp <= R2;
        if (h0 | h1 | h2 | h3) return true;
    }
    return false;
}

// Samples that a non-empty box of points certainly covers: a sample within
// Chebyshev distance q of every point of the box, with 2 q^2 <= R^2, is
// within Euclidean distance R of each of them, whatever the points are.  Per
// sample k, the lanes whose sample k lies in [x1 - q, x0 + q] x [y1 - q,
// y0 + q] (undecided ones only).  Exact: no sample is marked that the
// predicate would not cover, so no output depends on it.
__device__ __forceinline__ void certain_lanes(const Lane& s, int32_t x0, int32_t y0, int32_t x1, int32_t y1,
                                              uint32_t m[4]) {
    m[0] = m[1] = m[2] = m[3] = 0u;
    if (x0 > x1 || y0 > y1 || x0 < -kGridHalf || y0 < -kGridHalf) return;
    // clamping the differences only narrows the interval (conservative)
    const int32_t lx = max(x1 - s.bx0, -kGridHalf) - s.q, hx = min(x0 - s.bx0, kGridHalf) + s.q;
    const int32_t ly = max(y1 - s.by0, -kGridHalf) - s.q, hy = min(y0 - s.by0, kGridHalf) + s.q;
    if (lx > hx || ly > hy) return;   // the box is wider than 2q
    uint32_t col[2], row[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        // sample offset -off (k = 0) or +off (k = 1) from the pixel centre
        const int32_t o = k ? -s.off : s.off;
        const int32_t c0 = max(-((-(lx + o)) >> s.L), 0), c1 = min((hx + o) >> s.L, 7);
        const int32_t r0 = max(-((-(ly + o)) >> s.L), 0), r1 = min((hy + o) >> s.L, 3);
        col[k] = c0 > c1 ? 0u : (0xFFu << c0) & (0xFFu >> (7 - c1));
        row[k] = r0 > r1 ? 0u : (0x01010101u << (8 * r0)) & (0x01010101u >> (8 * (3 - r1)));
    }
#pragma unroll
    for (int k = 0; k < 4; k++) m[k] = (col[k & 1] * row[k >> 1]) & s.Uk[k];
}

// Each lane offers one box (a child of the node being visited); the samples
// any of them certainly covers are decided for the whole warp.
__device__ __forceinline__ void certain_cover(Lane& s, int32_t x0, int32_t y0, int32_t x1, int32_t y1, int lane) {
    if (s.q < 0) return;
    uint32_t m[4];
    certain_lanes(s, x0, y0, x1, y1, m);
    if (!__any_sync(kFull, (m[0] | m[1] | m[2] | m[3]) != 0u)) return;
    apply_cover(s, __reduce_or_sync(kFull, m[0]), __reduce_or_sync(kFull, m[1]), __reduce_or_sync(kFull, m[2]),
                __reduce_or_sync(kFull, m[3]), lane);
}

// Lanes `cm` can reach and one of their undecided samples really is within
// reach.  For the fill (R = 0, centres) the Chebyshev test is already exact.
template <class V>
__device__ __forceinline__ bool reaches(const Lane& s, uint32_t cm, int32_t x0, int32_t y0, int32_t x1, int32_t y1) {
    uint32_t cand = cm & s.U;
    if (!cand) return false;
    return V::kFill || round_reach<V::kNarrowReach>(s, x0, y0, x1, y1, cand);
}

// One box against the lanes' own undecided samples (lanes in `lanes` only,
// each lane its four samples, no loop): whether the box comes within R of
// any of them.  The same exact test as round_reach, transposed.
template <bool kNarrowOk>
__device__ __forceinline__ bool box_reach_lanes(const Lane& s, int32_t x0, int32_t y0, int32_t x1, int32_t y1,
                                                uint32_t lanes, int lane) {
    bool hit = false;
    if ((lanes >> lane) & 1u) {
        const int32_t ax = max(min(x0 - s.bx0, kGridHalf), -kGridHalf), bx = max(min(x1 - s.bx0, kGridHalf), -kGridHalf);
        const int32_t ay = max(min(y0 - s.by0, kGridHalf), -kGridHalf), by = max(min(y1 - s.by0, kGridHalf), -kGridHalf);
        const int32_t sx = (lane & 7) << s.L, sy = (lane >> 3) << s.L;
        const uint32_t gxm = (uint32_t)max(max(ax - (sx - s.off), (sx - s.off) - bx), 0);
        const uint32_t gxp = (uint32_t)max(max(ax - (sx + s.off), (sx + s.off) - bx), 0);
        const uint32_t gym = (uint32_t)max(max(ay - (sy - s.off), (sy - s.off) - by), 0);
        const uint32_t gyp = (uint32_t)max(max(ay - (sy + s.off), (sy + s.off) - by), 0);
        if (kNarrowOk && s.narrow) {
            // the lane is in the box's Chebyshev reach: gaps at most R + 2 off
            const uint32_t R2 = (uint32_t)s.R2;
            const uint32_t xm = gxm * gxm, xp = gxp * gxp, ym = gym * gym, yp = gyp * gyp;
            hit = ((s.und & 1u) && xm + ym <= R2) || ((s.und & 2u) && xp + ym <= R2) ||
                  ((s.und & 4u) && xm + yp <= R2) || ((s.und & 8u) && xp + yp <= R2);
        } else {
            const uint64_t R2 = (uint64_t)s.R2;
            const uint64_t xm = (uint64_t)gxm * gxm, xp = (uint64_t)gxp * gxp;
            const uint64_t ym = (uint64_t)gym * gym, yp = (uint64_t)gyp * gyp;
            hit = ((s.und & 1u) && xm + ym <= R2) || ((s.und & 2u) && xp + ym <= R2) ||
                  ((s.und & 4u) && xm + yp <= R2) || ((s.und & 8u) && xp + yp <= R2);
        }
    }
    return __any_sync(kFull, hit);
}

// Pixels of the block whose centre lies within E of the segment's line,
// E = R + 2 off + slack >= R + off * sqrt 2 (a covered sample's pixel centre
// is that close): in pixel row r the centres (c ps, r ps), relative to the
// block's first centre, satisfy |c A + K_r| <= B with A = ps dy,
// K_r = cross((0, r ps) - P, d), B = E |d|, P a point within 2 units of the
// line (the centre of the piece box: a piece runs corner to corner of it).
// Single precision with every bound widened by more than its rounding error
// (relative 2^-20 of the magnitudes involved, plus a column): a superset of
// the pixels the exact test can cover.
__device__ __forceinline__ uint32_t line_lanes(const Lane& s, int32_t px, int32_t py, int32_t dx, int32_t dy) {
    const float fdx = (float)dx, fdy = (float)dy, fpx = (float)px, fpy = (float)py;
    const float dn = sqrtf(fmaf(fdx, fdx, fdy * fdy));
    const float E = (float)(s.ext + s.off + 2) + (fabsf(fpx) + fabsf(fpy)) * 0x1p-22f;
    const float B = E * dn * (1.0f + 0x1p-20f);
    const float ps = (float)(1 << s.L);
    const float A = ps * fdy;
    const float inv = A != 0.f ? 1.0f / A : 0.f;
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < kBH; r++) {
        const float t1 = -fpx * fdy, t2 = fmaf((float)r, ps, -fpy) * fdx;
        const float K = t1 - t2;
        const float mag = fabsf(t1) + fabsf(t2) + B;
        uint32_t row;
        if (A == 0.f) {
            row = fabsf(K) <= B + mag * 0x1p-20f ? 0xFFu : 0u;
        } else {
            float lo = (-B - K) * inv, hi = (B - K) * inv;
            if (inv < 0.f) {
                const float t = lo;
                lo = hi;
                hi = t;
            }
            const float err = fmaf(mag * fabsf(inv), 0x1p-20f, 1.0f) + (fabsf(lo) + fabsf(hi)) * 0x1p-20f;
            lo = fmaxf(lo - err, -1.f);
            hi = fminf(hi + err, 8.f);
            const int c0 = max((int)ceilf(lo), 0), c1 = min((int)floorf(hi), 7);
            row = c0 <= c1 ? (0xFFu << c0) & (0xFFu >> (7 - c1)) : 0u;
        }
        m |= row << (8 * r);
    }
    return m;
}

// Pixels of the block whose centre the edge e crosses strictly to the right
// (Algorithm 2's ray test, half-open straddle in y): per pixel row the
// orientation num(c) = dx (y - ly) - (x_c - lx) dy of the edge ordered by y
// falls as the column c grows, so the crossed columns are a prefix 0..t-1,
// t found by a three-step binary search with exact 64-bit products.
// (ox, oy) offsets the samples from the pixel centres (the anti-aliased
// fill's super-samples); the column search is the same.
__device__ __forceinline__ uint32_t crossing_columns(int4 e, const Lane& s, int32_t ox = 0, int32_t oy = 0) {
    int32_t lx = e.x, ly = e.y, hx = e.z, hy = e.w;
    if (ly > hy) {
        lx = e.z; ly = e.w; hx = e.x; hy = e.y;
    }
    if (ly == hy) return 0u;   // a level edge straddles no scanline
    const int32_t ex = hx - lx, ey = hy - ly;
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < kBH; r++) {
        const int32_t y = s.by0 + (r << s.L) + oy;
        if (y < ly || y >= hy) continue;
        const int64_t n0 = (int64_t)ex * (y - ly) - ((int64_t)s.bx0 + ox - lx) * ey;
        // column c is crossed iff n0 > c ps ey
        int t = n0 > (int64_t)(3 << s.L) * ey ? 4 : 0;
        if (n0 > (int64_t)((t + 1) << s.L) * ey) t += 2;
        if (n0 > (int64_t)(t << s.L) * ey) t += 1;
        if (t == 7 && n0 > (int64_t)(7 << s.L) * ey) t = 8;
        m |= ((1u << t) - 1u) << (8 * r);
    }
    return m;
}

// ---- leaf visitors -----------------------------------------------------------
// Points and segments: each lane takes one object of the leaf and evaluates
// the exact predicate on the undecided samples within its reach; the
// per-sample hits are OR-reduced over the warp.

struct PointLeaf {
    static constexpr bool kFill = false;
    static constexpr bool kCertain = true;   // boxes of points certainly cover nearby samples
    static constexpr bool kOutline = false;
    static constexpr bool kNarrowReach = true;   // 32-bit node tests when R + 2 off is small
    // frontier entries and children filtered exactly when listed, by their
    // Chebyshev reach when taken (see blocks_pass)
    static constexpr bool kExactWhenTaken = false, kScanChebyshev = false, kChildChebyshev = false;
    static constexpr bool kOneVisitSite = false;
    __device__ static uint32_t visit(const Params& p, const Src& src, uint32_t leaf, Lane& s, int lane) {
        if ((uint64_t)leaf * 32 >= src.n) {
            if (lane == 0) check_failed(p, 4, leaf);
            return kVisitEmpty;
        }
        uint64_t i = (uint64_t)leaf * 32 + lane;
        log_read(p, kLogLeaf, leaf, lane);
        int2 o = make_int2(kEmptyHi, kEmptyHi);
        if (i < src.n) o = __ldg((const int2*)src.obj + i);
        // the exact test on the undecided samples in each point's reach
        uint32_t pm = rect_lanes(s, o.x, o.y, o.x, o.y) & s.U;
        if (!__any_sync(kFull, pm != 0)) return kVisitEmpty;
        const uint32_t U_before = s.U;
        // the point relative to the block's first pixel centre; lanes in pm
        // are within reach, so the 32-bit differences below are exact
        const int32_t dxo = max(min(o.x - s.bx0, kGridHalf), -kGridHalf);
        const int32_t dyo = max(min(o.y - s.by0, kGridHalf), -kGridHalf);
        const uint64_t R2 = (uint64_t)s.R2;
        uint32_t c[4] = {0u, 0u, 0u, 0u};
        if (s.narrow) {
            // lanes in pm lie within ext of the point along each axis, so
            // |dx -+ off|, |dy -+ off| <= R + 2 off <= kNarrow
            const uint32_t R2n = (uint32_t)R2;
            if (s.nk == 1) {
                while (pm) {
                    int l = __ffs(pm) - 1;
                    pm &= pm - 1;
                    const int32_t dx = dxo - ((l & 7) << s.L), dy = dyo - ((l >> 3) << s.L);
                    if ((uint32_t)(dx * dx) + (uint32_t)(dy * dy) <= R2n) c[0] |= 1u << l;
                }
            } else {
                while (pm) {
                    int l = __ffs(pm) - 1;
                    pm &= pm - 1;
                    const int32_t dx = dxo - ((l & 7) << s.L), dy = dyo - ((l >> 3) << s.L);
                    const uint32_t xm = (uint32_t)((dx + s.off) * (dx + s.off));
                    const uint32_t xp = (uint32_t)((dx - s.off) * (dx - s.off));
                    const uint32_t ym = (uint32_t)((dy + s.off) * (dy + s.off));
                    const uint32_t yp = (uint32_t)((dy - s.off) * (dy - s.off));
                    const uint32_t bit = 1u << l;
                    if (xm + ym <= R2n) c[0] |= bit;
                    if (xp + ym <= R2n) c[1] |= bit;
                    if (xm + yp <= R2n) c[2] |= bit;
                    if (xp + yp <= R2n) c[3] |= bit;
                }
            }
        } else if (s.nk == 1) {
            while (pm) {
                int l = __ffs(pm) - 1;
                pm &= pm - 1;
                const int32_t dx = dxo - ((l & 7) << s.L), dy = dyo - ((l >> 3) << s.L);
                if ((uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) <= R2) c[0] |= 1u << l;
            }
        } else {
            while (pm) {
                int l = __ffs(pm) - 1;
                pm &= pm - 1;
                // point minus sample: sample k sits at -+off in x (bit 0) and y (bit 1)
                const int32_t dx = dxo - ((l & 7) << s.L), dy = dyo - ((l >> 3) << s.L);
                const uint64_t xm = (uint64_t)((int64_t)(dx + s.off) * (dx + s.off));
                const uint64_t xp = (uint64_t)((int64_t)(dx - s.off) * (dx - s.off));
                const uint64_t ym = (uint64_t)((int64_t)(dy + s.off) * (dy + s.off));
                const uint64_t yp = (uint64_t)((int64_t)(dy - s.off) * (dy - s.off));
                const uint32_t bit = 1u << l;
                if (xm + ym <= R2) c[0] |= bit;
                if (xp + ym <= R2) c[1] |= bit;
                if (xm + yp <= R2) c[2] |= bit;
                if (xp + yp <= R2) c[3] |= bit;
            }
        }
        // decided samples may be hit again: apply_cover only clears bits
        const uint32_t c0 = __reduce_or_sync(kFull, c[0]), c1 = __reduce_or_sync(kFull, c[1]);
        const uint32_t c2 = __reduce_or_sync(kFull, c[2]), c3 = __reduce_or_sync(kFull, c[3]);
        apply_cover(s, c0, c1, c2, c3, lane);
        return (c0 | c1 | c2 | c3) & U_before ? kVisitDecided : kVisitTested;
    }
};

// Per warp, a segment leaf's pieces (their screen parameters, below) and its
// (piece, pixel) pairs in reach are staged
// in shared memory, and the warp's lanes take the pairs in turn: a leaf whose
// few pieces in reach each reach many pixels costs ceil(pairs / 32) rounds of
// exact tests instead of the largest piece's pixel count.
constexpr int kSegScratch = 64;   // 16-byte slots per warp: two per piece
constexpr int kPairCap = 128;     // pairs per warp and round of staging
static_assert(kSegScratch * kWarps <= kFCap, "segment scratch exceeds a frontier buffer");
static_assert(kPairCap * kWarps * 2 <= kFCap * 4, "pair scratch exceeds a frontier id buffer");

template <bool kLineLayer>
struct SegLeaf {
    static constexpr bool kFill = false;
    static constexpr bool kCertain = false;
    static constexpr bool kOutline = !kLineLayer;   // the outline of a polygon layer
    static constexpr bool kNarrowReach = false;
    // frontier entries listed by their Chebyshev reach, tested exactly when
    // taken (measured faster for segments, slower for points)
    static constexpr bool kExactWhenTaken = true, kScanChebyshev = true, kChildChebyshev = false;
    static constexpr bool kOneVisitSite = !kLineLayer;   // polygon outlines
    __device__ static uint32_t visit(const Params& p, const Src& src, uint32_t leaf, Lane& s, int lane) {
        if ((uint64_t)leaf * 32 >= src.n) {
            if (lane == 0) check_failed(p, 4, leaf);
            return kVisitEmpty;
        }
        uint64_t i = (uint64_t)leaf * 32 + lane;
        log_read(p, kLogLeaf, leaf, lane);
        // a record is a piece: the whole segment and the box of its piece
        int4 o = make_int4(0, 0, 0, 0);   // padding: never in reach (empty piece box)
        int4 pb = make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
        if (i < src.n) {
            o = __ldg((const int4*)src.obj + 2 * i);
            pb = __ldg((const int4*)src.obj + 2 * i + 1);
        }
        const int32_t sx0 = pb.x, sy0 = pb.y, sx1 = pb.z, sy1 = pb.w;
        uint32_t pm = rect_lanes(s, sx0, sy0, sx1, sy1) & s.U;
        if (!__any_sync(kFull, pm != 0)) return kVisitEmpty;
        const uint32_t U_before = s.U;
        // a piece box much larger than the pixels: keep the pixels near the line
        if (__reduce_max_sync(kFull, (uint32_t)__popc(pm)) > 8u)
            pm &= line_lanes(s, mid32(sx0, sx1) - s.bx0, mid32(sy0, sy1) - s.by0, o.z - o.x, o.w - o.y);
        // the segment relative to the block's first pixel centre (grid
        // coordinates lie in [-2^30, 2^30), so the differences fit 32 bits);
        // 32-bit products when both endpoints are within 2^30 of it, else the
        // absolute 64-bit test
        const int32_t ax = o.x - s.bx0, ay = o.y - s.by0, bx = o.z - s.bx0, by = o.w - s.by0;
        const bool near = max(max(abs(ax), abs(ay)), max(abs(bx), abs(by))) <= kGridHalf;
        uint32_t c[4] = {0u, 0u, 0u, 0u};
        if (__any_sync(kFull, pm != 0 && !near)) {
            // a segment reaching from beyond 2^30 of the block (grid-spanning
            // edges at low zoom): each lane its own piece, absolute 64-bit tests
            while (pm) {
                const int l = __ffs(pm) - 1;
                pm &= pm - 1;
                const int32_t px = (l & 7) << s.L, py = (l >> 3) << s.L;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (k < s.nk && ((s.Uk[k] >> l) & 1u)) {
                        const int32_t sx = s.bx0 + px + ((k & 1) ? s.off : -s.off);
                        const int32_t sy = s.by0 + py + ((k & 2) ? s.off : -s.off);
                        if (segment_within(o.x, o.y, o.z, o.w, sx, sy, s.R2)) c[k] |= 1u << l;
                    }
                }
            }
            return finish(s, c, U_before, lane);
        }
        const int warp = threadIdx.x >> 5;
        int4* const seg = src.seg_scratch + warp * kSegScratch;
        uint16_t* const pairs = src.pair_scratch + warp * kPairCap;
        // single-precision screen of the distance test.  Per piece, from exact
        // int64 values rounded once: the unit direction m = d / |d|, the
        // line's offset c0 = (d x a) / |d| and the projection offset
        // e0 = (d . a) / |d|, so that a sample s (relative to the block, its
        // coordinates exact in single precision) lies at signed distance
        // m x s - c0 from the line and at m . s - e0 along it from a; the
        // distance to the closed segment is then |(along - clamp(along, 0,
        // |d|), across)|.  Every rounding is bounded by 8 units in the last
        // place of the magnitudes involved (|s| <= 8 ps, |c0|, |e0|, |d|, R);
        // E1 takes 64 of them plus 2 grid units, and the squared thresholds
        // another 2^-20: a sample closer than R - E1 is within R, one farther
        // than R + E1 beyond it, and only the rest is decided exactly.
        {
            const int32_t dx = o.z - o.x, dy = o.w - o.y;
            const int64_t Ls = (int64_t)dx * dx + (int64_t)dy * dy;
            float mx = 1.f, my = 0.f, c0 = (float)ay, e0 = (float)ax, D = 0.f;   // a point: any direction
            if (Ls > 0) {
                D = sqrtf((float)Ls);
                const float inv = 1.0f / D;
                mx = (float)dx * inv;
                my = (float)dy * inv;
                c0 = (float)((int64_t)dx * ay - (int64_t)dy * ax) * inv;
                e0 = (float)((int64_t)dx * ax + (int64_t)dy * ay) * inv;
            }
            const float fR = (float)(s.ext - s.off);
            const float E1 = fmaf(0x1p-18f, 32.f * (float)(1 << s.L) + fabsf(c0) + fabsf(e0) + D + fR, 2.f);
            const float lo = fR - E1, hi = fR + E1;
            const float lo2 = lo > 0.f ? lo * lo * (1.f - 0x1p-20f) : -1.f;
            const float hi2 = hi * hi * (1.f + 0x1p-20f);
            reinterpret_cast<float4*>(seg)[lane] = make_float4(mx, my, c0, e0);
            reinterpret_cast<float4*>(seg + 32)[lane] = make_float4(D, lo2, hi2, 0.f);
        }
        // the lane's pairs are numbered first .. first + popc(pm) - 1
        const uint32_t cnt = (uint32_t)__popc(pm);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31), first = incl - cnt;
        const uint32_t tag = (uint32_t)lane << 5;
        for (uint32_t w0 = 0; w0 < total; w0 += kPairCap) {
            uint32_t m = pm, g = first - w0;   // unsigned: pairs before the round wrap above kPairCap
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                if (g < (uint32_t)kPairCap) pairs[g] = (uint16_t)(tag | (uint32_t)l);
                g++;
            }
            __syncwarp();
            const uint32_t n = min(total - w0, (uint32_t)kPairCap);
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t e = pairs[j];
                const int l = e & 31, pc = e >> 5;
                const float4 A = reinterpret_cast<const float4*>(seg)[pc];
                const float4 B = reinterpret_cast<const float4*>(seg + 32)[pc];
                // the pixel's column and row as exact floats (2^23 + c - 2^23)
                const float col = __int_as_float(0x4B000000 | (l & 7)) - 8388608.f;
                const float row = __int_as_float(0x4B000000 | (l >> 3)) - 8388608.f;
                const float fps = (float)(1 << s.L), foff = (float)s.off;
                const float sxs[2] = {fmaf(col, fps, -foff), fmaf(col, fps, foff)};
                const float sys[2] = {fmaf(row, fps, -foff), fmaf(row, fps, foff)};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (k < s.nk && ((s.Uk[k] >> l) & 1u)) {
                        const float sx = sxs[k & 1], sy = sys[k >> 1];
                        const float across = fmaf(A.x, sy, -fmaf(A.y, sx, A.z));
                        const float along = fmaf(A.x, sx, fmaf(A.y, sy, -A.w));
                        const float u = along - fminf(fmaxf(along, 0.f), B.x);
                        const float q = fmaf(u, u, across * across);
                        bool hit = q < B.y;
                        if (!hit && q <= B.z) {
                            // within the margin: the exact test on the piece's segment
                            const int4 og = __ldg((const int4*)src.obj + 2 * ((uint64_t)leaf * 32 + pc));
                            const int32_t gx = og.x - s.bx0, gy = og.y - s.by0, hx = og.z - s.bx0, hy = og.w - s.by0;
                            const int32_t dx = og.z - og.x, dy = og.w - og.y;
                            const int32_t isx = ((l & 7) << s.L) + ((k & 1) ? s.off : -s.off);
                            const int32_t isy = ((l >> 3) << s.L) + ((k & 2) ? s.off : -s.off);
                            hit = segment_within_rel(gx, gy, hx, hy, dx, dy, (int64_t)dx * dx + (int64_t)dy * dy, -1,
                                                     INT64_MAX, isx, isy, s.R2);
                        }
                        if (hit) c[k] |= 1u << l;
                    }
                }
            }
            __syncwarp();
        }
        return finish(s, c, U_before, lane);
    }

    // Fold the lanes' hits into the warp's undecided state.
    __device__ static uint32_t finish(Lane& s, const uint32_t c[4], uint32_t U_before, int lane) {
        const uint32_t c0 = __reduce_or_sync(kFull, c[0]), c1 = __reduce_or_sync(kFull, c[1]);
        const uint32_t c2 = __reduce_or_sync(kFull, c[2]), c3 = __reduce_or_sync(kFull, c[3]);
        apply_cover(s, c0, c1, c2, c3, lane);
        return (c0 | c1 | c2 | c3) & U_before ? kVisitDecided : kVisitTested;
    }
};

// Polygon boxes: a leaf holds 32 polygon boxes; for each box that contains an
// unfilled pixel centre, count that polygon's own edges crossing the ray.
struct FillLeaf {
    static constexpr bool kFill = true;
    static constexpr bool kCertain = false;
    static constexpr bool kOutline = false;
    static constexpr bool kNarrowReach = false;
    // R = 0 at the centres: the Chebyshev test is already exact
    static constexpr bool kExactWhenTaken = false, kScanChebyshev = false, kChildChebyshev = false;
    static constexpr bool kOneVisitSite = true;
    __device__ static uint32_t visit(const Params& p, const Src& src, uint32_t leaf, Lane& s, int lane) {
        if ((uint64_t)leaf * 32 >= src.n) {
            if (lane == 0) check_failed(p, 4, leaf);
            return kVisitEmpty;
        }
        uint64_t i = (uint64_t)leaf * 32 + lane;
        log_read(p, kLogPolyLeaf, leaf, lane);
        int4 b = make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
        uint32_t id = 0;
        if (i < src.n) {
            b = __ldg((const int4*)src.obj + i);
            id = __ldg(src.ids + i);
        }
        uint32_t pm = rect_lanes(s, b.x, b.y, b.z, b.w);
        uint32_t m = __ballot_sync(kFull, (pm & s.U) != 0);
        uint32_t outcome = m ? kVisitTested : kVisitEmpty;
        const uint32_t U_before = s.U;
        while (m) {
            int k = __ffs(m) - 1;
            m &= m - 1;
            int32_t bx0 = __shfl_sync(kFull, b.x, k), by0 = __shfl_sync(kFull, b.y, k);
            int32_t bx1 = __shfl_sync(kFull, b.z, k), by1 = __shfl_sync(kFull, b.w, k);
            uint32_t pid = __shfl_sync(kFull, id, k);
            // a sample of the lane (the centre, or a super-sample within off
            // of it) may lie in the box
            bool active = s.und && s.cx + s.off >= bx0 && s.cx - s.off <= bx1 && s.cy + s.off >= by0 &&
                          s.cy - s.off <= by1;
            if (__ballot_sync(kFull, active) == 0) continue;
            log_read(p, kLogPoly, pid, lane);
            if (pid >= p.n_poly) {
                if (lane == 0) check_failed(p, 5, pid);
                continue;
            }
            uint64_t e0 = __ldg(p.poly_edge_off + pid), e1 = __ldg(p.poly_edge_off + pid + 1);
            if (e0 > e1 || e1 > p.n_edges) {
                if (lane == 0) check_failed(p, 6, ((uint64_t)pid << 24) | (e1 & 0xffffff));
                continue;
            }
            // each lane takes an edge; the crossed pixels of all the edges,
            // XOR-reduced, are every pixel's parity at once (per sample)
            uint32_t inside = 0u;
            if (s.nk == 1) {
                uint32_t par = 0u;
                for (uint64_t base = e0; base < e1; base += 32) {
                    uint32_t cm = 0u;
                    if (base + lane < e1) cm = crossing_columns(__ldg(p.poly_edges + base + lane), s);
                    par ^= __reduce_xor_sync(kFull, cm);
                }
                inside = (par >> lane) & 1u;
            } else {
                // super-sample k sits at -+off in x (bit 0) and y (bit 1)
                uint32_t par[4] = {0u, 0u, 0u, 0u};
                for (uint64_t base = e0; base < e1; base += 32) {
                    int4 e = make_int4(0, 0, 0, 0);   // a level edge crosses nothing
                    if (base + lane < e1) e = __ldg(p.poly_edges + base + lane);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        par[k] ^= __reduce_xor_sync(kFull, crossing_columns(e, s, (k & 1) ? s.off : -s.off,
                                                                            (k & 2) ? s.off : -s.off));
                }
#pragma unroll
                for (int k = 0; k < 4; k++) inside |= ((par[k] >> lane) & 1u) << k;
            }
            if (active) s.und &= ~inside;
            uint32_t U2 = __ballot_sync(kFull, s.und != 0);
            if (U2 != s.U) {
                s.U = U2;
                s.Uk[0] = U2;
                m &= __ballot_sync(kFull, (pm & U2) != 0);
            }
        }
        return s.U != U_before ? kVisitDecided : outcome;
    }
};

// Child boxes of one inner node: lane c computes the lanes child c can
// reach, keeps it in `lm`, and the ballot selects the children to visit.
// Point trees first decide the samples the children certainly cover.
template <class V>
__device__ __forceinline__ uint32_t child_hits(const Params& p, const Src& src,
                                               const int32_t* base, Lane& s, int lane, uint32_t* lm) {
    if (p.log != nullptr)
        log_read(p, V::kFill ? kLogPolyNode : kLogNode, (uint64_t)(base - src.nodes) >> 7, lane);
    int32_t x0 = __ldg(base + lane), y0 = __ldg(base + 32 + lane);
    int32_t x1 = __ldg(base + 64 + lane), y1 = __ldg(base + 96 + lane);
    certain_cover(s, x0, y0, x1, y1, lane);
    uint32_t cm = rect_lanes(s, x0, y0, x1, y1);
    lm[lane] = cm;
    if constexpr (V::kChildChebyshev)
        return __ballot_sync(kFull, (cm & s.U) != 0u);
    else
        return __ballot_sync(kFull, reaches<V>(s, cm, x0, y0, x1, y1));
}

// Depth-first descent from node `node` at level `level` (>= 1).  The stack
// keeps, per level, the node whose children are being visited, the children
// still to visit, and each child's lane reach (re-tested against the
// shrinking undecided set before every visit).
template <class V, bool kProf>
__device__ void descend(const Params& p, Smem& sm, const Src& src, int level, uint32_t node, Lane& s,
                        int lane, int warp) {
    uint32_t* stk_node = sm.stk_node[warp];
    uint32_t* stk_mask = sm.stk_mask[warp];
    int lvl = level;
    if (level < 1 || level > kMaxLevels || node >= src.lvl_n[level]) {
        if (lane == 0) check_failed(p, 2, ((uint64_t)level << 40) | node);
        return;
    }
    uint32_t m0 = child_hits<V>(p, src, src.lvl[lvl] + (uint64_t)node * 128, s, lane,
                             sm.lanemask[warp][lvl]);
    prof_add<kProf>(sm, kPNodeVisits, 1, lane);
    if (s.U == 0) return;
    stk_node[lvl] = node;
    stk_mask[lvl] = m0;
    __syncwarp();
    while (true) {
        uint32_t m = stk_mask[lvl];
        m = __ballot_sync(kFull, ((m >> lane) & 1u) && (sm.lanemask[warp][lvl][lane] & s.U));
        if (m == 0) {
            if (lvl == level) break;
            lvl++;
            continue;
        }
        int c = __ffs(m) - 1;
        uint32_t child = stk_node[lvl] * 32u + (uint32_t)c;
        __syncwarp();
        stk_mask[lvl] = m & (m - 1);
        __syncwarp();
        if constexpr (V::kChildChebyshev) {
            // listed by its Chebyshev reach only: the exact test now
            const int32_t* nb = src.lvl[lvl] + (uint64_t)stk_node[lvl] * 128;
            if (!box_reach_lanes<V::kNarrowReach>(s, __ldg(nb + c), __ldg(nb + 32 + c), __ldg(nb + 64 + c),
                                                  __ldg(nb + 96 + c), sm.lanemask[warp][lvl][c] & s.U, lane))
                continue;
        }
        if (lvl == 1) {
            const long long t0 = tick<kProf>();
            const uint32_t how = V::visit(p, src, child, s, lane);
            prof_since<kProf>(sm, kPLeaf, t0, lane);
            prof_add<kProf>(sm, kPLeafVisits, 1, lane);
            prof_add<kProf>(sm, how == kVisitEmpty ? kPLeafEmpty : kPLeafDecided, how != kVisitTested, lane);
            if (s.U == 0) return;
        } else {
            if (child >= src.lvl_n[lvl - 1]) {
                if (lane == 0) check_failed(p, 3, ((uint64_t)(lvl - 1) << 40) | child);
                continue;
            }
            lvl--;
            uint32_t hm = child_hits<V>(p, src, src.lvl[lvl] + (uint64_t)child * 128, s, lane,
                                     sm.lanemask[warp][lvl]);
            prof_add<kProf>(sm, kPNodeVisits, 1, lane);
            if (s.U == 0) return;
            stk_node[lvl] = child;
            stk_mask[lvl] = hm;
            __syncwarp();
        }
    }
}

// The same descent for visitors with kOneVisitSite, also from a leaf (level
// 0, a frontier of leaves): their leaves are reached only through the one
// visit below, so the leaf code exists once in the kernel.  The polygon
// kernels measured faster that way (instruction fetch); points and line
// layers slower, so they keep the form above and visit a frontier of
// leaves directly.
template <class V, bool kProf>
__device__ void descend_one_site(const Params& p, Smem& sm, const Src& src, int level, uint32_t node, Lane& s,
                        int lane, int warp) {
    uint32_t* stk_node = sm.stk_node[warp];
    uint32_t* stk_mask = sm.stk_mask[warp];
    int lvl = level;
    if (level < 0 || level > kMaxLevels || (level > 0 && node >= src.lvl_n[level])) {
        if (lane == 0) check_failed(p, 2, ((uint64_t)level << 40) | node);
        return;
    }
    uint32_t leaf = node;
    if (level > 0) {
        uint32_t m0 = child_hits<V>(p, src, src.lvl[lvl] + (uint64_t)node * 128, s, lane, sm.lanemask[warp][lvl]);
        prof_add<kProf>(sm, kPNodeVisits, 1, lane);
        if (s.U == 0) return;
        stk_node[lvl] = node;
        stk_mask[lvl] = m0;
        __syncwarp();
    }
    while (true) {
        if (lvl > 0) {
            uint32_t m = stk_mask[lvl];
            m = __ballot_sync(kFull, ((m >> lane) & 1u) && (sm.lanemask[warp][lvl][lane] & s.U));
            if (m == 0) {
                if (lvl == level) break;
                lvl++;
                continue;
            }
            int c = __ffs(m) - 1;
            uint32_t child = stk_node[lvl] * 32u + (uint32_t)c;
            __syncwarp();
            stk_mask[lvl] = m & (m - 1);
            __syncwarp();
            if constexpr (V::kChildChebyshev) {
                // listed by its Chebyshev reach only: the exact test now
                const int32_t* nb = src.lvl[lvl] + (uint64_t)stk_node[lvl] * 128;
                if (!box_reach_lanes<V::kNarrowReach>(s, __ldg(nb + c), __ldg(nb + 32 + c), __ldg(nb + 64 + c),
                                                      __ldg(nb + 96 + c), sm.lanemask[warp][lvl][c] & s.U, lane))
                    continue;
            }
            if (lvl > 1) {
                if (child >= src.lvl_n[lvl - 1]) {
                    if (lane == 0) check_failed(p, 3, ((uint64_t)(lvl - 1) << 40) | child);
                    continue;
                }
                lvl--;
                uint32_t hm = child_hits<V>(p, src, src.lvl[lvl] + (uint64_t)child * 128, s, lane,
                                            sm.lanemask[warp][lvl]);
                prof_add<kProf>(sm, kPNodeVisits, 1, lane);
                if (s.U == 0) return;
                stk_node[lvl] = child;
                stk_mask[lvl] = hm;
                __syncwarp();
                continue;
            }
            leaf = child;
        }
        const long long t0 = tick<kProf>();
        const uint32_t how = V::visit(p, src, leaf, s, lane);
        prof_since<kProf>(sm, kPLeaf, t0, lane);
        prof_add<kProf>(sm, kPLeafVisits, 1, lane);
        prof_add<kProf>(sm, how == kVisitEmpty ? kPLeafEmpty : kPLeafDecided, how != kVisitTested, lane);
        if (s.U == 0 || level == 0) return;
    }
}

// Level bases of a tree into shared memory slot `slot` (0: the tree being
// traversed, 1: its side tree).
__device__ __forceinline__ void set_levels(Smem& sm, int slot, const TreeArg& t, int tid) {
#pragma unroll
    for (int l = 0; l <= kMaxLevels; l++)
        if (tid == l) {
            sm.lvl_base[slot][l] = (l >= 1 && l <= t.top) ? t.nodes + t.level_off[l] * 128 : nullptr;
            // level 0 counts leaves
            sm.lvl_n[slot][l] = l == 0 ? (uint32_t)((t.n_obj + 31) / 32) : (l <= t.top ? (uint32_t)t.level_n[l] : 0u);
        }
}

// Refine the shared frontier breadth first: replace every entry by its
// children that meet the box, one level at a time, while the next level fits
// (the deepest level that fits is kept).
__device__ void refine(const Params& p, const TreeArg& t, bool fill, Smem& sm, int32_t x0, int32_t y0,
                       int32_t x1, int32_t y1, int tid) {
    int lane = tid & 31, warp = tid >> 5;
    while (sm.f_level >= 1 && sm.f_count > 0) {
        int cur = sm.f_buf, lvl = sm.f_level, cnt = sm.f_count;
        __syncthreads();
        if (tid == 0) sm.next_count = 0;
        __syncthreads();
        const int32_t* base = sm.lvl_base[0][lvl];
        for (int e = warp; e < cnt; e += kWarps) {
            uint32_t node = sm.fid[cur][e];
            if (node >= sm.lvl_n[0][lvl]) {
                if (lane == 0) check_failed(p, 8, ((uint64_t)lvl << 40) | node);
                continue;
            }
            const int32_t* nd = base + (uint64_t)node * 128;
            if (p.log != nullptr)
                log_read(p, fill ? kLogPolyNode : kLogNode, (uint64_t)(nd - t.nodes) >> 7, lane);
            int4 b = make_int4(__ldg(nd + lane), __ldg(nd + 32 + lane), __ldg(nd + 64 + lane),
                               __ldg(nd + 96 + lane));
            bool hit = box_hit(b, x0, y0, x1, y1);
            uint32_t m = __ballot_sync(kFull, hit);
            int pos = 0;
            if (lane == 0 && m) pos = atomicAdd(&sm.next_count, __popc(m));
            pos = __shfl_sync(kFull, pos, 0);
            if (hit) {
                int slot = pos + __popc(m & ((1u << lane) - 1u));
                if (slot < kFCap) {
                    sm.fid[cur ^ 1][slot] = node * 32u + (uint32_t)lane;
                    sm.fbox[cur ^ 1][slot] = b;
                }
            }
        }
        __syncthreads();
        int nc = sm.next_count;
        __syncthreads();
        if (nc > kFCap) break;  // keep the current (coarser) frontier
        if (tid == 0) {
            sm.f_buf = cur ^ 1;
            sm.f_count = nc;
            sm.f_level = lvl - 1;
        }
        __syncthreads();
    }
}

// Breadth-first cull of a tree against a box into the shared frontier,
// starting from the root.
__device__ void cull(const Params& p, const TreeArg& t, bool fill, Smem& sm, int32_t x0, int32_t y0,
                     int32_t x1, int32_t y1, int tid) {
    if (tid == 0) {
        sm.f_buf = 0;
        sm.f_level = t.top;
        sm.f_count = 0;
        if (t.top > 0 && t.root_box.x <= x1 && t.root_box.z >= x0 && t.root_box.y <= y1 &&
            t.root_box.w >= y0) {
            sm.fid[0][0] = 0;
            sm.fbox[0][0] = t.root_box;
            sm.f_count = 1;
        }
    }
    __syncthreads();
    refine(p, t, fill, sm, x0, y0, x1, y1, tid);
}

// Learned cull (replaces the breadth-first R-tree cull): cover the strip's
// box, widened by the halo of object extents, with at most 256 aligned
// Hilbert cells (one per thread; a cell's keys are a contiguous run of the
// sorted order), find each cell's position range through the learned model,
// and turn the ranges into R-tree subtrees at the finest level whose entries
// fit the frontier.  Every object whose centre lies in the box is under one of
// the entries; the blocks then proceed exactly as after the R-tree cull.
__device__ void learned_cull(const Params& p, const TreeArg& t, const LModel& m, int32_t halo, Smem& sm,
                             int32_t bx0, int32_t by0, int32_t bx1, int32_t by1, int tid) {
    __shared__ unsigned long long cnt[kMaxLevels + 1];
    const int64_t lo_g = -(int64_t)kGridHalf, hi_g = (int64_t)kGridHalf - 1;
    const int64_t x0 = max((int64_t)bx0 - halo, lo_g), x1 = min((int64_t)bx1 + halo, hi_g);
    const int64_t y0 = max((int64_t)by0 - halo, lo_g), y1 = min((int64_t)by1 + halo, hi_g);
    // neighbouring cells share subtrees: a hash set in the (idle) second
    // frontier buffer keeps each entry once
    uint32_t* seen = (uint32_t*)sm.fbox[1];
    constexpr int kSeen = 1024;
    for (int i = tid; i < kSeen; i += kThreads) seen[i] = 0u;
    if (tid <= kMaxLevels) cnt[tid] = 0;
    if (tid == 0) {
        sm.f_buf = 0;
        sm.f_count = 0;
        sm.f_level = 0;
        sm.next_count = 0;
    }
    __syncthreads();
    if (t.top == 0 || m.n == 0 || x0 > x1 || y0 > y1) return;
    int k = 0;
    while (k < 31) {
        int64_t nx = ((x1 + kGridHalf) >> k) - ((x0 + kGridHalf) >> k) + 1;
        int64_t ny = ((y1 + kGridHalf) >> k) - ((y0 + kGridHalf) >> k) + 1;
        if (nx * ny <= kCullCells) break;
        k++;
    }
    const int64_t gx0 = (x0 + kGridHalf) >> k, gy0 = (y0 + kGridHalf) >> k;
    const int nx = (int)(((x1 + kGridHalf) >> k) - gx0 + 1), ny = (int)(((y1 + kGridHalf) >> k) - gy0 + 1);
    // kCullSub neighbouring threads (one warp) per cell: its two lookups run
    // at once on two of them, and they share its entries below
    const int cell = tid / kCullSub, sub = tid % kCullSub, lane = tid & 31;
    uint64_t pos = 0;
    if (cell < nx * ny && sub < 2) {
        int64_t cx = ((gx0 + cell % nx) << k) - kGridHalf, cy = ((gy0 + cell / nx) << k) - kGridHalf;
        uint64_t span = (k >= 31) ? (1ull << 62) : (1ull << (2 * k));
        uint64_t klo = (k >= 31) ? 0ull : (hilbert_key((int32_t)cx, (int32_t)cy) & ~(span - 1));
        bool fb;
        pos = learn_lower_bound(m, sub == 0 ? klo : klo + span, &fb);
    }
    const uint64_t plo = __shfl_sync(kFull, pos, lane & ~(kCullSub - 1));
    const uint64_t phi = __shfl_sync(kFull, pos, (lane & ~(kCullSub - 1)) + 1);
    uint64_t a = 1, b = 0;   // leaf range of this thread's cell (empty)
    if (cell < nx * ny && phi > plo) {
        a = plo >> 5;
        b = (phi - 1) >> 5;
    }
    // entries per level: the leaves [a, b] span (b >> 5l) - (a >> 5l) + 1 subtrees of level l
    for (int l = 0; l < t.top; l++)
        if (sub == 0 && a <= b) atomicAdd(&cnt[l], (unsigned long long)((b >> (5 * l)) - (a >> (5 * l)) + 1));
    __syncthreads();
    int lvl = t.top;   // no level fits: fall back to the root alone
    for (int l = 0; l < t.top; l++)
        if (cnt[l] <= (unsigned long long)kFCap) { lvl = l; break; }
    if (lvl == t.top) {
        if (tid == 0) {
            sm.fid[0][0] = 0;
            sm.fbox[0][0] = t.root_box;
            sm.f_count = 1;
            sm.f_level = t.top;
        }
        __syncthreads();
        refine(p, t, false, sm, bx0, by0, bx1, by1, tid);
        return;
    }
    if (a <= b) {
        uint64_t e0 = a >> (5 * lvl), e1 = b >> (5 * lvl);
        const int32_t* par = sm.lvl_base[0][lvl + 1];
        const bool inside = (e1 >> 5) < sm.lvl_n[0][lvl + 1];
        if (!inside) check_failed(p, 9, ((uint64_t)lvl << 40) | (e1 & ((1ull << 40) - 1)));
        for (uint64_t e = e0 + sub; inside && e <= e1; e += kCullSub) {
            const int32_t* nd = par + (e >> 5) * 128;
            int c = (int)(e & 31);
            int4 bb = make_int4(__ldg(nd + c), __ldg(nd + 32 + c), __ldg(nd + 64 + c), __ldg(nd + 96 + c));
            if (bb.x <= bx1 && bb.z >= bx0 && bb.y <= by1 && bb.w >= by0) {
                // at most kFCap distinct entries, so the set never fills
                uint32_t key = (uint32_t)e + 1u, h = (key * 2654435761u) & (kSeen - 1), prev;
                while ((prev = atomicCAS(&seen[h], 0u, key)) != 0u && prev != key) h = (h + 1) & (kSeen - 1);
                if (prev == key) continue;
                int slot = atomicAdd(&sm.next_count, 1);
                if (slot < kFCap) {
                    sm.fid[0][slot] = (uint32_t)e;
                    sm.fbox[0][slot] = bb;
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        sm.f_count = min(sm.next_count, kFCap);
        sm.f_level = lvl;
    }
    __syncthreads();
    refine(p, t, false, sm, bx0, by0, bx1, by1, tid);
}

// Column range [c0, c1] of 8-pixel block columns an entry box can reach: a
// column's samples span x in [X0 + 8c ps + ps/2 - off, X0 + (8c+7) ps + ps/2
// + off], widened by R.
__device__ __forceinline__ void entry_columns(int4 b, int32_t X0, int L, int32_t reach, int* c0, int* c1) {
    const int64_t base = (int64_t)X0 + ((int64_t)1 << L >> 1);
    int64_t lo = (int64_t)b.x - reach - base - 7 * ((int64_t)1 << L);
    int64_t hi = (int64_t)b.z + reach - base;
    int64_t a = -((-lo) >> (L + 3)), e = hi >> (L + 3);
    *c0 = (int)(a < 0 ? 0 : (a > kBlocksX ? kBlocksX : a));
    *c1 = (int)(e > kBlocksX - 1 ? kBlocksX - 1 : (e < -1 ? -1 : e));
}

// Bin the frontier by block column (falls back to the whole frontier when
// the lists would overflow).
__device__ void bin_frontier(Smem& sm, int32_t X0, int L, int32_t reach, int tid) {
    const int f_count = sm.f_count, fb = sm.f_buf;
    if (tid < kBlocksX) {
        sm.bucket_off[tid] = 0;
        sm.bucket_cur[tid] = 0;
    }
    __syncthreads();
    for (int e = tid; e < f_count; e += kThreads) {
        int c0, c1;
        entry_columns(sm.fbox[fb][e], X0, L, reach, &c0, &c1);
        for (int c = c0; c <= c1; c++) atomicAdd(&sm.bucket_off[c], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int sum = 0;
        for (int c = 0; c < kBlocksX; c++) {
            int n = sm.bucket_off[c];
            sm.bucket_off[c] = sum;
            sum += n;
        }
        sm.bucket_off[kBlocksX] = sum;
        sm.binned = sum <= kBucketCap;
    }
    __syncthreads();
    if (sm.binned) {
        for (int e = tid; e < f_count; e += kThreads) {
            int c0, c1;
            entry_columns(sm.fbox[fb][e], X0, L, reach, &c0, &c1);
            for (int c = c0; c <= c1; c++) {
                int pos = sm.bucket_off[c] + atomicAdd(&sm.bucket_cur[c], 1);
                if (pos < sm.bucket_off[c + 1]) sm.bucket[pos] = (uint16_t)e;
            }
        }
    }
    __syncthreads();
}

// Process every pixel block of the strip: against the culled frontier (R-tree)
// or through the learned lookup.
template <class V, bool kProf>
__device__ void blocks_pass(const Params& p, Smem& sm, const Src& src, const Src& side, int side_top, int32_t X0,
                            int32_t Y0, int strip, int col0, int col_shift, int z, int32_t R, bool mask_mode,
                            int tid) {
    int lane = tid & 31, warp = tid >> 5;
    const long long t_active = tick<kProf>();
    const int L = 23 - z;
    const int32_t ps = 1 << L;
    const int f_count = sm.f_count, f_level = sm.f_level, fb = sm.f_buf;
    // certain-cover half-side: the largest q with 2 q^2 <= R^2
    int32_t q = -1;
    if (V::kCertain) {
        const int64_t R2 = (int64_t)R * R;
        int64_t t = (int64_t)((double)R * 0.70710678118654752);
        while (t > 0 && 2 * t * t > R2) t--;
        while (2 * (t + 1) * (t + 1) <= R2) t++;
        q = (int32_t)t;
    }
    while (true) {
        int blk = 0;
        if (lane == 0) blk = atomicAdd(&sm.next_block, 1);
        blk = __shfl_sync(kFull, blk, 0);
        // the CTA's blocks: 2^col_shift block columns from col0, rows / 4 block rows
        if (blk >= (p.rows / kBH) << col_shift) break;
        prof_add<kProf>(sm, kPBlocks, 1, lane);
        int bx = col0 / kBW + (blk & ((1 << col_shift) - 1)), by = blk >> col_shift;
        int i = bx * kBW + (lane & 7);
        int jl = by * kBH + (lane >> 3);
        int j = strip * p.rows + jl;
        Lane s;
        s.L = L;
        s.cx = X0 + i * ps + (ps >> 1);
        s.cy = Y0 + j * ps + (ps >> 1);
        s.bx0 = X0 + (bx * kBW) * ps + (ps >> 1);
        s.by0 = Y0 + (strip * p.rows + by * kBH) * ps + (ps >> 1);
        s.R2 = (int64_t)R * R;
        bool centre_only = mask_mode;
        if constexpr (V::kFill) centre_only = mask_mode || !p.fill_aa;
        if (centre_only) {
            s.off = 0;
            s.und = 1u;
            s.nk = 1;
        } else {
            s.off = ps >> 2;
            s.und = 15u;
            s.nk = 4;
        }
        s.ext = (V::kFill ? 0 : R) + s.off;
        s.narrow = (int64_t)s.ext + s.off <= kNarrow;
        s.q = q;
        s.U = kFull;
        for (int k = 0; k < 4; k++) s.Uk[k] = k < s.nk ? kFull : 0u;
        if constexpr (V::kOutline) {
            if (mask_mode && p.pat_w == 0) {
                // a MASK pixel whose centre is already filled is decided
                // (unless a pattern may leave it transparent)
                const uint32_t open = __ballot_sync(kFull, (sm.res[jl * kTile + i] >> kResFillShift) == 0);
                s.U = s.Uk[0] = open;
                s.und = (open >> lane) & 1u;
            }
        }
        uint32_t und0 = s.und;
        {
            // this block's column list, or the whole frontier
            const bool binned = sm.binned;
            int lbeg = binned ? sm.bucket_off[bx] : 0;
            int lcnt = binned ? sm.bucket_off[bx + 1] - lbeg : f_count;
            if (binned && (lbeg < 0 || lcnt < 0 || lbeg + lcnt > kBucketCap)) {
                if (lane == 0) check_failed(p, 7, ((uint64_t)bx << 32) | (uint32_t)lbeg);
                lbeg = 0;
                lcnt = 0;
            }
            for (int c0 = 0; c0 < lcnt && s.U; c0 += 32) {
                int e = -1;
                uint32_t cm = 0;
                int4 fbx = make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
                if (c0 + lane < lcnt) {
                    e = binned ? (int)sm.bucket[lbeg + c0 + lane] : c0 + lane;
                    if (e >= f_count) {
                        check_failed(p, 1, ((uint64_t)bx << 32) | (uint32_t)e);
                        e = -1;
                    } else {
                        fbx = sm.fbox[fb][e];
                        cm = rect_lanes(s, fbx.x, fbx.y, fbx.z, fbx.w);
                    }
                }
                uint32_t mm;
                if constexpr (V::kScanChebyshev)
                    mm = __ballot_sync(kFull, (cm & s.U) != 0u);
                else
                    mm = __ballot_sync(kFull, reaches<V>(s, cm, fbx.x, fbx.y, fbx.z, fbx.w));
                prof_add<kProf>(sm, kPFrontierEntries, (unsigned long long)min(32, lcnt - c0), lane);
                while (mm) {
                    int k = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int ek = __shfl_sync(kFull, e, k);
                    if constexpr (V::kExactWhenTaken) {
                        const int4 bk = sm.fbox[fb][ek];
                        if (!box_reach_lanes<V::kNarrowReach>(s, bk.x, bk.y, bk.z, bk.w,
                                                              __shfl_sync(kFull, cm, k) & s.U, lane))
                            continue;
                    }
                    uint32_t id = sm.fid[fb][ek];
                    const long long t0 = tick<kProf>();
                    if constexpr (V::kOneVisitSite) {
                        descend_one_site<V, kProf>(p, sm, src, f_level, id, s, lane, warp);
                    } else if (f_level == 0) {
                        const uint32_t how = V::visit(p, src, id, s, lane);
                        prof_since<kProf>(sm, kPLeaf, t0, lane);
                        prof_add<kProf>(sm, kPLeafVisits, 1, lane);
                        prof_add<kProf>(sm, how == kVisitEmpty ? kPLeafEmpty : kPLeafDecided, how != kVisitTested,
                                        lane);
                    } else {
                        descend<V, kProf>(p, sm, src, f_level, id, s, lane, warp);
                    }
                    // everything below the frontier (leaves included)
                    prof_since<kProf>(sm, kPDescend, t0, lane);
                    // drop frontier entries that no longer reach an undecided lane
                    if constexpr (V::kExactWhenTaken)
                        mm &= __ballot_sync(kFull, ((mm >> lane) & 1u) && (cm & s.U) != 0u);
                    else
                        mm &= __ballot_sync(kFull, ((mm >> lane) & 1u) &&
                                                       reaches<V>(s, cm, fbx.x, fbx.y, fbx.z, fbx.w));
                }
            }
            // objects longer than the learned index's halo live in a side tree
            if (side_top > 0 && s.U) {
                const long long t0 = tick<kProf>();
                if constexpr (V::kOneVisitSite)
                    descend_one_site<V, kProf>(p, sm, side, side_top, 0, s, lane, warp);
                else
                    descend<V, kProf>(p, sm, side, side_top, 0, s, lane, warp);
                prof_since<kProf>(sm, kPDescend, t0, lane);
            }
        }
        uint32_t covered = und0 & ~s.und;
        uint8_t r = sm.res[jl * kTile + i];
        if (V::kFill) {
            // the centre (1), or the number of super-samples inside (0..4)
            if (covered) r |= (s.nk == 1 ? 1u : (uint32_t)__popc(covered)) << kResFillShift;
        } else if (mask_mode) {
            if (covered) r |= kResCentre;
        } else {
            r |= (uint8_t)covered;
        }
        sm.res[jl * kTile + i] = r;
    }
    prof_since<kProf>(sm, kPBlocksWarp, t_active, lane);
}

// One stage (Algorithm 1 over points / segments / edges, or Algorithm 2 over
// polygon boxes) for the strip: cull through the R-tree or the learned
// index, then every block.
template <class V, bool kProf>
__device__ void stage(const Params& p, Smem& sm, const TreeArg& t, const void* obj, const uint32_t* ids,
                      const TreeArg& st, const void* sobj, const uint32_t* sids, const LModel* m, int32_t halo,
                      int32_t X0, int32_t Y0, int strip, int col0, int col_shift, int z, int32_t R, bool mask_mode,
                      int32_t bx0, int32_t by0, int32_t bx1, int32_t by1, int tid) {
    const long long t_cull = tick<kProf>();
    set_levels(sm, 0, t, tid);
    set_levels(sm, 1, st, tid);
    if (tid == 0) sm.next_block = 0;
    __syncthreads();
    if (m == nullptr)
        cull(p, t, V::kFill, sm, bx0, by0, bx1, by1, tid);
    else
        learned_cull(p, t, *m, halo, sm, bx0, by0, bx1, by1, tid);
    if (tid == 0) prof_since<kProf>(sm, kPCull, t_cull, 0);
    int4 sb = st.root_box;
    bool side_hit = st.top > 0 && sb.x <= bx1 && sb.z >= bx0 && sb.y <= by1 && sb.w >= by0;
    if (sm.f_count > 0 || side_hit) {
        // the column lists are rebuilt for every pass, also for an empty
        // frontier (a strip reached only by the side tree), so that the
        // blocks never read the lists of an earlier stage
        bool sub = !mask_mode;   // super-samples
        if constexpr (V::kFill) sub = !mask_mode && p.fill_aa;
        const int32_t off = sub ? ((1 << (23 - z)) >> 2) : 0;
        const long long t_bin = tick<kProf>();
        bin_frontier(sm, X0, 23 - z, (V::kFill ? 0 : R) + off, tid);
        if (tid == 0) prof_since<kProf>(sm, kPBin, t_bin, 0);
        const long long t_blocks = tick<kProf>();
        // the frontier's idle buffer: scratch for segment leaves
        int4* const seg_scratch = sm.fbox[1 - sm.f_buf];
        uint16_t* const pair_scratch = reinterpret_cast<uint16_t*>(sm.fid[1 - sm.f_buf]);
        Src src{obj, ids, t.n_obj, t.nodes, sm.lvl_base[0], sm.lvl_n[0], seg_scratch, pair_scratch};
        Src side{sobj, sids, st.n_obj, st.nodes, sm.lvl_base[1], sm.lvl_n[1], seg_scratch, pair_scratch};
        blocks_pass<V, kProf>(p, sm, src, side, side_hit ? st.top : 0, X0, Y0, strip, col0, col_shift, z, R, mask_mode,
                              tid);
        __syncthreads();
        if (tid == 0) prof_since<kProf>(sm, kPBlocksCta, t_blocks, 0);
    }
    __syncthreads();
}

// Kernel parts: one per layer kind, and polygon layers in two launches --
// first the fill (kPolyFill: Algorithm 2), which leaves the strip's fill bits
// as a bit mask (MASK layout, 32 bytes per pixel row) at the start of the
// strip's own part of the output, then the outline (the HV_LAYER_POLYGONS
// part: Algorithm 1 over the edges), which reads those bits back, decides
// the samples and encodes the composed strip over them.  Each CTA reads and
// writes only its own strip's part of the output, so the bits never meet
// another CTA's writes.  Apart, each part's traversal stays small enough for
// the instruction cache; fused, the polygon kernel measured 40% slower.
constexpr int kPolyFill = 3;

// CTAs per SM: four (64 registers) for every kind, measured best for each
// since the segment leaves share their pairs over the lanes (the line and
// outline kernels keep a 12-16 byte spill and still run faster than with
// three).
template <int kKind>
struct KindTraits {
    static constexpr int kBlocksPerSM = 4;
};

// The pattern texel of global pixel (gx, gy).
__device__ __forceinline__ uchar4 fill_texel(const Params& p, uint32_t gx, uint32_t gy) {
    return p.pattern[(gy % (uint32_t)p.pat_h) * (uint32_t)p.pat_w + gx % (uint32_t)p.pat_w];
}

// Byte offset, in a tile's output, of pixel (c, j) (column c a multiple of 32).
__device__ __forceinline__ uint64_t px_offset(int mode, int j, int c) {
    if (mode == HV_MODE_MASK) return (uint64_t)j * (kTile / 8) + (uint64_t)(c >> 3);
    return ((uint64_t)j * kTile + (uint64_t)c) * (mode == HV_MODE_COVERAGE ? 1u : 4u);
}

// The fill launch of a polygon layer hands the outline launch its results in
// the CTA's own part of the output (which the outline overwrites): per pixel
// row of the CTA, at the start of that row's part (cols pixels, at least
// cols / 8 bytes in every mode), a bit per pixel (centre fill), or with the
// anti-aliased fill a byte per pixel holding the number of super-samples
// inside.  This reads them back into the strip's shared results.
__device__ void decode_fill(const Params& p, const uint8_t* tile_out, Smem& sm, int strip, int col0, int cols,
                            int tid, bool aa_bytes) {
    const int rows = p.rows;
    if (aa_bytes) {
        const int wpr = cols / 4, wsh = __ffs(wpr) - 1;   // words per row, as a shift
        for (int k = tid; k < rows * wpr; k += kThreads) {
            const int jl = k >> wsh, w = k & (wpr - 1);
            const uint32_t v = ((const uint32_t*)(tile_out + px_offset(p.mode, strip * rows + jl, col0)))[w];
            ((uint32_t*)(sm.res + jl * kTile + col0))[w] = (v & 0x07070707u) << kResFillShift;
        }
        return;
    }
    const int wpr = cols / 32, wsh = __ffs(wpr) - 1;
    for (int k = tid; k < rows * wpr; k += kThreads) {
        const int jl = k >> wsh, w = k & (wpr - 1);
        const uint32_t word = ((const uint32_t*)(tile_out + px_offset(p.mode, strip * rows + jl, col0)))[w];
        uint32_t* r4 = (uint32_t*)(sm.res + jl * kTile + col0 + 32 * w);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t b = word >> (4 * q);
            r4[q] = ((b & 1u) ? kResFill : 0u) | ((b & 2u) ? kResFill << 8 : 0u) | ((b & 4u) ? kResFill << 16 : 0u) |
                    ((b & 8u) ? kResFill << 24 : 0u);
        }
    }
}

// The outline launch of a polygon layer encodes the strip composed over the
// fill results: per pixel v outline samples, the fill field (centre, or the
// anti-aliased count), a pattern texel by the global pixel coordinate.
__device__ void encode_polygons(const Params& p, const Smem& sm, uint8_t* out, int strip, int col0, int cols,
                                uint32_t tile, int tid) {
    const int rows = p.rows;
    const hv_tile_req q = p.reqs[tile];
    const uint32_t gx0 = q.x * (uint32_t)kTile, gy0 = q.y * (uint32_t)kTile + (uint32_t)(strip * rows);
    if (p.mode == HV_MODE_MASK) {
        const int wpr = cols / 32, wsh = __ffs(wpr) - 1;
        if (tid < rows * wpr) {
            const int jl = tid >> wsh, c = col0 + 32 * (tid & (wpr - 1));
            uint32_t word = 0;
            for (int b = 0; b < 32; b++) {
                const uint32_t f = sm.res[jl * kTile + c + b];
                bool filled = (f >> kResFillShift) != 0;
                if (filled && p.pat_w) filled = fill_texel(p, gx0 + c + b, gy0 + jl).w != 0;
                if ((f & kResCentre) || filled) word |= 1u << b;
            }
            *(uint32_t*)(out + px_offset(p.mode, strip * rows + jl, c)) = word;
        }
    } else if (p.mode == HV_MODE_COVERAGE) {
        // 16 pixels (one uint4) per thread and step
        const int upr = cols / 16, ush = __ffs(upr) - 1;
        for (int u = tid; u < rows * upr; u += kThreads) {
            const int jl = u >> ush, c = col0 + 16 * (u & (upr - 1));
            const uint8_t* r = sm.res + jl * kTile + c;
            uint32_t w4[4];
            for (int k = 0; k < 4; k++) {
                uint32_t v = 0;
                for (int b = 0; b < 4; b++) {
                    const uint32_t f = r[4 * k + b];
                    uint32_t fill = f >> kResFillShift;
                    if (fill && p.pat_w && fill_texel(p, gx0 + c + 4 * k + b, gy0 + jl).w == 0) fill = 0;
                    // anti-aliased: the fill count in bits 4-6; else bit 3 for a filled centre
                    const uint32_t cv = __popc(f & 15u) | (p.fill_aa ? fill << 4 : (fill ? 8u : 0u));
                    v |= cv << (8 * b);
                }
                w4[k] = v;
            }
            *(uint4*)(out + px_offset(p.mode, strip * rows + jl, c)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    } else {
        // 4 pixels (one uint4) per thread and step
        const int upr = cols / 4, ush = __ffs(upr) - 1;
        for (int u = tid; u < rows * upr; u += kThreads) {
            const int jl = u >> ush, c = col0 + 4 * (u & (upr - 1));
            uint32_t w[4];
            for (int b = 0; b < 4; b++) {
                uint32_t f = sm.res[jl * kTile + c + b];
                uint32_t v = __popc(f & 15u);
                uint32_t a = (255u * v + 2u) >> 2;
                // fill count: 0..4 anti-aliased, else 4 for a filled centre
                uint32_t fc = f >> kResFillShift;
                if (!p.fill_aa && fc) fc = 4;
                uchar4 fill = p.fill;
                if (fc && p.pat_w) {
                    fill = fill_texel(p, gx0 + c + b, gy0 + jl);
                    if (fill.w == 0) fc = 0;   // a transparent texel: not filled
                }
                uint32_t rgba = 0;
                if (fc == 4) {
                    uint32_t r = (p.line.x * a + fill.x * (255u - a) + 127u) / 255u;
                    uint32_t g = (p.line.y * a + fill.y * (255u - a) + 127u) / 255u;
                    uint32_t bl = (p.line.z * a + fill.z * (255u - a) + 127u) / 255u;
                    rgba = r | (g << 8) | (bl << 16) | (255u << 24);
                } else if (fc) {
                    // the outline over a partly covered fill
                    const uint32_t af = (255u * fc + 2u) >> 2;
                    const uint32_t A = (255u * a + af * (255u - a) + 127u) / 255u;
                    const uint32_t den = 255u * A, wf = af * (255u - a), wl = a * 255u;
                    const uint32_t r = (p.line.x * wl + fill.x * wf + 127u * A) / den;
                    const uint32_t g = (p.line.y * wl + fill.y * wf + 127u * A) / den;
                    const uint32_t bl = (p.line.z * wl + fill.z * wf + 127u * A) / den;
                    rgba = r | (g << 8) | (bl << 16) | (A << 24);
                } else if (v) {
                    rgba = (uint32_t)p.line.x | ((uint32_t)p.line.y << 8) | ((uint32_t)p.line.z << 16) | (a << 24);
                }
                w[b] = rgba;
            }
            *(uint4*)(out + px_offset(p.mode, strip * rows + jl, c)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// kSplit: the launch splits strips into column parts (p.parts > 1); the
// full-width instantiation keeps the column arithmetic compile-time constant.
template <int kKind, bool kProf, bool kSplit>
__global__ void __launch_bounds__(kThreads, KindTraits<kKind>::kBlocksPerSM) k_render(const Params p) {
    __shared__ Smem sm;
    const int tid = threadIdx.x;
    const long long t_start = tick<kProf>();
    if constexpr (kProf) {
        if (tid < kPN) sm.prof[tid] = 0;
    }
    const int rows = p.rows;
    const int parts = kSplit ? p.parts : 1, cols = kTile / parts, col_shift = kSplit ? p.col_shift : 5;
    // CTA -> tile, strip of rows pixel rows, part of cols pixel columns
    const uint32_t tile = blockIdx.x / (p.strips * parts);
    const int sp = (int)(blockIdx.x % (p.strips * parts));
    const int strip = sp / parts, col0 = (sp % parts) * cols;
    const uint32_t n = p.n_dev ? min(*p.n_dev, p.n) : p.n;
    if (tile >= n) return;
    hv_tile_req q = p.reqs[tile];
    bool ok = q.z <= 19 && q.x < (1u << q.z) && q.y < (1u << q.z) && (p.R_units >= 0 || (q.r16 >= 1 && q.r16 <= 1024));
    if constexpr (kKind == HV_LAYER_POLYGONS)
        decode_fill(p, p.out + (uint64_t)tile * p.tile_bytes, sm, strip, col0, cols, tid,
                    p.fill_aa && p.mode != HV_MODE_MASK);
    else
        for (int k = tid; k < rows * kTile / 4; k += kThreads) ((uint32_t*)sm.res)[k] = 0u;
    if (!ok) {
        if (tid == 0 && sp == 0) atomicOr(p.status, 1u);
    }
    __syncthreads();
    if (tid == 0) prof_since<kProf>(sm, kPPrologue, t_start, 0);
    const bool mask_mode = p.mode == HV_MODE_MASK;
    if (ok) {
        const int z = q.z;
        const int32_t ps = 1 << (23 - z);
        const int32_t X0 = (int32_t)(-(int64_t)kGridHalf + (int64_t)q.x * ((int64_t)1 << (31 - z)));
        const int32_t Y0 = (int32_t)(-(int64_t)kGridHalf + (int64_t)q.y * ((int64_t)1 << (31 - z)));
        // at most 2^29 either way (r16 <= 1024, or the buffer limit)
        int32_t R = (int32_t)q.r16 << (19 - z);
        if (p.R_units >= 0) R = p.R_units;
        const int32_t off = mask_mode ? 0 : (ps >> 2);
        // the CTA's sample box
        const int32_t sx0 = X0 + col0 * ps + (ps >> 1) - off, sx1 = X0 + (col0 + cols - 1) * ps + (ps >> 1) + off;
        const int32_t sy0 = Y0 + strip * rows * ps + (ps >> 1) - off;
        const int32_t sy1 = Y0 + (strip * rows + rows - 1) * ps + (ps >> 1) + off;
        const bool learned = p.use_learned != 0;
        // Algorithm 1 over points / segments / polygon edges
        if constexpr (kKind == HV_LAYER_POINTS)
            stage<PointLeaf, kProf>(p, sm, p.tree, p.obj, nullptr, p.side, p.side_obj, p.side_ids, learned ? &p.lm : nullptr,
                             p.halo, X0, Y0, strip, col0, col_shift, z, R, mask_mode, sx0 - R, sy0 - R, sx1 + R, sy1 + R, tid);
        else if constexpr (kKind != kPolyFill)
            stage<SegLeaf<kKind == HV_LAYER_LINES>, kProf>(p, sm, p.tree, p.obj, nullptr, p.side, p.side_obj, p.side_ids, learned ? &p.lm : nullptr,
                           p.halo, X0, Y0, strip, col0, col_shift, z, R, mask_mode, sx0 - R, sy0 - R, sx1 + R, sy1 + R, tid);
        // Algorithm 2 over polygon boxes and edges
        if constexpr (kKind == kPolyFill) {
            // the CTA's centres, or its super-samples
            const int32_t fo = (p.fill_aa && p.mode != HV_MODE_MASK) ? (ps >> 2) : 0;
            const int32_t cx0 = X0 + col0 * ps + (ps >> 1) - fo, cx1 = X0 + (col0 + cols - 1) * ps + (ps >> 1) + fo;
            const int32_t cy0 = Y0 + strip * rows * ps + (ps >> 1) - fo;
            const int32_t cy1 = Y0 + (strip * rows + rows - 1) * ps + (ps >> 1) + fo;
            stage<FillLeaf, kProf>(p, sm, p.mtree, p.mbr_obj, p.mbr_ids, p.mside, p.mside_obj, p.mside_ids,
                            learned ? &p.mlm : nullptr, p.mhalo, X0, Y0, strip, col0, col_shift, z, 0, mask_mode,
                            cx0, cy0,
                            cx1, cy1, tid);
        }
    }
    // ---- encode the strip (Sec. 4.1 Render Tiles) ----
    const long long t_enc = tick<kProf>();
    uint8_t* out = p.out + (uint64_t)tile * p.tile_bytes;
    if constexpr (kKind == kPolyFill) {
        // the fill results for the outline part, per pixel row at the start
        // of the row's part of the CTA's own output (see decode_fill)
        if (p.fill_aa && p.mode != HV_MODE_MASK) {
            const int wpr = cols / 4, wsh = __ffs(wpr) - 1;
            for (int k = tid; k < rows * wpr; k += kThreads) {
                const int jl = k >> wsh, w = k & (wpr - 1);
                ((uint32_t*)(out + px_offset(p.mode, strip * rows + jl, col0)))[w] =
                    (((const uint32_t*)(sm.res + jl * kTile + col0))[w] >> kResFillShift) & 0x07070707u;
            }
        } else {
            const int wpr = cols / 32, wsh = __ffs(wpr) - 1;
            if (tid < rows * wpr) {
                const int jl = tid >> wsh, w = tid & (wpr - 1);
                uint32_t word = 0;
                for (int b = 0; b < 32; b++)
                    if (sm.res[jl * kTile + col0 + 32 * w + b] >> kResFillShift) word |= 1u << b;
                ((uint32_t*)(out + px_offset(p.mode, strip * rows + jl, col0)))[w] = word;
            }
        }
    } else if constexpr (kKind == HV_LAYER_POLYGONS) {
        encode_polygons(p, sm, out, strip, col0, cols, tile, tid);
    } else if (p.mode == HV_MODE_MASK) {
        // word w of row j = pixels 32w .. 32w+31
        const int wpr = cols / 32, wsh = __ffs(wpr) - 1;
        if (tid < rows * wpr) {
            const int jl = tid >> wsh, c = col0 + 32 * (tid & (wpr - 1));
            uint32_t word = 0;
            for (int b = 0; b < 32; b++)
                if (sm.res[jl * kTile + c + b] & kResCentre) word |= 1u << b;
            *(uint32_t*)(out + px_offset(p.mode, strip * rows + jl, c)) = word;
        }
    } else if (p.mode == HV_MODE_COVERAGE) {
        // one uint4 (16 pixels) per thread and step
        const int upr = cols / 16, ush = __ffs(upr) - 1;
        for (int u = tid; u < rows * upr; u += kThreads) {
            const int jl = u >> ush, c = col0 + 16 * (u & (upr - 1));
            const uint8_t* r = sm.res + jl * kTile + c;
            uint32_t w4[4];
            for (int k = 0; k < 4; k++) {
                uint32_t v = 0;
                for (int b = 0; b < 4; b++) v |= (uint32_t)__popc(r[4 * k + b] & 15u) << (8 * b);
                w4[k] = v;
            }
            *(uint4*)(out + px_offset(p.mode, strip * rows + jl, c)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    } else {
        // one uint4 (4 pixels) per thread and step
        const int upr = cols / 4, ush = __ffs(upr) - 1;
        for (int u = tid; u < rows * upr; u += kThreads) {
            const int jl = u >> ush, c = col0 + 4 * (u & (upr - 1));
            uint32_t w[4];
            for (int b = 0; b < 4; b++) {
                const uint32_t v = __popc(sm.res[jl * kTile + c + b] & 15u);
                const uint32_t a = (255u * v + 2u) >> 2;
                w[b] = v ? ((uint32_t)p.line.x | ((uint32_t)p.line.y << 8) | ((uint32_t)p.line.z << 16) | (a << 24))
                         : 0u;
            }
            *(uint4*)(out + px_offset(p.mode, strip * rows + jl, c)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    if constexpr (kProf) {
        __syncthreads();
        if (tid == 0) {
            const unsigned long long now = (unsigned long long)clock64();
            sm.prof[kPEncode] += now - (unsigned long long)t_enc;
            sm.prof[kPTotal] += now - (unsigned long long)t_start;
            sm.prof[kPCtas] = 1;
            // CTA-wide phases hold every warp of the CTA
            const int cta_phases[6] = {kPTotal, kPPrologue, kPCull, kPBin, kPBlocksCta, kPEncode};
            for (int k = 0; k < 6; k++) sm.prof[cta_phases[k]] *= kWarps;
        }
        __syncthreads();
        if (tid < kPN && sm.prof[tid]) atomicAdd(p.phases + tid, sm.prof[tid]);
    }
}

TreeArg tree_arg(const TreeView& v) {
    TreeArg a;
    a.nodes = v.nodes;
    for (int l = 0; l <= kMaxLevels; l++) {
        a.level_off[l] = v.level_off[l];
        a.level_n[l] = v.level_n[l];
    }
    a.top = v.top;
    a.n_obj = v.n_obj;
    a.root_box = v.root_box;
    return a;
}

}  // namespace

LModel learned_model(const LearnedView& v);

uint32_t render_launch_count(Layer* L, int) { return L->kind == HV_LAYER_POLYGONS ? 2u : 1u; }

bool fill_style_ok(const hv_fill_style* f) {
    if (!f) return true;
    if (f->flags & ~(uint32_t)HV_FILL_AA) return false;
    if (f->pattern_w == 0 && f->pattern_h == 0) return true;
    if (f->pattern_w < 1 || f->pattern_h < 1 || f->pattern_w > kMaxPattern || f->pattern_h > kMaxPattern ||
        !f->pattern_rgba)
        return false;
    for (uint32_t k = 0; k < f->pattern_w * f->pattern_h; k++)
        if (f->pattern_rgba[4 * k + 3] != 0 && f->pattern_rgba[4 * k + 3] != 255) return false;
    return true;
}

int launch_render(Layer* L, const hv_tile_req* d_reqs, uint32_t n, int mode, int index_kind,
                  const hv_style* style, uint8_t* d_out, cudaStream_t stream, const RenderLog* log,
                  const uint32_t* n_dev, int32_t R_units, const hv_fill_style* fill, const void* pattern_dev) {
    (void)index_kind;
    if (n == 0) return HV_OK;
    Params p;
    memset(&p, 0, sizeof(p));
    p.R_units = R_units < 0 ? -1 : R_units;
    if (fill && L->kind == HV_LAYER_POLYGONS) {
        if (!fill_style_ok(fill)) {
            set_error("invalid fill style (flags, pattern size 1..16, texel alpha 0 or 255)");
            return HV_EINVAL;
        }
        p.fill_aa = (fill->flags & HV_FILL_AA) ? 1 : 0;
        if (fill->pattern_w) {
            if (!pattern_dev) {
                set_error("a fill pattern needs its device copy");
                return HV_EINVAL;
            }
            p.pat_w = (int)fill->pattern_w;
            p.pat_h = (int)fill->pattern_h;
            p.pattern = (const uchar4*)pattern_dev;
        }
    }
    p.reqs = d_reqs;
    p.n = n;
    p.n_dev = n_dev;
    p.mode = mode;
    p.kind = L->kind;
    if (style) {
        p.line = make_uchar4(style->line_rgba[0], style->line_rgba[1], style->line_rgba[2], 0);
        p.fill = make_uchar4(style->fill_rgba[0], style->fill_rgba[1], style->fill_rgba[2], 0);
    }
    p.out = d_out;
    p.tile_bytes = (uint32_t)hv_tile_bytes(mode);
    p.tree = tree_arg(L->tree.view);
    p.obj = L->obj;
    p.mtree = tree_arg(L->mbr_tree.view);
    p.mbr_obj = L->mbr_obj;
    p.mbr_ids = L->mbr_ids;
    p.poly_edges = L->poly_edges;
    p.poly_edge_off = L->poly_edge_off;
    p.status = L->status;
    p.fault = (unsigned long long*)(L->status + 2);
    p.n_poly = L->n_poly;
    p.n_edges = L->n_src;
    if (index_kind == HV_INDEX_LEARNED) {
        const LearnedView& a = L->learned.view;
        const LearnedView& b = L->mbr_learned.view;
        if (!a.ready || (L->kind == HV_LAYER_POLYGONS && !b.ready)) {
            set_error("learned index not built");
            return HV_ESTATE;
        }
        p.use_learned = 1;
        p.lm = learned_model(a);
        p.halo = a.halo;
        p.side = tree_arg(a.outliers);
        p.side_obj = a.outlier_obj;
        p.side_ids = a.outlier_ids;
        if (L->kind == HV_LAYER_POLYGONS) {
            p.mlm = learned_model(b);
            p.mhalo = b.halo;
            p.mside = tree_arg(b.outliers);
            p.mside_obj = b.outlier_obj;
            p.mside_ids = b.outlier_ids;
        }
    }
    if (log) {
        p.log = (unsigned long long*)log->log;
        p.log_cap = log->cap;
        p.log_n = (unsigned long long*)log->count;
        p.phases = (unsigned long long*)log->phases;
    }
    const bool prof = p.phases != nullptr;
    // strip height: 16 rows (16 CTAs per tile) when the batch fills the GPU,
    // 8 or 4 rows for small batches so that a few tiles still spread over
    // many SMs (lower latency)
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = L->kind == HV_LAYER_POINTS ? KindTraits<HV_LAYER_POINTS>::kBlocksPerSM
                                                  : KindTraits<HV_LAYER_LINES>::kBlocksPerSM;
    const uint64_t resident = (uint64_t)sms * per_sm;
    p.rows = (uint64_t)n * 16 >= 2 * resident ? 16 : ((uint64_t)n * 32 >= 2 * resident ? 8 : 4);
    p.strips = kTile / p.rows;
    // batches too small for the GPU even in 4-row strips also split each
    // strip into 2 or 4 column parts (a CTA per 128 or 64 columns)
    p.parts = 1;
    if (p.rows == 4 && !prof)
        while (p.parts < 4 && (uint64_t)n * p.strips * p.parts * 2 <= resident) p.parts *= 2;
    p.cols = kTile / p.parts;
    p.col_shift = p.parts == 1 ? 5 : (p.parts == 2 ? 4 : 3);
    uint64_t grid = (uint64_t)n * p.strips * p.parts;
    if (grid > 0x7fffffffull) {
        set_error("too many tiles in one call");
        return HV_EINVAL;
    }
    if (prof) {
        // the instrumented instantiations (phase profile, full-width strips);
        // polygon layers profile their two launches (fill, outline) into two
        // sets of counters
        if (L->kind == HV_LAYER_POINTS)
            k_render<HV_LAYER_POINTS, true, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        else if (L->kind == HV_LAYER_LINES)
            k_render<HV_LAYER_LINES, true, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        else {
            k_render<kPolyFill, true, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
            Params q = p;
            q.phases = p.phases + kPN;
            k_render<HV_LAYER_POLYGONS, true, false><<<(unsigned)grid, kThreads, 0, stream>>>(q);
        }
    } else if (p.parts > 1) {
        if (L->kind == HV_LAYER_POINTS)
            k_render<HV_LAYER_POINTS, false, true><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        else if (L->kind == HV_LAYER_LINES)
            k_render<HV_LAYER_LINES, false, true><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        else {
            k_render<kPolyFill, false, true><<<(unsigned)grid, kThreads, 0, stream>>>(p);
            k_render<HV_LAYER_POLYGONS, false, true><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        }
    } else if (L->kind == HV_LAYER_POINTS)
        k_render<HV_LAYER_POINTS, false, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
    else if (L->kind == HV_LAYER_LINES)
        k_render<HV_LAYER_LINES, false, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
    else {
        // the fill first: the outline reads its bits and writes the tile
        k_render<kPolyFill, false, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
        k_render<HV_LAYER_POLYGONS, false, false><<<(unsigned)grid, kThreads, 0, stream>>>(p);
    }
    HV_CUDA(cudaGetLastError());
    return HV_OK;
}

}  // namespace hv
