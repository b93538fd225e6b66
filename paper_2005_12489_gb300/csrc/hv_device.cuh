// Device-side grid arithmetic and exact predicates (HiVision Sec. 3.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hv {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kGridHalf = 1 << 30;
constexpr int32_t kEmptyLo = 0x7fffffff;          // min-corner of an empty box
constexpr int32_t kEmptyHi = (int32_t)0x80000000; // max-corner of an empty box

// Hilbert curve index of (x, y) on a 2^31 grid (x, y shifted to [0, 2^31)),
// the classic quadrant-rotation construction; 62-bit result.
__host__ __device__ inline uint64_t hilbert_key(int32_t gx, int32_t gy) {
    uint32_t x = (uint32_t)(gx + kGridHalf);
    uint32_t y = (uint32_t)(gy + kGridHalf);
    uint64_t d = 0;
    for (uint32_t s = 1u << 30; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * (uint64_t)s * (uint64_t)((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = ~x;
                y = ~y;
            }
            uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Centre of a box, rounded down, computed without overflow.
__host__ __device__ inline int32_t mid32(int32_t a, int32_t b) {
    return (int32_t)(((int64_t)a + (int64_t)b) >> 1);
}

// |o - s|^2 <= R^2 (Algorithm 1, closed comparison).  |dx|, |dy| < 2^31.
__device__ __forceinline__ bool point_within(int32_t ox, int32_t oy, int32_t sx, int32_t sy,
                                             int64_t R2) {
    int64_t dx = (int64_t)ox - sx, dy = (int64_t)oy - sy;
    return dx * dx + dy * dy <= R2;
}

// Unsigned 64 x 64 -> 128-bit product compare: a*a <= b*c.
__device__ __forceinline__ bool sq_le_prod(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t lo1 = a * a, hi1 = __umul64hi(a, a);
    uint64_t lo2 = b * c, hi2 = __umul64hi(b, c);
    return hi1 < hi2 || (hi1 == hi2 && lo1 <= lo2);
}

// Distance from s to the closed segment [a, b] is <= R.  With d = b - a,
// w = s - a, t = w.d and L = d.d the nearest point is a when t <= 0, b when
// t >= L, and otherwise the squared distance is (w x d)^2 / L, compared as
// (w x d)^2 <= R^2 L in 128 bits (|w x d| < 2^63, R^2 L < 2^121).
__device__ __forceinline__ bool segment_within(int32_t ax, int32_t ay, int32_t bx, int32_t by,
                                               int32_t sx, int32_t sy, int64_t R2) {
    int64_t dx = (int64_t)bx - ax, dy = (int64_t)by - ay;
    int64_t wx = (int64_t)sx - ax, wy = (int64_t)sy - ay;
    int64_t t = wx * dx + wy * dy;
    if (t <= 0) return wx * wx + wy * wy <= R2;
    int64_t L = dx * dx + dy * dy;
    if (t >= L) {
        int64_t ex = (int64_t)sx - bx, ey = (int64_t)sy - by;
        return ex * ex + ey * ey <= R2;
    }
    int64_t cr = wx * dy - wy * dx;
    uint64_t c = (uint64_t)(cr < 0 ? -cr : cr);
    return sq_le_prod(c, (uint64_t)R2, (uint64_t)L);
}

// The same test with the segment and the sample given relative to a nearby
// origin: every endpoint within 2^30 of it and the sample within 2^27, so the
// differences below fit 32 bits and each product is one 32 x 32 -> 64-bit
// multiply.  d = b - a and L = d.d are passed in (fixed per segment), and so
// are bounds c_lo <= R |d| <= c_hi (c_lo = -1, c_hi = INT64_MAX when unknown):
// |cross| <= c_lo means (w x d)^2 < R^2 L, |cross| > c_hi the opposite, and
// only a cross product between them needs the 128-bit comparison.
__device__ __forceinline__ bool segment_within_rel(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t dx,
                                                   int32_t dy, int64_t L, int64_t c_lo, int64_t c_hi, int32_t sx,
                                                   int32_t sy, int64_t R2) {
    const int32_t wx = sx - ax, wy = sy - ay;
    const int64_t t = (int64_t)wx * dx + (int64_t)wy * dy;
    if (t <= 0) return (int64_t)wx * wx + (int64_t)wy * wy <= R2;
    if (t >= L) {
        const int32_t ex = sx - bx, ey = sy - by;
        return (int64_t)ex * ex + (int64_t)ey * ey <= R2;
    }
    const int64_t cr = (int64_t)wx * dy - (int64_t)wy * dx;
    const int64_t c = cr < 0 ? -cr : cr;
    if (c <= c_lo) return true;
    if (c > c_hi) return false;
    return sq_le_prod((uint64_t)c, (uint64_t)R2, (uint64_t)L);
}

// Edge (a, b) crosses the ray from c towards +x: half-open straddle in y,
// crossing strictly right of c (Algorithm 2 ray casting).  All points lie in
// the grid, so every difference fits 32 bits.
__device__ __forceinline__ bool edge_crosses_right(int32_t ax, int32_t ay, int32_t bx, int32_t by,
                                                   int32_t cx, int32_t cy) {
    if ((ay > cy) == (by > cy)) return false;
    int32_t lx = ax, ly = ay, hx = bx, hy = by;
    if (ay > by) {
        lx = bx; ly = by; hx = ax; hy = ay;
    }
    int64_t num = (int64_t)(hx - lx) * (cy - ly) - (int64_t)(cx - lx) * (hy - ly);
    return num > 0;
}

__device__ __forceinline__ bool box_hit(int4 b, int32_t x0, int32_t y0, int32_t x1, int32_t y1) {
    return b.x <= x1 && b.z >= x0 && b.y <= y1 && b.w >= y0;
}

}  // namespace hv
