// Index build: Hilbert-packed R-trees on the device (replaces the Boost
// R-trees RtreeP / RtreeL / RtreeE / RtreeMBR of HiVision Sec. 3.1).
//
// Objects are sorted by the 62-bit Hilbert key of their box centre, packed
// 32 to a leaf, and every inner node stores the 32 boxes of its children as
// SoA int32 so one warp reads a node with four coalesced 128-byte loads.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "hv_device.cuh"
#include "hv_internal.h"

namespace hv {

namespace {

struct PointObj {
    using T = int2;
    __device__ static int4 box(int2 p) { return make_int4(p.x, p.y, p.x, p.y); }
};
struct SegObj {
    using T = int4;
    __device__ static int4 box(int4 s) {
        return make_int4(min(s.x, s.z), min(s.y, s.w), max(s.x, s.z), max(s.y, s.w));
    }
};
struct BoxObj {
    using T = int4;
    __device__ static int4 box(int4 b) { return b; }
};
struct PieceObj {
    using T = Piece;
    __device__ static int4 box(const Piece& p) { return p.box; }
};

template <class O>
__global__ void k_keys(const typename O::T* obj, uint64_t n, uint64_t* keys, uint32_t* idx) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const typename O::T o = obj[i];
    int4 b = O::box(o);
    uint64_t k;
    if (b.x > b.z) {
        k = (1ull << 62) - 1;  // empty box: sorts last, never intersects
    } else {
        k = hilbert_key(mid32(b.x, b.z), mid32(b.y, b.w));
    }
    keys[i] = k;
    idx[i] = (uint32_t)i;
}

template <class T>
__global__ void k_gather(const T* src, const uint32_t* idx, uint64_t n, T* dst) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

__device__ __forceinline__ int4 warp_union(int4 b) {
    return make_int4(__reduce_min_sync(kFull, b.x), __reduce_min_sync(kFull, b.y),
                     __reduce_max_sync(kFull, b.z), __reduce_max_sync(kFull, b.w));
}

// Leaf boxes: one warp per leaf of 32 consecutive objects.
template <class O>
__global__ void k_leaf_boxes(const typename O::T* obj, uint64_t n, uint64_t n_leaf, int4* box) {
    uint64_t leaf = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (leaf >= n_leaf) return;
    uint64_t i = leaf * 32 + lane;
    int4 b = make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
    if (i < n) {
        const typename O::T o = obj[i];
        b = O::box(o);
    }
    b = warp_union(b);
    if (lane == 0) box[leaf] = b;
}

// One inner level: node k stores the boxes of children [32k, 32k+32) as SoA
// and its own box is their union.
__global__ void k_level(const int4* child_box, uint64_t n_child, uint64_t n_node, int32_t* nodes,
                        int4* node_box) {
    uint64_t k = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= n_node) return;
    uint64_t c = k * 32 + lane;
    int4 b = c < n_child ? child_box[c] : make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
    int32_t* nd = nodes + k * 128;
    nd[lane] = b.x;
    nd[32 + lane] = b.y;
    nd[64 + lane] = b.z;
    nd[96 + lane] = b.w;
    b = warp_union(b);
    if (lane == 0) node_box[k] = b;
}

uint32_t grid_for(uint64_t threads, uint32_t block) { return (uint32_t)((threads + block - 1) / block); }

struct Tmp {
    Ctx* c;
    std::vector<std::pair<void*, uint64_t>> v;
    explicit Tmp(Ctx* c_) : c(c_) {}
    int get(void** p, uint64_t bytes) {
        int rc = dev_alloc(c, p, bytes ? bytes : 16);
        if (rc == HV_OK) v.push_back({*p, bytes ? bytes : 16});
        return rc;
    }
    ~Tmp() {
        for (auto& a : v) dev_free(c, a.first, a.second);
    }
};

// Sort objects by Hilbert key; returns sorted objects (replacing *obj), the
// sorted keys and optionally the permutation.
template <class O>
int sort_objects(Ctx* c, typename O::T** obj, uint64_t n, uint64_t** keys_out, uint32_t** perm_out) {
    using T = typename O::T;
    Tmp tmp(c);
    uint64_t *k_in, *k_out;
    uint32_t *i_in, *i_out;
    HV_TRY(tmp.get((void**)&k_in, n * 8));
    HV_TRY(tmp.get((void**)&i_in, n * 4));
    HV_TRY(dev_alloc(c, (void**)&k_out, n * 8));
    int rc = tmp.get((void**)&i_out, n * 4);
    if (rc != HV_OK) { dev_free(c, k_out, n * 8); return rc; }
    k_keys<O><<<grid_for(n, 256), 256>>>(*obj, n, k_in, i_in);
    size_t temp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, k_in, k_out, i_in, i_out, (int64_t)n, 0, 62);
    void* temp;
    rc = tmp.get(&temp, temp_bytes);
    if (rc != HV_OK) { dev_free(c, k_out, n * 8); return rc; }
    cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, k_in, k_out, i_in, i_out,
                                                    (int64_t)n, 0, 62);
    if (e != cudaSuccess) {
        dev_free(c, k_out, n * 8);
        set_error("radix sort failed: %s", cudaGetErrorString(e));
        return HV_ECUDA;
    }
    T* sorted;
    rc = dev_alloc(c, (void**)&sorted, n * sizeof(T));
    if (rc != HV_OK) { dev_free(c, k_out, n * 8); return rc; }
    k_gather<T><<<grid_for(n, 256), 256>>>(*obj, i_out, n, sorted);
    if (perm_out) {
        uint32_t* perm;
        rc = dev_alloc(c, (void**)&perm, n * 4);
        if (rc != HV_OK) { dev_free(c, k_out, n * 8); dev_free(c, sorted, n * sizeof(T)); return rc; }
        cudaMemcpyAsync(perm, i_out, n * 4, cudaMemcpyDeviceToDevice);
        *perm_out = perm;
    }
    HV_CUDA(cudaGetLastError());
    HV_CUDA(cudaDeviceSynchronize());
    dev_free(c, *obj, n * sizeof(T));
    *obj = sorted;
    *keys_out = k_out;
    return HV_OK;
}

// Build the inner levels over sorted objects.
template <class O>
int build_levels(Ctx* c, const typename O::T* obj, uint64_t n, Tree* t) {
    *t = Tree();
    t->view.n_obj = n;
    if (n == 0) return HV_OK;
    Tmp tmp(c);
    uint64_t n_leaf = (n + 31) / 32;
    // count nodes per level
    uint64_t counts[kMaxLevels + 1] = {};
    uint64_t below = n_leaf, total = 0;
    int top = 0;
    do {
        top++;
        if (top > kMaxLevels) { set_error("tree too deep"); return HV_EINVAL; }
        counts[top] = (below + 31) / 32;
        total += counts[top];
        below = counts[top];
    } while (below > 1);
    int4 *box_a, *box_b;
    HV_TRY(tmp.get((void**)&box_a, n_leaf * 16));
    HV_TRY(tmp.get((void**)&box_b, ((n_leaf + 31) / 32) * 16 + 16));
    HV_TRY(dev_alloc(c, (void**)&t->nodes, total * 512));
    t->nodes_bytes = total * 512;
    t->n_nodes = total;
    k_leaf_boxes<O><<<grid_for(n_leaf * 32, 256), 256>>>(obj, n, n_leaf, box_a);
    uint64_t off = 0, n_child = n_leaf;
    for (int l = 1; l <= top; l++) {
        t->view.level_off[l] = off;
        t->view.level_n[l] = counts[l];
        k_level<<<grid_for(counts[l] * 32, 256), 256>>>(box_a, n_child, counts[l],
                                                        t->nodes + off * 128, box_b);
        off += counts[l];
        n_child = counts[l];
        int4* s = box_a; box_a = box_b; box_b = s;
    }
    HV_CUDA(cudaGetLastError());
    int4 root;
    HV_CUDA(cudaMemcpy(&root, box_a, 16, cudaMemcpyDeviceToHost));
    t->view.nodes = t->nodes;
    t->view.top = top;
    t->view.root_box = root;
    return HV_OK;
}

// ---- polygon preparation ----------------------------------------------------

__device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t* a, uint64_t n, uint64_t v) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Edge v joins vertex v to the next vertex of its ring (rings close implicitly).
__global__ void k_ring_edges(const int2* xy, uint64_t n_vert, const uint64_t* ring_off,
                             uint64_t n_rings, int4* edges) {
    uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= n_vert) return;
    uint64_t r = upper_bound_u64(ring_off, n_rings + 1, v) - 1;
    uint64_t w = v + 1 < ring_off[r + 1] ? v + 1 : ring_off[r];
    int2 a = xy[v], b = xy[w];
    edges[v] = make_int4(a.x, a.y, b.x, b.y);
}

// Segment for vertex v of line l when v + 1 is still in the line.
__global__ void k_line_segments(const int2* xy, uint64_t n_vert, const uint64_t* line_off,
                                uint64_t n_lines, const uint64_t* seg_start, int4* segs) {
    uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= n_vert) return;
    uint64_t l = upper_bound_u64(line_off, n_lines + 1, v) - 1;
    if (v + 1 >= line_off[l + 1]) return;
    int2 a = xy[v], b = xy[v + 1];
    segs[seg_start[l] + (v - line_off[l])] = make_int4(a.x, a.y, b.x, b.y);
}

// Polygon boxes and edge offsets: one warp per polygon.
__global__ void k_poly_boxes(const int4* edges, const uint64_t* ring_off, const uint64_t* poly_ring_off,
                             uint64_t n_poly, uint64_t* edge_off, int4* boxes) {
    uint64_t p = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (p >= n_poly) return;
    uint64_t e0 = ring_off[poly_ring_off[p]], e1 = ring_off[poly_ring_off[p + 1]];
    int4 b = make_int4(kEmptyLo, kEmptyLo, kEmptyHi, kEmptyHi);
    for (uint64_t e = e0 + lane; e < e1; e += 32) {
        int4 s = edges[e];
        b.x = min(b.x, min(s.x, s.z));
        b.y = min(b.y, min(s.y, s.w));
        b.z = max(b.z, max(s.x, s.z));
        b.w = max(b.w, max(s.y, s.w));
    }
    b = warp_union(b);
    if (lane == 0) {
        boxes[p] = b;
        edge_off[p] = e0;
        if (p + 1 == n_poly) edge_off[n_poly] = e1;
    }
}

// ---- segment pieces ----------------------------------------------------------

__device__ __forceinline__ int64_t seg_extent(int4 s) {
    int64_t dx = (int64_t)s.z - s.x, dy = (int64_t)s.w - s.y;
    dx = dx < 0 ? -dx : dx;
    dy = dy < 0 ? -dy : dy;
    return dx > dy ? dx : dy;
}

// Histogram of the bit lengths of the segments' extents: counted per block
// in shared memory, then added to the 65 global counters once per block
// (one global atomic per object contended on 65 addresses).
__global__ void k_extent_bits(const int4* segs, uint64_t n, unsigned long long* hist) {
    __shared__ unsigned int h[65];
    for (int k = threadIdx.x; k < 65; k += blockDim.x) h[k] = 0u;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[64 - __clzll((unsigned long long)seg_extent(segs[i]))], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < 65; k += blockDim.x)
        if (h[k]) atomicAdd(hist + k, (unsigned long long)h[k]);
}

constexpr uint32_t kMaxPieces = 4096;

__global__ void k_widen(const uint32_t* a, uint64_t n, uint64_t* b) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void k_piece_count(const int4* segs, uint64_t n, int shift, uint32_t* cnt) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t m = ((uint64_t)seg_extent(segs[i]) >> shift) + 1;
    cnt[i] = (uint32_t)(m < kMaxPieces ? m : kMaxPieces);
}

__device__ __forceinline__ int64_t floordiv64(int64_t a, int64_t b) {
    int64_t q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Piece k of m covers the parameter interval [k/m, (k+1)/m]; along each axis
// the segment moves monotonically, so the piece lies between its two end
// positions, rounded outwards to the grid.
__global__ void k_emit_pieces(const int4* segs, uint64_t n, const uint32_t* cnt, const uint64_t* off,
                              Piece* out) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 s = segs[i];
    int64_t m = cnt[i];
    int64_t dx = (int64_t)s.z - s.x, dy = (int64_t)s.w - s.y;
    uint64_t o = off[i];
    for (int64_t k = 0; k < m; k++) {
        int64_t xa = floordiv64(dx * k, m), xb = floordiv64(dx * (k + 1), m);
        int64_t ya = floordiv64(dy * k, m), yb = floordiv64(dy * (k + 1), m);
        // exact positions lie in [floor, floor + 1)
        int64_t x0 = s.x + (xa < xb ? xa : xb), x1 = s.x + (xa > xb ? xa : xb) + 1;
        int64_t y0 = s.y + (ya < yb ? ya : yb), y1 = s.y + (ya > yb ? ya : yb) + 1;
        int4 b = make_int4((int32_t)max(x0, (int64_t)min(s.x, s.z)), (int32_t)max(y0, (int64_t)min(s.y, s.w)),
                           (int32_t)min(x1, (int64_t)max(s.x, s.z)), (int32_t)min(y1, (int64_t)max(s.y, s.w)));
        out[o + k] = Piece{s, b};
    }
}

}  // namespace

// Split n segments into pieces of extent at most 2^shift (the smallest power
// of two, at least 2^12, for which the pieces number at most 4n).
int make_pieces(Ctx* c, const int4* segs, uint64_t n, Piece** out, uint64_t* n_out, int32_t* extent) {
    *out = nullptr;
    *n_out = 0;
    *extent = 0;
    if (n == 0) return HV_OK;
    Tmp tmp(c);
    unsigned long long* hist;
    HV_TRY(tmp.get((void**)&hist, 65 * 8));
    HV_CUDA(cudaMemset(hist, 0, 65 * 8));
    k_extent_bits<<<(uint32_t)std::min<uint64_t>(grid_for(n, 256), 4096), 256>>>(segs, n, hist);
    unsigned long long h[65];
    HV_CUDA(cudaMemcpy(h, hist, sizeof(h), cudaMemcpyDeviceToHost));
    int shift = 12;
    for (; shift < 31; shift++) {
        // an extent of bit length b is < 2^b: at most (2^b >> shift) + 1 pieces
        double total = 0;
        for (int b = 0; b < 65; b++) total += (double)h[b] * (double)(((b >= 63 ? ~0ull : (1ull << b)) >> shift) + 1);
        if (total <= 4.0 * (double)n) break;
    }
    uint32_t* cnt;
    uint64_t *cnt64, *off;
    HV_TRY(tmp.get((void**)&cnt, n * 4));
    HV_TRY(tmp.get((void**)&cnt64, (n + 1) * 8));
    HV_TRY(tmp.get((void**)&off, (n + 1) * 8));
    k_piece_count<<<grid_for(n, 256), 256>>>(segs, n, shift, cnt);
    // 64-bit exclusive prefix sum of the counts (entry n holds the total)
    HV_CUDA(cudaMemset(cnt64, 0, (n + 1) * 8));
    k_widen<<<grid_for(n, 256), 256>>>(cnt, n, cnt64);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt64, off, (int64_t)(n + 1));
    void* temp;
    HV_TRY(tmp.get(&temp, tb));
    HV_CUDA(cub::DeviceScan::ExclusiveSum(temp, tb, cnt64, off, (int64_t)(n + 1)));
    uint64_t total = 0;
    HV_CUDA(cudaMemcpy(&total, off + n, 8, cudaMemcpyDeviceToHost));
    if (total >= (1ull << 32)) { set_error("too many segment pieces"); return HV_EINVAL; }
    HV_TRY(dev_alloc(c, (void**)out, total * sizeof(Piece)));
    k_emit_pieces<<<grid_for(n, 256), 256>>>(segs, n, cnt, off, *out);
    HV_CUDA(cudaGetLastError());
    HV_CUDA(cudaDeviceSynchronize());
    *n_out = total;
    *extent = (int32_t)(1u << shift);
    return HV_OK;
}

void free_tree(Ctx* c, Tree* t) {
    if (t->nodes) dev_free(c, t->nodes, t->nodes_bytes);
    *t = Tree();
}

int build_tree_points(Layer* L) {
    Ctx* c = L->ctx;
    if (L->n_obj) {
        HV_TRY(sort_objects<PointObj>(c, (int2**)&L->obj, L->n_obj, &L->keys, nullptr));
    }
    HV_TRY(build_levels<PointObj>(c, (const int2*)L->obj, L->n_obj, &L->tree));
    HV_CUDA(cudaDeviceSynchronize());
    return HV_OK;
}

// Segments (and polygon edges) are indexed as pieces: sort the pieces by
// the Hilbert key of their box centre and build the tree over their boxes.
static int build_piece_tree(Layer* L, const int4* segs, uint64_t n_seg) {
    Ctx* c = L->ctx;
    Piece* pieces = nullptr;
    uint64_t n = 0;
    HV_TRY(make_pieces(c, segs, n_seg, &pieces, &n, &L->piece_extent));
    if (L->obj) dev_free(c, L->obj, L->obj_bytes);
    L->obj = pieces;
    L->obj_bytes = n * sizeof(Piece);
    L->n_obj = n;
    if (n) HV_TRY(sort_objects<PieceObj>(c, (Piece**)&L->obj, n, &L->keys, nullptr));
    HV_TRY(build_levels<PieceObj>(c, (const Piece*)L->obj, n, &L->tree));
    return HV_OK;
}

int build_tree_segments(Layer* L) {
    // the input segments are replaced by their pieces
    int4* segs = (int4*)L->obj;
    uint64_t n = L->n_src, bytes = L->obj_bytes;
    L->obj = nullptr;
    L->obj_bytes = 0;
    int rc = build_piece_tree(L, segs, n);
    dev_free(L->ctx, segs, bytes);
    HV_TRY(rc);
    HV_CUDA(cudaDeviceSynchronize());
    return HV_OK;
}

int build_tree_polygons(Layer* L) {
    Ctx* c = L->ctx;
    // the edge tree (outline) over pieces of the polygon-order edges
    HV_TRY(build_piece_tree(L, L->poly_edges, L->n_src));
    // the polygon-box tree (fill)
    if (L->n_poly) {
        HV_TRY(sort_objects<BoxObj>(c, &L->mbr_obj, L->n_poly, &L->mbr_keys, &L->mbr_ids));
    }
    HV_TRY(build_levels<BoxObj>(c, L->mbr_obj, L->n_poly, &L->mbr_tree));
    HV_CUDA(cudaDeviceSynchronize());
    return HV_OK;
}

// A side R-tree over `n` boxes or segments (the learned index's long
// objects), with the ids carried along; takes ownership of objs and ids.
int build_side_tree(Ctx* c, int4* objs, uint32_t* ids, uint64_t n, Tree* t, int4** sorted_objs,
                    uint32_t** sorted_ids) {
    uint64_t* keys = nullptr;
    uint32_t* perm = nullptr;
    HV_TRY(sort_objects<SegObj>(c, &objs, n, &keys, &perm));
    // ids follow the sort
    uint32_t* sid;
    HV_TRY(dev_alloc(c, (void**)&sid, n * 4));
    k_gather<uint32_t><<<grid_for(n, 256), 256>>>(ids, perm, n, sid);
    HV_CUDA(cudaDeviceSynchronize());
    dev_free(c, ids, n * 4);
    dev_free(c, perm, n * 4);
    dev_free(c, keys, n * 8);
    HV_TRY(build_levels<SegObj>(c, objs, n, t));
    *sorted_objs = objs;
    *sorted_ids = sid;
    return HV_OK;
}

// ---- A0: layer preparation on the device (used by hv_api.cu) ---------------

int prepare_lines(Ctx* c, const int2* d_xy, uint64_t n_vert, const uint64_t* h_line_off,
                  uint64_t n_lines, int4** segs_out, uint64_t* n_seg_out) {
    std::vector<uint64_t> start(n_lines + 1, 0);
    for (uint64_t l = 0; l < n_lines; l++) {
        uint64_t nv = h_line_off[l + 1] - h_line_off[l];
        start[l + 1] = start[l] + (nv >= 2 ? nv - 1 : 0);
    }
    uint64_t n_seg = start[n_lines];
    *n_seg_out = n_seg;
    *segs_out = nullptr;
    if (n_seg == 0) return HV_OK;
    Tmp tmp(c);
    uint64_t *d_off, *d_start;
    HV_TRY(tmp.get((void**)&d_off, (n_lines + 1) * 8));
    HV_TRY(tmp.get((void**)&d_start, (n_lines + 1) * 8));
    HV_CUDA(cudaMemcpy(d_off, h_line_off, (n_lines + 1) * 8, cudaMemcpyHostToDevice));
    HV_CUDA(cudaMemcpy(d_start, start.data(), (n_lines + 1) * 8, cudaMemcpyHostToDevice));
    HV_TRY(dev_alloc(c, (void**)segs_out, n_seg * 16));
    k_line_segments<<<grid_for(n_vert, 256), 256>>>(d_xy, n_vert, d_off, n_lines, d_start, *segs_out);
    HV_CUDA(cudaGetLastError());
    HV_CUDA(cudaDeviceSynchronize());
    return HV_OK;
}

int prepare_polygons(Ctx* c, const int2* d_xy, uint64_t n_vert, const uint64_t* h_ring_off,
                     uint64_t n_rings, const uint64_t* h_poly_ring_off, uint64_t n_polys, Layer* L) {
    Tmp tmp(c);
    uint64_t *d_ro, *d_pro;
    HV_TRY(tmp.get((void**)&d_ro, (n_rings + 1) * 8));
    HV_TRY(tmp.get((void**)&d_pro, (n_polys + 1) * 8));
    HV_CUDA(cudaMemcpy(d_ro, h_ring_off, (n_rings + 1) * 8, cudaMemcpyHostToDevice));
    HV_CUDA(cudaMemcpy(d_pro, h_poly_ring_off, (n_polys + 1) * 8, cudaMemcpyHostToDevice));
    L->n_obj = n_vert;
    L->n_src = n_vert;
    L->n_poly = n_polys;
    HV_TRY(dev_alloc(c, (void**)&L->poly_edges, (n_vert ? n_vert : 1) * 16));
    HV_TRY(dev_alloc(c, (void**)&L->poly_edge_off, (n_polys + 1) * 8));
    HV_TRY(dev_alloc(c, (void**)&L->mbr_obj, (n_polys ? n_polys : 1) * 16));
    if (n_vert) k_ring_edges<<<grid_for(n_vert, 256), 256>>>(d_xy, n_vert, d_ro, n_rings, L->poly_edges);
    if (n_polys) {
        k_poly_boxes<<<grid_for(n_polys * 32, 256), 256>>>(L->poly_edges, d_ro, d_pro, n_polys,
                                                           L->poly_edge_off, L->mbr_obj);
    } else {
        HV_CUDA(cudaMemset(L->poly_edge_off, 0, 8));
    }
    HV_CUDA(cudaGetLastError());
    HV_CUDA(cudaDeviceSynchronize());
    return HV_OK;
}

}  // namespace hv
