// The C ABI: contexts, layer registration (HiVision Sec. 4.1, Register Vector
// Data), index builds and tile rendering (Sec. 4.1, Parse Tasks / Render Tiles).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "hv_device.cuh"
#include "hv_internal.h"

namespace hv {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int dev_alloc(Ctx* c, void** p, uint64_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (c->budget && c->held + bytes > c->budget) {
            set_error("device memory budget exceeded: %llu held + %llu requested > %llu",
                      (unsigned long long)c->held, (unsigned long long)bytes,
                      (unsigned long long)c->budget);
            return HV_ENOMEM;
        }
        c->held += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> g(c->mu);
        c->held -= bytes;
        *p = nullptr;
        set_error("cudaMalloc(%llu) failed: %s", (unsigned long long)bytes, cudaGetErrorString(e));
        return HV_ENOMEM;
    }
    return HV_OK;
}

void dev_free(Ctx* c, void* p, uint64_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    cudaFree(p);
    std::lock_guard<std::mutex> g(c->mu);
    c->held -= std::min(c->held, bytes);
}

// The device address of pinned (page-locked) host memory, or NULL for other
// memory: pinned host memory is mapped into the device's address space.
static void* pinned_device_view(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Is `p` device-accessible memory that is not host memory?
static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int prepare_lines(Ctx* c, const int2* d_xy, uint64_t n_vert, const uint64_t* h_line_off,
                  uint64_t n_lines, int4** segs_out, uint64_t* n_seg_out);
int prepare_polygons(Ctx* c, const int2* d_xy, uint64_t n_vert, const uint64_t* h_ring_off,
                     uint64_t n_rings, const uint64_t* h_poly_ring_off, uint64_t n_polys, Layer* L);

namespace {

__global__ void k_check_coords(const int32_t* xy, uint64_t n, uint32_t* bad) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        int32_t v = xy[i];
        if (v < -kGridHalf || v > kGridHalf - 1) atomicOr(bad, 1u);
    }
}

// Copy `n` vertices (host or device) into a fresh device array and check the
// grid range on the device (A0: coordinates arrive quantised to the grid).
int upload_vertices(Ctx* c, const int32_t* xy, uint64_t n, int2** out) {
    *out = nullptr;
    HV_TRY(dev_alloc(c, (void**)out, n * 8));
    if (n == 0) return HV_OK;
    cudaMemcpyKind kind = is_device_ptr(xy) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpy(*out, xy, n * 8, kind);
    uint32_t* bad = nullptr;
    if (e == cudaSuccess) {
        int rc = dev_alloc(c, (void**)&bad, 4);
        if (rc != HV_OK) { dev_free(c, *out, n * 8); *out = nullptr; return rc; }
        cudaMemset(bad, 0, 4);
        uint64_t cnt = 2 * n;
        k_check_coords<<<(unsigned)((cnt + 255) / 256), 256>>>((const int32_t*)*out, cnt, bad);
        uint32_t h = 0;
        e = cudaMemcpy(&h, bad, 4, cudaMemcpyDeviceToHost);
        dev_free(c, bad, 4);
        if (e == cudaSuccess && h) {
            dev_free(c, *out, n * 8);
            *out = nullptr;
            set_error("a coordinate lies outside [-2^30, 2^30)");
            return HV_ERANGE;
        }
    }
    if (e != cudaSuccess) {
        dev_free(c, *out, n * 8);
        *out = nullptr;
        set_error("vertex upload failed: %s", cudaGetErrorString(e));
        return HV_ECUDA;
    }
    return HV_OK;
}

int check_offsets(const uint64_t* off, uint64_t n, uint64_t total, const char* what) {
    if (!off) { set_error("%s offsets are NULL", what); return HV_EINVAL; }
    if (off[0] != 0 || off[n] != total) {
        set_error("%s offsets must start at 0 and end at %llu", what, (unsigned long long)total);
        return HV_EINVAL;
    }
    for (uint64_t i = 0; i < n; i++)
        if (off[i + 1] < off[i]) { set_error("%s offsets decrease at %llu", what, (unsigned long long)i); return HV_EINVAL; }
    return HV_OK;
}

Layer* new_layer(Ctx* c, int kind) {
    Layer* L = new Layer();
    L->ctx = c;
    L->kind = kind;
    return L;
}

void free_layer(Layer* L) {
    Ctx* c = L->ctx;
    if (L->obj_host)
        cudaFreeHost(L->obj_host);
    else
        dev_free(c, L->obj, L->obj_bytes);
    if (L->keys) dev_free(c, L->keys, L->n_obj * 8);
    free_tree(c, &L->tree);
    if (L->kind == HV_LAYER_POLYGONS) {
        if (L->edges_host)
            cudaFreeHost(L->edges_host);
        else
            dev_free(c, L->poly_edges, (L->n_src ? L->n_src : 1) * 16);
        dev_free(c, L->poly_edge_off, (L->n_poly + 1) * 8);
        dev_free(c, L->mbr_obj, (L->n_poly ? L->n_poly : 1) * 16);
        if (L->mbr_ids) dev_free(c, L->mbr_ids, L->n_poly * 4);
        if (L->mbr_keys) dev_free(c, L->mbr_keys, L->n_poly * 8);
        free_tree(c, &L->mbr_tree);
    }
    free_learned(c, &L->learned);
    free_learned(c, &L->mbr_learned);
    if (L->status) dev_free(c, L->status, 16);
    for (auto& a : L->extra) dev_free(c, a.first, a.second);
    delete L;
}

int finish_layer(Layer* L, hv_layer** out) {
    // status word, pad, and the record of the first failed internal check
    int rc = dev_alloc(L->ctx, (void**)&L->status, 16);
    if (rc == HV_OK && cudaMemset(L->status, 0, 16) != cudaSuccess) rc = HV_ECUDA;
    if (rc != HV_OK) { free_layer(L); return rc; }
    *out = (hv_layer*)L;
    return HV_OK;
}

int grow(Ctx* c, void** buf, uint64_t* cap, uint64_t need) {
    if (*cap >= need) return HV_OK;
    if (*buf) dev_free(c, *buf, *cap);
    *buf = nullptr;
    *cap = 0;
    uint64_t want = std::max<uint64_t>(need, 1 << 20);
    HV_TRY(dev_alloc(c, buf, want));
    *cap = want;
    return HV_OK;
}

}  // namespace

void free_layer_public(Layer* L) { free_layer(L); }

}  // namespace hv

using namespace hv;

extern "C" {

const char* hv_last_error(void) { return g_err; }

uint64_t hv_tile_bytes(int mode) {
    switch (mode) {
        case HV_MODE_MASK: return kTile * kTile / 8;
        case HV_MODE_COVERAGE: return kTile * kTile;
        case HV_MODE_RGBA: return kTile * kTile * 4;
        default: return 0;
    }
}

int hv_create(hv_ctx** out, int device, uint64_t mem_budget) {
    if (!out) { set_error("hv_create: out is NULL"); return HV_EINVAL; }
    *out = nullptr;
    int n = 0;
    HV_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) { set_error("hv_create: no CUDA device %d", device); return HV_EINVAL; }
    HV_CUDA(cudaSetDevice(device));
    Ctx* c = new Ctx();
    c->device = device;
    c->budget = mem_budget;
    *out = (hv_ctx*)c;
    return HV_OK;
}

int hv_destroy(hv_ctx* ctx) {
    if (!ctx) return HV_EINVAL;
    Ctx* c = (Ctx*)ctx;
    cudaSetDevice(c->device);
    if (c->req_buf) dev_free(c, c->req_buf, c->req_cap);
    if (c->out_buf) dev_free(c, c->out_buf, c->out_cap);
    if (c->overlay_buf) dev_free(c, c->overlay_buf, c->overlay_cap);
    if (c->pinned_req) cudaFreeHost(c->pinned_req);
    for (int k = 0; k < 2; k++) {
        if (c->ev_rendered[k]) cudaEventDestroy(c->ev_rendered[k]);
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    delete c;
    return HV_OK;
}

int hv_lonlat_to_grid(const double* lonlat, uint64_t n, int32_t* xy) {
    if (n && (!lonlat || !xy)) { set_error("hv_lonlat_to_grid: NULL argument"); return HV_EINVAL; }
    const double kPi = 3.14159265358979323846;
    // atan(sinh(pi)) in degrees, with room for the rounding of a caller's own copy
    const double lat_max = atan(sinh(kPi)) * 180.0 / kPi + 1e-9;
    for (uint64_t i = 0; i < n; i++) {
        const double lon = lonlat[2 * i], lat = lonlat[2 * i + 1];
        if (!(lon >= -180.0 && lon <= 180.0 && lat >= -lat_max && lat <= lat_max)) {
            set_error("hv_lonlat_to_grid: point %llu (%g, %g) outside the Web-Mercator square",
                      (unsigned long long)i, lon, lat);
            return HV_ERANGE;
        }
    }
    const double scale = 2147483648.0;   // 2^31 grid units per axis
    for (uint64_t i = 0; i < n; i++) {
        const double u = (lonlat[2 * i] + 180.0) / 360.0;
        const double v = 0.5 - asinh(tan(lonlat[2 * i + 1] * kPi / 180.0)) / (2.0 * kPi);
        const int64_t gx = (int64_t)floor(u * scale) - kGridHalf, gy = (int64_t)floor(v * scale) - kGridHalf;
        xy[2 * i] = (int32_t)std::min<int64_t>(std::max<int64_t>(gx, -kGridHalf), kGridHalf - 1);
        xy[2 * i + 1] = (int32_t)std::min<int64_t>(std::max<int64_t>(gy, -kGridHalf), kGridHalf - 1);
    }
    return HV_OK;
}

int hv_route_tiles(const hv_tile_req* reqs, uint64_t n, uint32_t n_ranks, uint32_t* rank_out) {
    if ((n && (!reqs || !rank_out)) || n_ranks == 0) { set_error("hv_route_tiles: bad arguments"); return HV_EINVAL; }
    for (uint64_t i = 0; i < n; i++) {
        const hv_tile_req& q = reqs[i];
        // a unique key per tile (x, y < 2^20 at z <= 19), mixed (splitmix64),
        // then scaled to the ranks by the high half of a 64 x 32-bit product
        uint64_t h = ((uint64_t)q.layer << 45) ^ ((uint64_t)(q.z & 31) << 40) ^ ((uint64_t)(q.x & 0xFFFFF) << 20) ^
                     (uint64_t)(q.y & 0xFFFFF);
        h += 0x9E3779B97F4A7C15ull;
        h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
        h = (h ^ (h >> 27)) * 0x94D049BB133111EBull;
        h ^= h >> 31;
        rank_out[i] = (uint32_t)(((h >> 32) * (uint64_t)n_ranks) >> 32);
    }
    return HV_OK;
}

int hv_ctx_device_bytes(hv_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) { set_error("hv_ctx_device_bytes: NULL argument"); return HV_EINVAL; }
    Ctx* c = (Ctx*)ctx;
    std::lock_guard<std::mutex> g(c->mu);
    *out = c->held;
    return HV_OK;
}

int hv_layer_load_points(hv_ctx* ctx, const int32_t* xy, uint64_t n, hv_layer** out) {
    if (!ctx || !out || (!xy && n)) { set_error("hv_layer_load_points: NULL argument"); return HV_EINVAL; }
    if (n >= (1ull << 32)) { set_error("a layer holds fewer than 2^32 objects"); return HV_EINVAL; }
    Ctx* c = (Ctx*)ctx;
    HV_CUDA(cudaSetDevice(c->device));
    Layer* L = new_layer(c, HV_LAYER_POINTS);
    int2* d;
    int rc = upload_vertices(c, xy, n, &d);
    if (rc != HV_OK) { free_layer(L); return rc; }
    L->obj = d;
    L->obj_bytes = n * 8;
    L->n_obj = n;
    L->n_src = n;
    return finish_layer(L, out);
}

int hv_layer_load_linestrings(hv_ctx* ctx, const int32_t* xy, uint64_t n_vert, const uint64_t* line_off,
                              uint64_t n_lines, hv_layer** out) {
    if (!ctx || !out || (!xy && n_vert)) { set_error("hv_layer_load_linestrings: NULL argument"); return HV_EINVAL; }
    HV_TRY(check_offsets(line_off, n_lines, n_vert, "line"));
    if (n_vert >= (1ull << 32)) { set_error("a layer holds fewer than 2^32 vertices"); return HV_EINVAL; }
    Ctx* c = (Ctx*)ctx;
    HV_CUDA(cudaSetDevice(c->device));
    Layer* L = new_layer(c, HV_LAYER_LINES);
    int2* d;
    int rc = upload_vertices(c, xy, n_vert, &d);
    if (rc != HV_OK) { free_layer(L); return rc; }
    int4* segs = nullptr;
    uint64_t n_seg = 0;
    rc = prepare_lines(c, d, n_vert, line_off, n_lines, &segs, &n_seg);
    dev_free(c, d, n_vert * 8);
    if (rc != HV_OK) { free_layer(L); return rc; }
    L->obj = segs;
    L->obj_bytes = n_seg ? n_seg * 16 : 0;
    L->n_obj = n_seg;
    L->n_src = n_seg;
    return finish_layer(L, out);
}

int hv_layer_load_polygons(hv_ctx* ctx, const int32_t* xy, uint64_t n_vert, const uint64_t* ring_off,
                           uint64_t n_rings, const uint64_t* poly_ring_off, uint64_t n_polys, hv_layer** out) {
    if (!ctx || !out || (!xy && n_vert)) { set_error("hv_layer_load_polygons: NULL argument"); return HV_EINVAL; }
    HV_TRY(check_offsets(ring_off, n_rings, n_vert, "ring"));
    HV_TRY(check_offsets(poly_ring_off, n_polys, n_rings, "polygon"));
    if (n_vert >= (1ull << 32) || n_polys >= (1ull << 32)) { set_error("a layer holds fewer than 2^32 edges"); return HV_EINVAL; }
    Ctx* c = (Ctx*)ctx;
    HV_CUDA(cudaSetDevice(c->device));
    Layer* L = new_layer(c, HV_LAYER_POLYGONS);
    int2* d;
    int rc = upload_vertices(c, xy, n_vert, &d);
    if (rc != HV_OK) { free_layer(L); return rc; }
    rc = prepare_polygons(c, d, n_vert, ring_off, n_rings, poly_ring_off, n_polys, L);
    dev_free(c, d, n_vert * 8);
    if (rc != HV_OK) { free_layer(L); return rc; }
    return finish_layer(L, out);
}

}  // extern "C"

namespace hv {

// Move a device array into mapped pinned host memory; *p becomes its device
// address (read over the CPU-GPU link), *host its host address.
static int move_to_host(Ctx* c, void** p, uint64_t bytes, void** host) {
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, bytes ? bytes : 16, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        set_error("pinned host allocation of %llu bytes failed", (unsigned long long)bytes);
        return HV_ENOMEM;
    }
    cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
    if (e == cudaSuccess && bytes) e = cudaMemcpy(h, *p, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        set_error("moving %llu bytes to host memory: %s", (unsigned long long)bytes, cudaGetErrorString(e));
        return HV_ECUDA;
    }
    dev_free(c, *p, bytes);
    *p = d;
    *host = h;
    return HV_OK;
}

}  // namespace hv

extern "C" {

int hv_layer_build_index(hv_layer* layer, uint32_t kinds, const hv_build_opts* opts) {
    if (!layer) { set_error("hv_layer_build_index: NULL layer"); return HV_EINVAL; }
    if (kinds & ~(uint32_t)(HV_INDEX_RTREE | HV_INDEX_LEARNED)) { set_error("unknown index kind"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    HV_CUDA(cudaSetDevice(L->ctx->device));
    if (!(L->indexes & HV_INDEX_RTREE)) {
        cudaEvent_t e0, e1;
        HV_CUDA(cudaEventCreate(&e0));
        HV_CUDA(cudaEventCreate(&e1));
        cudaEventRecord(e0);
        int rc = L->kind == HV_LAYER_POINTS ? build_tree_points(L)
                 : L->kind == HV_LAYER_LINES ? build_tree_segments(L)
                                             : build_tree_polygons(L);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != HV_OK) return rc;
        L->build_ms = ms;
        L->indexes |= HV_INDEX_RTREE;
        L->mbr = L->tree.view.top ? L->tree.view.root_box : make_int4(0, 0, -1, -1);
    }
    if ((kinds & HV_INDEX_LEARNED) && !(L->indexes & HV_INDEX_LEARNED)) {
        HV_TRY(build_learned(L, opts));
        L->indexes |= HV_INDEX_LEARNED;
    }
    if (opts && opts->object_placement == HV_PLACE_HOST) {
        HV_CUDA(cudaDeviceSynchronize());
        if (!L->obj_host && L->obj) HV_TRY(move_to_host(L->ctx, &L->obj, L->obj_bytes, &L->obj_host));
        if (L->kind == HV_LAYER_POLYGONS && !L->edges_host && L->poly_edges)
            HV_TRY(move_to_host(L->ctx, (void**)&L->poly_edges, (L->n_src ? L->n_src : 1) * 16, &L->edges_host));
    } else if (opts && opts->object_placement != HV_PLACE_DEVICE) {
        set_error("hv_layer_build_index: unknown object placement %u", opts->object_placement);
        return HV_EINVAL;
    }
    return HV_OK;
}

int hv_layer_info_get(hv_layer* layer, hv_layer_info* out) {
    if (!layer || !out) { set_error("hv_layer_info_get: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    memset(out, 0, sizeof(*out));
    out->kind = L->kind;
    out->indexes = L->indexes;
    out->n_objects = L->n_src;
    out->n_polygons = L->n_poly;
    out->index_records = L->n_obj;
    out->piece_extent = L->piece_extent;
    if (L->tree.view.top) {
        out->mbr[0] = L->mbr.x; out->mbr[1] = L->mbr.y; out->mbr[2] = L->mbr.z; out->mbr[3] = L->mbr.w;
    }
    out->tree_levels = L->tree.view.top;
    out->tree_nodes = L->tree.n_nodes;
    out->learned_error = L->learned.view.ready ? L->learned.view.eps : -1;
    out->learned_outliers = L->learned.n_outliers + L->mbr_learned.n_outliers;
    out->build_ms = L->build_ms;
    out->train_ms = L->learned.train_ms + L->mbr_learned.train_ms;
    const LearnedView& lv = L->learned.view;
    if (lv.ready) {
        out->learned_error_linear = lv.eps_linear;
        out->learned_error_mlp = lv.eps_mlp;
        out->learned_mean_error = lv.mean_err;
        out->learned_pieces = lv.n_seg;
        out->learned_mlp = lv.hidden > 0 ? lv.pieces_mlp : 0u;
        out->learned_mean_window = lv.mean_window;
        out->learned_mean_window_linear = lv.mean_window_linear;
        out->learned_halo = lv.halo;
    }
    uint64_t bytes = (L->obj_host ? 0 : L->obj_bytes) + (L->keys ? L->n_obj * 8 : 0) + L->tree.nodes_bytes;
    if (L->kind == HV_LAYER_POLYGONS)
        bytes += (L->edges_host ? 0 : L->n_src * 16) + (L->n_poly + 1) * 8 + L->n_poly * (16 + 4 + 8) +
                 L->mbr_tree.nodes_bytes;
    out->host_bytes = (L->obj_host ? L->obj_bytes : 0) + (L->edges_host ? L->n_src * 16 : 0);
    for (auto& a : L->learned.allocs) bytes += a.second;
    for (auto& a : L->mbr_learned.allocs) bytes += a.second;
    out->device_bytes = bytes;
    return HV_OK;
}

int hv_layer_free(hv_layer* layer) {
    if (!layer) return HV_EINVAL;
    Layer* L = (Layer*)layer;
    cudaSetDevice(L->ctx->device);
    cudaDeviceSynchronize();
    free_layer(L);
    return HV_OK;
}

}  // extern "C"

namespace hv {

// hv_render_tiles and hv_render_buffer: R_units < 0 takes each request's
// radius r16 (R = r16 * 2^(19 - z)), else R = R_units for every tile.
static int render_impl(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                       const hv_style* style, void* out, uint64_t out_bytes, void* stream, int32_t R_units,
                       const hv_fill_style* fill = nullptr) {
    if (!layer) { set_error("hv_render_tiles: NULL layer"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    uint64_t tb = hv_tile_bytes(mode);
    if (tb == 0) { set_error("hv_render_tiles: unknown mode %d", mode); return HV_EINVAL; }
    if (index_kind != HV_INDEX_RTREE && index_kind != HV_INDEX_LEARNED) {
        set_error("hv_render_tiles: index_kind must be HV_INDEX_RTREE or HV_INDEX_LEARNED");
        return HV_EINVAL;
    }
    if (!(L->indexes & index_kind)) { set_error("hv_render_tiles: index not built"); return HV_ESTATE; }
    if (n == 0) return HV_OK;
    if (!reqs || !out) { set_error("hv_render_tiles: NULL reqs or out"); return HV_EINVAL; }
    if (out_bytes < (uint64_t)n * tb) {
        set_error("hv_render_tiles: out_bytes %llu < %u tiles x %llu", (unsigned long long)out_bytes, n,
                  (unsigned long long)tb);
        return HV_EINVAL;
    }
    if (((uintptr_t)out & 15u) != 0) { set_error("hv_render_tiles: out must be 16-byte aligned"); return HV_EINVAL; }
    if (!fill_style_ok(fill)) {
        set_error("hv_render_tiles_styled: invalid fill style (flags, pattern size 1..16, texel alpha 0 or 255)");
        return HV_EINVAL;
    }
    Ctx* c = L->ctx;
    HV_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    bool dev_reqs = is_device_ptr(reqs);
    bool dev_out = is_device_ptr(out);
    // pinned host output: the kernels write the tiles straight into it over
    // the CPU-GPU link (NVLink-C2C), no staging and no copies
    void* pinned_out = dev_out ? nullptr : pinned_device_view(out);
    if (!dev_reqs) {
        for (uint32_t k = 0; k < n; k++) {
            const hv_tile_req& q = reqs[k];
            if (q.z > 19 || q.x >= (1u << q.z) || q.y >= (1u << q.z) ||
                (R_units < 0 && (q.r16 < 1 || q.r16 > 1024))) {
                set_error("hv_render_tiles: request %u (z=%u x=%u y=%u r16=%u) out of range", k, q.z, q.x,
                          q.y, q.r16);
                return HV_ERANGE;
            }
        }
    }
    // a fill pattern's texels go to a stream-ordered device copy, freed in
    // stream order after the launches that read it
    void* pattern_dev = nullptr;
    if (fill && fill->pattern_w && L->kind == HV_LAYER_POLYGONS) {
        const uint64_t pb = (uint64_t)fill->pattern_w * fill->pattern_h * 4;
        HV_CUDA(cudaMallocAsync(&pattern_dev, pb, st));
        HV_CUDA(cudaMemcpyAsync(pattern_dev, fill->pattern_rgba, pb, cudaMemcpyHostToDevice, st));
    }
    struct PatternRelease {
        void* p;
        cudaStream_t st;
        ~PatternRelease() {
            if (p) cudaFreeAsync(p, st);
        }
    } release{pattern_dev, st};
    if (dev_reqs && dev_out)
        return launch_render(L, reqs, n, mode, index_kind, style, (uint8_t*)out, st, nullptr, nullptr, R_units, fill,
                             pattern_dev);
    std::lock_guard<std::mutex> g(c->render_mu);
    const hv_tile_req* d_reqs = reqs;
    if (!dev_reqs) {
        uint64_t rb = (uint64_t)n * sizeof(hv_tile_req);
        HV_TRY(grow(c, &c->req_buf, &c->req_cap, rb));
        HV_CUDA(cudaMemcpyAsync(c->req_buf, reqs, rb, cudaMemcpyHostToDevice, st));
        d_reqs = (const hv_tile_req*)c->req_buf;
    }
    if (dev_out || pinned_out) {
        HV_TRY(launch_render(L, d_reqs, n, mode, index_kind, style, (uint8_t*)(dev_out ? out : pinned_out), st,
                             nullptr, nullptr, R_units, fill, pattern_dev));
        // the request staging must be consumed before the next call reuses
        // it, and host output must be complete when the call returns
        HV_CUDA(cudaStreamSynchronize(st));
        return HV_OK;
    }
    // Host output: render in chunks into two device buffers and copy each
    // finished chunk to the host on a second stream while the next renders.
    if (!c->copy_stream) {
        HV_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; k++) {
            HV_CUDA(cudaEventCreateWithFlags(&c->ev_rendered[k], cudaEventDisableTiming));
            HV_CUDA(cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
        }
    }
    const uint32_t chunk = n < 1024 ? n : 1024;
    HV_TRY(grow(c, &c->out_buf, &c->out_cap, 2ull * chunk * tb));
    uint8_t* bufs[2] = {(uint8_t*)c->out_buf, (uint8_t*)c->out_buf + (uint64_t)chunk * tb};
    const uint32_t n_chunks = (n + chunk - 1) / chunk;
    auto render_chunk = [&](uint32_t i) -> int {
        uint32_t first = i * chunk, cnt = n - first < chunk ? n - first : chunk;
        int b = i & 1;
        HV_CUDA(cudaStreamWaitEvent(st, c->ev_copied[b], 0));   // buffer free
        HV_TRY(launch_render(L, d_reqs + first, cnt, mode, index_kind, style, bufs[b], st, nullptr, nullptr,
                             R_units, fill, pattern_dev));
        HV_CUDA(cudaEventRecord(c->ev_rendered[b], st));
        return HV_OK;
    };
    // fresh events are complete, so the first two waits pass at once
    HV_CUDA(cudaEventRecord(c->ev_copied[0], c->copy_stream));
    HV_CUDA(cudaEventRecord(c->ev_copied[1], c->copy_stream));
    HV_TRY(render_chunk(0));
    for (uint32_t i = 0; i < n_chunks; i++) {
        if (i + 1 < n_chunks) HV_TRY(render_chunk(i + 1));
        uint32_t first = i * chunk, cnt = n - first < chunk ? n - first : chunk;
        int b = i & 1;
        HV_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_rendered[b], 0));
        HV_CUDA(cudaMemcpyAsync((uint8_t*)out + (uint64_t)first * tb, bufs[b], (uint64_t)cnt * tb,
                                cudaMemcpyDeviceToHost, c->copy_stream));
        HV_CUDA(cudaEventRecord(c->ev_copied[b], c->copy_stream));
    }
    HV_CUDA(cudaStreamSynchronize(c->copy_stream));
    HV_CUDA(cudaStreamSynchronize(st));
    return HV_OK;
}

namespace {

// Bitwise combination of two MASK results, word by word (overlay).
__global__ void k_combine(uint32_t* a, const uint32_t* b, uint64_t n, int op) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t x = a[i], y = b[i];
    a[i] = op == HV_OVERLAY_AND ? (x & y) : op == HV_OVERLAY_OR ? (x | y) : op == HV_OVERLAY_XOR ? (x ^ y) : (x & ~y);
}

}  // namespace

}  // namespace hv

extern "C" {

int hv_render_tiles(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                    const hv_style* style, void* out, uint64_t out_bytes, void* stream) {
    return render_impl(layer, reqs, n, mode, index_kind, style, out, out_bytes, stream, -1);
}

int hv_render_tiles_styled(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                           const hv_style* style, const hv_fill_style* fill, void* out, uint64_t out_bytes,
                           void* stream) {
    return render_impl(layer, reqs, n, mode, index_kind, style, out, out_bytes, stream, -1, fill);
}

int hv_render_buffer(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                     int32_t radius_units, const hv_style* style, void* out, uint64_t out_bytes, void* stream) {
    if (radius_units < 0 || radius_units > kMaxBufferRadius) {
        set_error("hv_render_buffer: radius %d outside 0..2^29 units", radius_units);
        return HV_ERANGE;
    }
    return render_impl(layer, reqs, n, mode, index_kind, style, out, out_bytes, stream, radius_units);
}

int hv_overlay_tiles(hv_layer* layer_a, int32_t radius_a, hv_layer* layer_b, int32_t radius_b, int op,
                     const hv_tile_req* reqs, uint32_t n, int index_kind, void* out, uint64_t out_bytes,
                     void* stream) {
    if (!layer_a || !layer_b) { set_error("hv_overlay_tiles: NULL layer"); return HV_EINVAL; }
    if (op < HV_OVERLAY_AND || op > HV_OVERLAY_DIFF) { set_error("hv_overlay_tiles: unknown op %d", op); return HV_EINVAL; }
    Layer* A = (Layer*)layer_a;
    Layer* B = (Layer*)layer_b;
    if (A->ctx != B->ctx) { set_error("hv_overlay_tiles: the layers belong to different contexts"); return HV_EINVAL; }
    if (n == 0) return HV_OK;
    if (!out || !is_device_ptr(out)) { set_error("hv_overlay_tiles: out must be device memory"); return HV_EINVAL; }
    const uint64_t tb = hv_tile_bytes(HV_MODE_MASK);
    if (out_bytes < (uint64_t)n * tb) { set_error("hv_overlay_tiles: out_bytes too small"); return HV_EINVAL; }
    Ctx* c = A->ctx;
    HV_CUDA(cudaSetDevice(c->device));
    std::lock_guard<std::mutex> g(c->overlay_mu);
    HV_TRY(grow(c, &c->overlay_buf, &c->overlay_cap, (uint64_t)n * tb));
    HV_TRY(hv_render_buffer(layer_a, reqs, n, HV_MODE_MASK, index_kind, radius_a, nullptr, out, out_bytes, stream));
    HV_TRY(hv_render_buffer(layer_b, reqs, n, HV_MODE_MASK, index_kind, radius_b, nullptr, c->overlay_buf,
                            (uint64_t)n * tb, stream));
    const uint64_t words = (uint64_t)n * tb / 4;
    k_combine<<<(unsigned)((words + 255) / 256), 256, 0, (cudaStream_t)stream>>>((uint32_t*)out,
                                                                                (const uint32_t*)c->overlay_buf, words, op);
    HV_CUDA(cudaGetLastError());
    // the scratch holds B's masks until the combine has read them
    HV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return HV_OK;
}

int hv_layer_keys(hv_layer* layer, int which, uint64_t* out, uint64_t n) {
    if (!layer || !out) { set_error("hv_layer_keys: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    if (!(L->indexes & HV_INDEX_RTREE)) { set_error("hv_layer_keys: index not built"); return HV_ESTATE; }
    const uint64_t* k = which == 0 ? L->keys : L->mbr_keys;
    uint64_t cnt = which == 0 ? L->n_obj : (L->kind == HV_LAYER_POLYGONS ? L->n_poly : 0);
    if (which != 0 && which != 1) { set_error("hv_layer_keys: which must be 0 or 1"); return HV_EINVAL; }
    if (n != cnt) { set_error("hv_layer_keys: n must be %llu", (unsigned long long)cnt); return HV_EINVAL; }
    if (!is_device_ptr(out)) { set_error("hv_layer_keys: out must be device memory"); return HV_EINVAL; }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    if (cnt) HV_CUDA(cudaMemcpy(out, k, cnt * 8, cudaMemcpyDeviceToDevice));
    return HV_OK;
}

int hv_learned_lookup(hv_layer* layer, int which, const uint64_t* keys, uint32_t n, uint64_t* out,
                      uint64_t* fallbacks, void* stream) {
    if (!layer || (!keys && n) || (!out && n) || !fallbacks) { set_error("hv_learned_lookup: NULL argument"); return HV_EINVAL; }
    if (which != 0 && which != 1) { set_error("hv_learned_lookup: which must be 0 or 1"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    if (n && (!is_device_ptr(keys) || !is_device_ptr(out))) { set_error("hv_learned_lookup: device arrays required"); return HV_EINVAL; }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    return learned_lookup(L, which, keys, n, out, fallbacks, (cudaStream_t)stream);
}

int hv_render_tiles_counted(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode,
                            int index_kind, const hv_style* style, void* out, uint64_t out_bytes,
                            int64_t* log, uint64_t log_cap, int64_t* log_count, void* stream) {
    if (!layer || !reqs || !out || !log || !log_count) { set_error("hv_render_tiles_counted: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    uint64_t tb = hv_tile_bytes(mode);
    if (tb == 0 || out_bytes < (uint64_t)n * tb) { set_error("hv_render_tiles_counted: bad mode or size"); return HV_EINVAL; }
    if (!(L->indexes & index_kind)) { set_error("hv_render_tiles_counted: index not built"); return HV_ESTATE; }
    if (!is_device_ptr(reqs) || !is_device_ptr(out) || !is_device_ptr(log) || !is_device_ptr(log_count)) {
        set_error("hv_render_tiles_counted: all buffers must be device memory");
        return HV_EINVAL;
    }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    RenderLog rl{log, log_cap, log_count};
    return launch_render(L, reqs, n, mode, index_kind, style, (uint8_t*)out, (cudaStream_t)stream, &rl);
}

int hv_render_tiles_phases(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                           const hv_style* style, void* out, uint64_t out_bytes, uint64_t* phases, void* stream) {
    if (!layer || !reqs || !out || !phases) { set_error("hv_render_tiles_phases: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    uint64_t tb = hv_tile_bytes(mode);
    if (tb == 0 || out_bytes < (uint64_t)n * tb) { set_error("hv_render_tiles_phases: bad mode or size"); return HV_EINVAL; }
    if (!(L->indexes & index_kind)) { set_error("hv_render_tiles_phases: index not built"); return HV_ESTATE; }
    if (!is_device_ptr(reqs) || !is_device_ptr(out) || !is_device_ptr(phases)) {
        set_error("hv_render_tiles_phases: all buffers must be device memory");
        return HV_EINVAL;
    }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    RenderLog rl{nullptr, 0, nullptr, phases};
    return launch_render(L, reqs, n, mode, index_kind, style, (uint8_t*)out, (cudaStream_t)stream, &rl);
}

int hv_layer_take_status(hv_layer* layer, void* stream, uint32_t* status) {
    if (!layer || !status) { set_error("hv_layer_take_status: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    cudaStream_t st = (cudaStream_t)stream;
    HV_CUDA(cudaSetDevice(L->ctx->device));
    uint32_t h[4] = {0, 0, 0, 0};
    HV_CUDA(cudaMemcpyAsync(h, L->status, 16, cudaMemcpyDeviceToHost, st));
    HV_CUDA(cudaMemsetAsync(L->status, 0, 16, st));
    HV_CUDA(cudaStreamSynchronize(st));
    *status = h[0];
    if (h[0] & 2u) {
        unsigned long long rec = (unsigned long long)h[2] | ((unsigned long long)h[3] << 32);
        set_error("internal check %llu failed at value %llu", rec >> 56, rec & ((1ull << 56) - 1));
    }
    return HV_OK;
}

int hv_render_launches(hv_layer* layer, int index_kind, uint32_t* launches) {
    if (!layer || !launches) { set_error("hv_render_launches: NULL argument"); return HV_EINVAL; }
    *launches = render_launch_count((Layer*)layer, index_kind);
    return HV_OK;
}

}  // extern "C"
