/*
 * hivision.h -- C ABI of the GB300 display-driven tile renderer.
 *
 * A reimplementation, for one GPU, of the per-pixel spatial-index query of
 * HiVision (Ma et al., "HiVision: Rapid Visualization of Large-Scale Spatial
 * Vector Data", arXiv 2005.12489): every pixel of a requested 256 x 256 tile
 * is decided by index queries against the layer's objects instead of
 * rasterising every object (Sec. 1, Sec. 2.3 display-driven computing).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid.      Coordinates are int32 units of a 2^31 x 2^31 Web-Mercator grid,
 *            each in [-2^30, 2^30); y grows southward.  Zoom z is 0..19; at
 *            zoom z there are 2^z x 2^z tiles (Sec. 2.2) of 256 x 256 pixels
 *            (Sec. 4) and a pixel is 2^(23-z) units wide (resolution R_z of
 *            Algorithm 1).  Pixel (i, j) of tile (z, x, y) has its centre at
 *            (-2^30 + x*2^(31-z) + i*2^(23-z) + 2^(22-z), same for y, j);
 *            row j = 0 is the north edge.
 * Radius.    r16 is the style radius (points) or half-width (lines, polygon
 *            outlines) in 1/16 px, 1..1024; R = r16 * 2^(19-z) units
 *            (Algorithm 1: R = N * R_z).
 * Samples.   A sample s is covered when some object lies within distance
 *            <= R of it (closed; Algorithm 1).  COVERAGE and RGBA use the
 *            four super-samples at the pixel centre +-(2^(21-z), 2^(21-z))
 *            (Algorithm 1, P1..P4); MASK uses the pixel centre.
 * Fill.      A polygon layer also fills the pixel centres that lie inside
 *            some polygon: that polygon's own edges (all its rings) cross the
 *            ray from the centre towards +x an odd number of times, an edge
 *            (a, b) crossing when (a.y > c.y) != (b.y > c.y) and its crossing
 *            lies strictly right of c (Algorithm 2; this half-open rule
 *            stands in for the paper's IsLevel flag and segment cutting,
 *            Sec. 3.1).  Polygons are tested one by one, so two overlapping
 *            polygons both fill; rings of one polygon combine by parity.
 * Results are exact integer decisions: identical, bit for bit, to the plain
 * definition above.
 *
 * Ownership.  Input arrays are copied by the library; the caller keeps them.
 * Handles belong to the library until their *_free / hv_destroy.  Output
 * buffers belong to the caller.  Pointers documented as "host or device" are
 * classified with cudaPointerGetAttributes.  A stream argument is a
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Errors.  Every call returns an hv_status.  On failure nothing is written
 * to caller-visible outputs unless stated, and hv_last_error() returns a
 * message for the calling thread.
 */
#ifndef HIVISION_H
#define HIVISION_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hv_status {
    HV_OK = 0,
    HV_EINVAL = 1,    /* bad argument: null pointer, wrong size, bad mode, state */
    HV_ERANGE = 2,    /* coordinate outside the grid, z > 19, x or y >= 2^z,
                         r16 outside 1..1024 */
    HV_ENOMEM = 3,    /* device allocation failed or the context's budget is spent */
    HV_ECUDA = 4,     /* a CUDA runtime call failed */
    HV_ETIMEOUT = 5,  /* a bounded wait ran out */
    HV_EBUSY = 6,     /* the server's queue is full; retry later */
    HV_ESTATE = 7     /* call not valid in the object's current state */
} hv_status;

/* Output modes; bytes per tile in brackets. */
enum {
    HV_MODE_MASK = 0,     /* [8192] 1 bit per pixel: bit b of little-endian
                             uint32 word w of row j is pixel (32w + b, j).
                             Set when the centre is covered, or filled. */
    HV_MODE_COVERAGE = 1, /* [65536] 1 byte per pixel, row-major: the number
                             of covered super-samples 0..4, plus 8 when the
                             centre is filled (polygon layers). */
    HV_MODE_RGBA = 2      /* [262144] 4 bytes per pixel R, G, B, A, row-major.
                             v = covered super-samples, a = (255 v + 2) >> 2;
                             filled: rgb = (line*a + fill*(255 - a) + 127) / 255
                             per channel, A = 255; else v > 0: (line rgb, a);
                             else (0, 0, 0, 0).  Not premultiplied. */
};

enum { HV_LAYER_POINTS = 0, HV_LAYER_LINES = 1, HV_LAYER_POLYGONS = 2 };

/* Index kinds (bit flags for hv_layer_build_index; one value for rendering). */
enum { HV_INDEX_RTREE = 1, HV_INDEX_LEARNED = 2 };

typedef struct hv_ctx hv_ctx;
typedef struct hv_layer hv_layer;
typedef struct hv_server hv_server;

/* One tile request, 16 bytes. */
typedef struct hv_tile_req {
    uint32_t x, y;    /* tile column and row, < 2^z */
    uint16_t r16;     /* radius or half-width in 1/16 px, 1..1024 */
    uint8_t z;        /* zoom 0..19 */
    uint8_t mode;     /* server only: HV_MODE_*; ignored by hv_render_tiles */
    uint32_t layer;   /* server only: index into the server's layers */
} hv_tile_req;

/* Colours; the alpha bytes are reserved (alpha comes from coverage). */
typedef struct hv_style {
    uint8_t line_rgba[4];  /* points, lines, polygon outlines */
    uint8_t fill_rgba[4];  /* polygon interiors */
} hv_style;

/* Fill style of polygon layers (Sec. 3.2.2 fill styles; Sec. 4.1 Pattern
 * Library).  HV_FILL_AA decides the fill at the four super-samples, as
 * Algorithm 1 does for outlines: f = number of them inside a polygon (0..4);
 * COVERAGE then holds v | f << 4 (bits 4-6; bit 3 unused) and RGBA composes
 * the outline over the partly covered fill (below); MASK keeps the centre
 * rule.  A pattern of pattern_w x pattern_h texels (1..16 each, RGBA, row
 * major, alpha 0 or 255) is laid over the global pixel grid: pixel
 * (256 x + i, 256 y + j) of tile (z, x, y) takes texel
 * ((256 y + j) mod pattern_h, (256 x + i) mod pattern_w); a transparent
 * texel leaves the pixel unfilled, an opaque one gives the fill colour.
 * The texels go to a small stream-ordered device copy for the call
 * (cudaMallocAsync / cudaFreeAsync on `stream`).
 * RGBA with fill count f and outline count v: a = (255 v + 2) >> 2,
 * a_f = (255 f + 2) >> 2, A = (255 a + a_f (255 - a) + 127) / 255, each
 * channel (line a 255 + fill a_f (255 - a) + 127 A) / (255 A); for f = 4 this
 * is the HV_MODE_RGBA formula above, for f = 0 the unfilled one. */
enum { HV_FILL_AA = 1 };
typedef struct hv_fill_style {
    uint32_t flags;              /* HV_FILL_AA or 0 */
    uint32_t pattern_w, pattern_h;  /* 0, 0: no pattern */
    const uint8_t* pattern_rgba; /* host memory, pattern_w * pattern_h * 4 bytes
                                    (copied at the call) */
} hv_fill_style;

/* hv_build_opts.learned_hidden value: train no MLP residual. */
#define HV_LEARNED_NO_MLP 0xFFFFFFFFu

typedef struct hv_build_opts {
    uint32_t learned_segments;   /* piecewise-linear pieces (0 = one piece per
                                    512 sorted keys) */
    uint32_t learned_hidden;     /* 0: pieces with the residual MLP 5 -> 16 ->
                                    16 -> 1 (kept where it narrows a piece's
                                    bound); HV_LEARNED_NO_MLP: linear pieces
                                    only; other values are reserved */
    uint32_t learned_steps;      /* training steps (0 = default 300) */
    uint32_t learned_seed;       /* initialisation seed */
    uint32_t max_error;          /* accept the learned index only if its
                                    position error bound is <= this (0 = 4096) */
    uint32_t object_placement;   /* HV_PLACE_DEVICE (0) or HV_PLACE_HOST */
    uint32_t reserved[2];
} hv_build_opts;

/* hv_build_opts.object_placement.  HV_PLACE_HOST keeps the layer's index
 * records (points, segment pieces; for polygon layers also the edges in
 * polygon order) in pinned host memory after the build, mapped into the
 * device's address space: the kernels read them over the CPU-GPU link
 * (NVLink-C2C on GB300) while the tree nodes, keys and learned model stay in
 * device memory.  For layers whose records do not fit the device (the
 * paper's layers are read from memory-mapped index files, Sec. 4).  A layer
 * file loaded back holds its records in device memory again. */
enum { HV_PLACE_DEVICE = 0, HV_PLACE_HOST = 1 };

typedef struct hv_layer_info {
    uint32_t kind;               /* HV_LAYER_* */
    uint32_t indexes;            /* HV_INDEX_* bits built */
    uint64_t n_objects;          /* points, segments or polygon edges */
    uint64_t n_polygons;         /* polygon layers: polygons */
    int32_t mbr[4];              /* minx, miny, maxx, maxy of the layer (empty: 0) */
    uint32_t tree_levels;        /* inner levels of the object R-tree */
    uint64_t tree_nodes;         /* inner nodes of the object R-tree */
    uint64_t device_bytes;       /* device memory held by the layer */
    int64_t learned_error;       /* learned index: max |predicted - true| position
                                    (-1: not built) */
    uint64_t learned_outliers;   /* learned index: records kept in side trees (objects and polygon boxes) */
    double build_ms;             /* last index build, device time */
    double train_ms;             /* learned-index training, device time */
    int64_t learned_error_linear;  /* error bound of the linear pieces alone */
    int64_t learned_error_mlp;     /* error bound with the MLP residual */
    double learned_mean_error;     /* mean |predicted - true| position */
    uint32_t learned_pieces;       /* piecewise-linear pieces */
    uint32_t learned_mlp;          /* pieces that add the MLP residual (a piece
                                      uses it only where it narrows its bound) */
    int32_t learned_halo;          /* half-extent covered through centre keys */
    int32_t piece_extent;          /* segment layers: segments are indexed as
                                      pieces of at most this extent */
    uint64_t index_records;        /* records in the object R-tree (points, or
                                      segment pieces) */
    double learned_mean_window;    /* mean per-piece error bound (search window) */
    double learned_mean_window_linear;  /* ... of the linear pieces alone */
    uint64_t host_bytes;           /* pinned host memory held by the layer
                                      (HV_PLACE_HOST) */
} hv_layer_info;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  mem_budget caps the device bytes
 * the context may hold (layers, indexes, scratch); 0 = no cap. */
int hv_create(hv_ctx** out, int device, uint64_t mem_budget);
int hv_destroy(hv_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none). */
const char* hv_last_error(void);
/* Bytes currently held by the context on its device. */
int hv_ctx_device_bytes(hv_ctx* ctx, uint64_t* out);

/* ---- quantisation (host only) ------------------------------------------- */

/* Longitude / latitude in degrees (WGS 84, interleaved lon, lat; n pairs,
 * host memory) -> grid coordinates (interleaved x, y; host memory): the
 * spherical Web-Mercator projection the tile pyramid is defined in (Sec. 3.2,
 * resolution(Z) in Web-Mercator metres), u = (lon + 180) / 360 and
 * v = 1/2 - asinh(tan lat) / (2 pi) (v = 0 at the north edge), each scaled
 * by 2^31, floored and shifted by -2^30; the east and south edges (u or
 * v = 1) fall into the last grid unit.  lon outside [-180, 180] or |lat| above
 * atan(sinh pi) = 85.0511287798... degrees (+1e-9, for the rounding of a
 * caller's own copy; not a number counts as outside) -> HV_ERANGE,
 * nothing written.  Floating point: outside the exact contract of the
 * rendering, which starts from the grid integers. */
int hv_lonlat_to_grid(const double* lonlat, uint64_t n, int32_t* xy);

/* Tile router for replicas on several GPUs (every GPU holds the layers; a
 * tile goes to one of them): rank_out[i] = the rank in 0..n_ranks-1 of request
 * i, a hash of its (layer, z, x, y) -- the same tile always goes to the same
 * rank, whatever its radius or mode, and tiles spread evenly.  Host only. */
int hv_route_tiles(const hv_tile_req* reqs, uint64_t n, uint32_t n_ranks, uint32_t* rank_out);

/* ---- layers (Sec. 3.1 data organisation; Sec. 4.1 Register Vector Data) -- */

/* Points: xy holds n interleaved (x, y) pairs, host or device memory. */
int hv_layer_load_points(hv_ctx* ctx, const int32_t* xy, uint64_t n, hv_layer** out);

/* Linestrings, split into their segments (Sec. 3.1: segments, not whole
 * objects, are the index records).  xy: n_vert interleaved (x, y) pairs (host
 * or device); line_off: n_lines + 1 non-decreasing offsets (host), line l =
 * vertices [line_off[l], line_off[l+1]), line_off[n_lines] == n_vert.  A line
 * with fewer than two vertices draws nothing. */
int hv_layer_load_linestrings(hv_ctx* ctx, const int32_t* xy, uint64_t n_vert,
                              const uint64_t* line_off, uint64_t n_lines, hv_layer** out);

/* Polygons (Sec. 3.1, the multi-level index of edges and polygon MBRs).
 * Ring r = vertices [ring_off[r], ring_off[r+1]) and closes implicitly (its
 * last vertex joins its first); polygon p = rings
 * [poly_ring_off[p], poly_ring_off[p+1]), outer ring and holes alike.
 * Offsets are host arrays, non-decreasing, ending at n_vert and n_rings. */
int hv_layer_load_polygons(hv_ctx* ctx, const int32_t* xy, uint64_t n_vert,
                           const uint64_t* ring_off, uint64_t n_rings,
                           const uint64_t* poly_ring_off, uint64_t n_polys, hv_layer** out);

/* Build the indexes named by `kinds` (HV_INDEX_RTREE is always built).
 * R-tree: objects sorted by the Hilbert key of their box centre, packed 32 to
 * a leaf, inner nodes of 32 child boxes (replaces the paper's Boost R-trees,
 * Sec. 3.1, Sec. 5).  Learned: a piecewise-linear + MLP model of position vs
 * Hilbert key with a measured error bound, confirmed by exact search, with
 * the R-tree as its fallback.  opts may be NULL.  Synchronous. */
int hv_layer_build_index(hv_layer* layer, uint32_t kinds, const hv_build_opts* opts);

int hv_layer_info_get(hv_layer* layer, hv_layer_info* out);

/* Copy the sorted Hilbert keys of a built layer (which = 0: index records,
 * 1: polygon boxes) into `out` (device memory, n entries, n = index_records /
 * polygons of hv_layer_info). */
int hv_layer_keys(hv_layer* layer, int which, uint64_t* out, uint64_t n);

/* lower_bound of each query key in the sorted keys through the learned model
 * (which = 0: objects, 1: polygon boxes): keys and out are device arrays of n
 * entries; *fallbacks receives how many lookups left the model's error window
 * and were answered by a full binary search.  Synchronises `stream`. */
int hv_learned_lookup(hv_layer* layer, int which, const uint64_t* keys, uint32_t n, uint64_t* out,
                      uint64_t* fallbacks, void* stream);
int hv_layer_free(hv_layer* layer);

/* Write / read a built layer (objects, R-tree, learned model) to / from a
 * binary file with a version header (the paper keeps its indexes as files,
 * Sec. 4).  Loading restores the device arrays without rebuilding. */
int hv_layer_save(hv_layer* layer, const char* path);
int hv_layer_load_file(hv_ctx* ctx, const char* path, hv_layer** out);

/* ---- rendering (Algorithm 1 SIBV, Algorithm 2 SIBF, Sec. 4.1 Render Tiles) */

/* Bytes of one tile in `mode` (0 for an unknown mode). */
uint64_t hv_tile_bytes(int mode);

/* Render n tiles of `layer` into `out` (n * hv_tile_bytes(mode) bytes, tile k
 * at offset k * hv_tile_bytes(mode)), using index `index_kind`.
 *
 * reqs: host or device.  Host requests are checked first (HV_ERANGE, nothing
 *   written).  Device requests are checked by the kernel: an invalid request
 *   yields an all-zero tile and sets a sticky flag read by
 *   hv_layer_take_status().
 * out: host or device.  When reqs and out are both device memory the call is
 *   asynchronous on `stream`.  Otherwise requests are staged, tiles for
 *   pinned (page-locked) host memory are written by the kernels straight into
 *   it over the CPU-GPU link, tiles for other host memory are rendered into
 *   device scratch and copied back, and the call returns after the stream has
 *   synchronised.
 * style: colours for HV_MODE_RGBA (may be NULL otherwise).
 * Tiles that the layer cannot reach are written as zeros without index work
 * (Sec. 4.1, Parse Tasks). */
int hv_render_tiles(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode,
                    int index_kind, const hv_style* style, void* out, uint64_t out_bytes,
                    void* stream);

/* ---- display-driven buffer and overlay analysis (HiBuffer, HiBO; Sec. 2.3,
 *      Sec. 3.2: the widths of Algorithm 1 as a buffer distance) ---------- */

/* hv_render_tiles with the distance given on the ground instead of in
 * pixels: every tile decides its samples against R = radius_units grid units
 * (0..2^29, else HV_ERANGE), whatever its zoom, so the result is the buffer of
 * the layer's objects at that distance (a polygon layer's buffer also holds
 * its interiors) as seen in the tile.  The requests' r16 fields are ignored;
 * everything else is as in hv_render_tiles. */
int hv_render_buffer(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                     int32_t radius_units, const hv_style* style, void* out, uint64_t out_bytes, void* stream);

/* Overlay operations on two buffers A and B, per pixel centre. */
enum { HV_OVERLAY_AND = 0, HV_OVERLAY_OR = 1, HV_OVERLAY_XOR = 2, HV_OVERLAY_DIFF = 3 /* A and not B */ };

/* Overlay of two buffers (HiBO): the MASK tiles of layer_a's buffer at
 * radius_a and of layer_b's at radius_b (grid units, as hv_render_buffer),
 * combined bit by bit with `op`.  The layers belong to one context; `out` is
 * device memory of n * hv_tile_bytes(HV_MODE_MASK) bytes; reqs host or
 * device.  The second buffer is rendered into scratch of the context, and
 * the call returns after `stream` has synchronised. */
int hv_overlay_tiles(hv_layer* layer_a, int32_t radius_a, hv_layer* layer_b, int32_t radius_b, int op,
                     const hv_tile_req* reqs, uint32_t n, int index_kind, void* out, uint64_t out_bytes,
                     void* stream);

/* hv_render_tiles with a fill style for polygon layers (NULL fill: as
 * hv_render_tiles; other layer kinds ignore it).  A pattern larger than
 * 16 x 16 or with a texel alpha other than 0 and 255 -> HV_EINVAL. */
int hv_render_tiles_styled(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                           const hv_style* style, const hv_fill_style* fill, void* out, uint64_t out_bytes,
                           void* stream);

/* Read and clear the layer's sticky device status (bit 0: an invalid device
 * request was seen; bit 1: an internal bounds check in the render kernel
 * failed and an access was skipped -- hv_last_error() then names the check and
 * the offending value).  Synchronises `stream`. */
int hv_layer_take_status(hv_layer* layer, void* stream, uint32_t* status);

/* Instrumented hv_render_tiles for measurement (not for production use):
 * the same tiles, plus a log of every index read.  All buffers are device
 * memory.  Each inner-node, leaf or polygon read appends one int64
 *   (tile << 38) | (kind << 35) | id
 * with kind 0 = inner node (id = node number across levels, 512 B read),
 * 1 = leaf (id = leaf number, 32 objects read), 2 / 3 = node / leaf of the
 * polygon-box tree, 4 = a polygon whose edges were scanned (id = polygon).
 * *log_count receives the number of reads (entries past log_cap are dropped).
 * Used to count the unique bytes the early-exit traversal must read. */
int hv_render_tiles_counted(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode,
                            int index_kind, const hv_style* style, void* out, uint64_t out_bytes,
                            int64_t* log, uint64_t log_cap, int64_t* log_count, void* stream);

/* Phase profile counters of hv_render_tiles_phases (indices into its array;
 * a polygon layer profiles its fill launch in the first set and its outline
 * launch in a second set at HV_PHASE_COUNT + i). */
enum {
    HV_PHASE_TOTAL = 0,       /* warp-cycles of the launch (CTA lifetimes x warps) */
    HV_PHASE_PROLOGUE,        /* request decode, result init (fill: outline decode) */
    HV_PHASE_CULL,            /* tile cull of the strip: R-tree or learned lookup */
    HV_PHASE_BIN,             /* binning the frontier by block column */
    HV_PHASE_BLOCKS_CTA,      /* the pixel-block phase, CTA time x warps */
    HV_PHASE_BLOCKS_WARP,     /* ... of which warps were busy (rest: waiting) */
    HV_PHASE_LEAF,            /* ... of which in leaf visits (exact predicates) */
    HV_PHASE_DESCEND,         /* ... of which below the frontier: node tests and
                                 leaf visits (the rest of the busy time is the
                                 blocks' scans of the frontier) */
    HV_PHASE_ENCODE,          /* output encode */
    HV_PHASE_CTAS,            /* counts: CTAs, */
    HV_PHASE_BLOCK_COUNT,     /*   8 x 4 pixel blocks, */
    HV_PHASE_LEAF_VISITS,     /*   leaf visits, */
    HV_PHASE_NODE_VISITS,     /*   inner-node visits in descents, */
    HV_PHASE_FRONTIER_TESTS,  /*   frontier entries tested by blocks, */
    HV_PHASE_LEAF_EMPTY,      /*   leaf visits with no record in reach of an
                                   undecided sample, */
    HV_PHASE_LEAF_DECIDED,    /*   leaf visits that decided a sample */
    HV_PHASE_COUNT = 16
};

/* Instrumented hv_render_tiles for measurement (not for production use):
 * the same tiles, rendered by an instrumented copy of the kernel that times
 * its phases with the SM clock and adds the warp-cycles of each phase (and a
 * few counts) to `phases` (device memory, HV_PHASE_COUNT entries, or 2 x
 * HV_PHASE_COUNT for polygon layers; the caller zeroes them).  All buffers are
 * device memory.  The instrumented copy always renders full-width strips
 * (no column parts for small batches).  Used to find where the render
 * kernel's time goes. */
int hv_render_tiles_phases(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode,
                           int index_kind, const hv_style* style, void* out, uint64_t out_bytes,
                           uint64_t* phases, void* stream);

/* Number of kernels hv_render_tiles launches per call (for launch accounting):
 * 1 for point and linestring layers, 2 for polygon layers (fill, then
 * outline); a call with host buffers launches that many per chunk of tiles. */
int hv_render_launches(hv_layer* layer, int index_kind, uint32_t* launches);

/* ---- result pool (Sec. 4.2 IMMF Result Pool; Sec. 4.1 Parse Tasks) ------ */

/* A key-value store of rendered tiles in host memory: key (layer, z, x, y,
 * r16, mode of an hv_tile_req, and the style's colours for HV_MODE_RGBA),
 * value the tile's bytes.  Bounded by a byte capacity (the least recently
 * used entries are evicted to make room) and an optional time to live
 * (entries older than it are dropped when met).  Thread-safe.  The server
 * consults it when a request is submitted (a hit completes the request
 * without GPU work, as Parse Tasks drops already rendered tiles) and stores
 * every tile it renders; measurement runs leave it off. */
typedef struct hv_result_pool hv_result_pool;

typedef struct hv_pool_stats {
    uint64_t hits;          /* lookups answered from the pool */
    uint64_t misses;        /* lookups not answered (absent or expired) */
    uint64_t inserts;       /* tiles stored */
    uint64_t evictions;     /* entries dropped to make room (least recently used first) */
    uint64_t expirations;   /* entries dropped because they outlived the time to live */
    uint64_t rejected;      /* tiles larger than the whole capacity (not stored) */
    uint64_t entries;       /* entries held now */
    uint64_t bytes;         /* tile bytes held now */
    uint64_t capacity;      /* the byte capacity */
} hv_pool_stats;

/* capacity_bytes > 0; ttl_ms = 0: entries never expire. */
int hv_result_pool_create(uint64_t capacity_bytes, uint32_t ttl_ms, hv_result_pool** out);
int hv_result_pool_destroy(hv_result_pool* pool);
/* Store a copy of `bytes` bytes of host memory `data` as the tile of `req`
 * (its layer, z, x, y, r16 and mode fields) in `style` (may be NULL; used
 * for HV_MODE_RGBA only); replaces an entry of the same key.  HV_ENOMEM if
 * the tile alone exceeds the capacity. */
int hv_result_pool_put(hv_result_pool* pool, const hv_tile_req* req, const hv_style* style,
                       const void* data, uint64_t bytes);
/* Look a tile up: on a hit copy it to `out` (host memory, out_bytes at least
 * the tile's size) and set *hit = 1, else *hit = 0. */
int hv_result_pool_get(hv_result_pool* pool, const hv_tile_req* req, const hv_style* style, void* out,
                       uint64_t out_bytes, uint32_t* hit);
int hv_result_pool_stats(hv_result_pool* pool, hv_pool_stats* out);
/* Drop every entry (the counters are kept). */
int hv_result_pool_clear(hv_result_pool* pool);

/* ---- serving (Sec. 4: MTVS task pool, IMMF, HPVE as one GPU loop) ------ */

/* A native worker thread keeps the layers resident and serves tile requests
 * of mixed layer, zoom, radius and mode as they arrive: requests wait in a
 * FIFO queue (Sec. 4.2 Task Pool); whenever one of the server's slots is free
 * the worker batches the oldest request's (layer, mode) group, admitting
 * requests while the slot's output memory and max_batch allow, and launches
 * the batch on the slot's own stream (captured CUDA graphs per slot and
 * group when use_graphs is set: one for a single request on an otherwise
 * idle device and one for batches of up to 8 tiles, whose grids split each
 * tile into short strips, and for the single request into column parts
 * too, for latency; one for larger batches).  Batches in different slots
 * overlap on the device.  Completed tiles are handed out by hv_server_poll (Sec. 4.2 Result
 * Pool, without expiry). */
typedef struct hv_server_opts {
    uint32_t max_batch;        /* tiles per batch (0 = 64, at most 4096) */
    uint32_t queue_capacity;   /* queued requests before HV_EBUSY (0 = 65536) */
    uint64_t scratch_bytes;    /* device (and pinned host) bytes for slots: each
                                  slot holds max_batch RGBA tiles; the number of
                                  slots is scratch_bytes / slot size, 1..64
                                  (0 = 1 GiB) */
    uint32_t index_kind;       /* HV_INDEX_LEARNED to use learned indexes where
                                  built; else the R-tree */
    uint32_t use_graphs;       /* launch batches as captured CUDA graphs */
    hv_style style;
    hv_result_pool* pool;      /* NULL: no result pool; else consulted at
                                  submission and filled with every rendered
                                  tile (the pool must outlive the server) */
} hv_server_opts;

typedef struct hv_done {
    uint64_t tag;              /* the tag given to hv_server_submit */
    int32_t status;            /* HV_OK or an error code */
    uint32_t bytes;            /* tile bytes at `data` */
    const uint8_t* data;       /* pinned host memory, valid until the next poll */
    double t_submit_us, t_start_us, t_done_us;  /* steady host clock, microseconds */
} hv_done;

/* Start a server over n_layers built layers of `ctx`; a request's `layer`
 * field indexes this array and its `mode` field selects the output. */
int hv_server_start(hv_ctx* ctx, hv_layer* const* layers, uint32_t n_layers,
                    const hv_server_opts* opts, hv_server** out);
/* Queue one request (checked as in hv_render_tiles): HV_EBUSY when the queue
 * is full, HV_ESTATE once the server is stopping.  Thread-safe. */
int hv_server_submit(hv_server* srv, const hv_tile_req* req, uint64_t tag);
/* Hand out up to `max` completed requests; the data of the previous poll's
 * results is released by this call. */
int hv_server_poll(hv_server* srv, hv_done* out, uint32_t max, uint32_t* n_out);
/* Finish queued and in-flight work, drop unpolled results and free the server
 * (HV_ETIMEOUT if batches are still in flight after 120 s). */
int hv_server_stop(hv_server* srv);
/* Open-loop load: submit reqs[i] at arrival_us[i] microseconds after the call
 * (as the queue allows), poll until all complete, and write each request's
 * latency (completion - scheduled arrival, microseconds) to latency_us[i] and
 * the total time to *wall_us.  Meant for measurement; do not poll
 * concurrently. */
int hv_server_replay(hv_server* srv, const hv_tile_req* reqs, const double* arrival_us, uint64_t n,
                     double* latency_us, double* wall_us);
/* hv_server_replay that also writes each request's latency in parts
 * (microseconds): parts_us[4i .. 4i+3] = wait before submission (queue
 * full), wait in the task pool (submission -> its batch is launched),
 * service (launch -> the worker sees the batch complete: copies and
 * kernels), hand-out (completion -> the replay's poll).  The first three sum
 * to latency_us[i] up to clock reads. */
int hv_server_replay_detail(hv_server* srv, const hv_tile_req* reqs, const double* arrival_us, uint64_t n,
                            double* latency_us, double* parts_us, double* wall_us);
/* Counters: batches launched, tiles launched, graph launches, slots. */
int hv_server_stats(hv_server* srv, uint64_t* batches, uint64_t* tiles, uint64_t* graph_launches,
                    uint32_t* slots);
/* Requests completed at submission without GPU work (Sec. 4.1 Parse Tasks):
 * answered by the result pool, and tiles that the layer cannot reach (its
 * objects' box, widened by the request's radius, misses the tile), which
 * are all zero. */
int hv_server_shortcuts(hv_server* srv, uint64_t* pool_hits, uint64_t* empty_tiles);

/* ---- rendering without allocation (no counterpart in the paper) --------- */

/* hv_render_tiles for callers that cannot allocate device memory: hosts whose
 * device memory is owned by another allocator or memory pool (a cudaMalloc of
 * their own would fail, or fragment the pool), and latency-critical paths that
 * cannot take the device-wide synchronisation that cudaMalloc / cudaFree may
 * imply.  It calls no allocator and takes at most 4096 tiles per call.
 * Requests in device memory are read where they are.  Requests in host
 * memory are staged in a fixed 64 KiB device array inside the library (4096
 * requests), which every device that loads the library holds until the
 * process exits.  `out` must be device
 * memory of n * hv_tile_bytes(mode) bytes, 16-byte aligned; the call is
 * asynchronous on `stream`.
 * Set-up: the first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and keeps it; make that
 * first call before any stream capture.  The address belongs to the device's
 * primary context: after a device reset the library's handles and this
 * address are all invalid.
 * Sharing: all calls with host requests use the one array, which keeps the
 * last call's requests; such calls whose work overlaps on the GPU (other
 * streams, other threads) race on it, so order them on one stream or
 * synchronise between them.
 * More than 4096 tiles -> HV_EINVAL; other errors as hv_render_tiles. */
int hv_render_tiles_static(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode,
                           int index_kind, const hv_style* style, void* out, uint64_t out_bytes,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HIVISION_H */
