// Internal host-side structures of libhivision (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/hivision.h"

namespace hv {

constexpr int kFanout = 32;        // children per inner node, objects per leaf
constexpr int kMaxLevels = 16;     // inner levels of a tree (32^16 >> 2^64)
constexpr int kTile = 256;         // tile side in pixels (Sec. 4)
constexpr int32_t kMaxBufferRadius = 1 << 29;   // largest buffer radius (grid units)

void set_error(const char* fmt, ...);

// Device memory accounting against the context's budget.
struct Ctx {
    int device = 0;
    uint64_t budget = 0;     // 0 = unlimited
    uint64_t held = 0;
    std::mutex mu;
    // render scratch (request copies, host-output staging), grown on demand
    void* req_buf = nullptr;
    uint64_t req_cap = 0;
    void* out_buf = nullptr;
    uint64_t out_cap = 0;
    void* pinned_req = nullptr;   // pinned staging for host requests
    uint64_t pinned_req_cap = 0;
    cudaStream_t copy_stream = nullptr;   // device -> host copies of rendered chunks
    cudaEvent_t ev_rendered[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    std::mutex render_mu;         // serialises use of the scratch above
    void* overlay_buf = nullptr;  // the second layer's masks of an overlay
    uint64_t overlay_cap = 0;
    std::mutex overlay_mu;
};

int dev_alloc(Ctx* c, void** p, uint64_t bytes);
void dev_free(Ctx* c, void* p, uint64_t bytes);

// A segment piece: the whole segment (for the exact distance test) and a
// conservative box of the part of it the piece stands for (for pruning).
// Stored as 32-byte records: a leaf visit loads both halves at once (a
// layout with the boxes and the segments in two arrays, the segment read only
// by lanes whose box is in reach, measured slower: the dependent second load
// costs more latency than the bytes it saves).
struct __align__(16) Piece {
    int4 seg;
    int4 box;
};

// A packed R-tree over n objects sorted by Hilbert key.  Inner nodes hold 32
// child boxes as SoA int32 [minx x32][miny x32][maxx x32][maxy x32] (512 B).
// Level 1 nodes hold leaf boxes (a leaf = 32 consecutive objects), level l
// nodes hold the boxes of level l-1 nodes, the root is the single node of the
// top level.  Nodes of all levels live in one array; level l starts at
// level_off[l].
struct TreeView {
    const int32_t* nodes = nullptr;
    uint64_t level_off[kMaxLevels + 1] = {};
    uint64_t level_n[kMaxLevels + 1] = {};
    int top = 0;                 // level of the root, 0 = empty tree
    uint64_t n_obj = 0;
    int4 root_box = {0, 0, -1, -1};
};

struct Tree {
    TreeView view;
    int32_t* nodes = nullptr;
    uint64_t nodes_bytes = 0;
    uint64_t n_nodes = 0;
};

// Learned position index over the sorted Hilbert keys of a tree's objects
// (model layout in hv_learned.cuh).
struct LearnedView {
    const uint64_t* keys = nullptr;     // sorted keys, n_obj
    const uint64_t* seg_k0 = nullptr;   // first key of each piece
    const float* seg_a = nullptr;       // slope of each piece
    const float* seg_b = nullptr;       // intercept of each piece
    const float* pinv = nullptr;        // 1 / key span of each piece
    const uint32_t* eps_piece = nullptr;  // per-piece position error bound
    const uint32_t* radix = nullptr;    // top-bits table -> first piece
    const uint16_t* mlp = nullptr;      // bf16 MLP weights (NULL: linear only)
    const uint16_t* emb = nullptr;      // bf16 piece embeddings
    const uint8_t* use_mlp = nullptr;   // per piece: MLP term in use
    uint32_t n_seg = 0;
    uint32_t P = 0;                     // keys per piece
    int hidden = 0;                     // MLP width, 0 = not used
    int64_t eps = 0;                    // max position error of the model
    int64_t eps_linear = 0;             // ... of the linear pieces alone
    int64_t eps_mlp = 0;                // ... with the MLP residual
    double mean_err = 0;
    double mean_err_linear = 0;
    double mean_window = 0;             // mean per-piece bound (search window)
    double mean_window_linear = 0;
    uint32_t pieces_mlp = 0;            // pieces that use the MLP term
    int32_t halo = 0;                   // max half-extent of indexed objects
    uint64_t n_obj = 0;
    // objects whose extent exceeds `halo` are also kept in a small side
    // R-tree that every lookup searches
    TreeView outliers;
    const int4* outlier_obj = nullptr;
    const uint32_t* outlier_ids = nullptr;
    bool ready = false;
};

struct Learned {
    LearnedView view;
    std::vector<std::pair<void*, uint64_t>> allocs;
    Tree outlier_tree;
    double train_ms = 0;
    uint64_t n_outliers = 0;
};

struct Layer {
    Ctx* ctx = nullptr;
    int kind = HV_LAYER_POINTS;
    uint32_t indexes = 0;
    // objects: input order until the index is built, then the sorted index
    // records (points, or segment pieces: the full segment plus the box of a
    // bounded-extent piece of it)
    uint64_t n_src = 0;          // points, segments or polygon edges
    uint64_t n_obj = 0;          // index records (points or pieces)
    void* obj = nullptr;
    uint64_t obj_bytes = 0;
    int32_t piece_extent = 0;    // max extent of a piece (segment layers)
    uint64_t* keys = nullptr;    // sorted Hilbert keys of obj (after build)
    Tree tree;                   // R-tree over obj
    // polygons
    uint64_t n_poly = 0;
    int4* poly_edges = nullptr;      // edges in polygon order (a.x, a.y, b.x, b.y)
    uint64_t* poly_edge_off = nullptr;  // n_poly + 1
    int4* mbr_obj = nullptr;         // polygon boxes, sorted by Hilbert key
    uint32_t* mbr_ids = nullptr;     // polygon id of each sorted box
    uint64_t* mbr_keys = nullptr;
    Tree mbr_tree;
    Learned learned;                 // over obj
    Learned mbr_learned;             // over polygon boxes
    int4 mbr = {0, 0, -1, -1};
    // HV_PLACE_HOST: obj (and poly_edges) live in mapped pinned host memory
    void* obj_host = nullptr;        // host address of obj (NULL: device memory)
    void* edges_host = nullptr;      // host address of poly_edges (NULL: device memory)
    uint32_t* status = nullptr;      // sticky device status word
    double build_ms = 0;
    std::vector<std::pair<void*, uint64_t>> extra;  // other allocations
};

// index build (hv_build.cu)
int build_tree_points(Layer* L);
int build_tree_segments(Layer* L);
int make_pieces(Ctx* c, const int4* segs, uint64_t n, Piece** out, uint64_t* n_out, int32_t* extent);
int build_tree_polygons(Layer* L);
void free_tree(Ctx* c, Tree* t);
// learned index (hv_learned.cu)
int build_learned(Layer* L, const hv_build_opts* opts);
void free_learned(Ctx* c, Learned* l);
int learned_lookup(Layer* L, int which, const uint64_t* q, uint32_t n, uint64_t* out, uint64_t* fallbacks,
                   cudaStream_t st);
// render (hv_render.cu)
struct RenderLog {
    int64_t* log;
    uint64_t cap;
    int64_t* count;
    uint64_t* phases = nullptr;   // phase profile counters (instrumented launch)
};
// R_units < 0: each request's radius r16 * 2^(19 - z); else the radius of
// every tile in grid units (buffer analysis), at most kMaxBufferRadius.
int launch_render(Layer* L, const hv_tile_req* d_reqs, uint32_t n, int mode, int index_kind,
                  const hv_style* style, uint8_t* d_out, cudaStream_t stream,
                  const RenderLog* log = nullptr, const uint32_t* n_dev = nullptr, int32_t R_units = -1,
                  const hv_fill_style* fill = nullptr, const void* pattern_dev = nullptr);
// A fill style is valid: HV_FILL_AA or 0, and a pattern of at most 16 x 16
// texels with alpha 0 or 255 (or none).
bool fill_style_ok(const hv_fill_style* fill);
uint32_t render_launch_count(Layer* L, int index_kind);
// result pool (hv_pool.cu)
struct ResultPool;
bool pool_lookup(ResultPool* P, const hv_tile_req& r, const hv_style* style, std::vector<uint8_t>* out);
int pool_insert(ResultPool* P, const hv_tile_req& r, const hv_style* style, const void* data, uint64_t n);

}  // namespace hv

#define HV_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            hv::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                          __LINE__);                                                    \
            return HV_ECUDA;                                                            \
        }                                                                               \
    } while (0)

#define HV_TRY(expr)             \
    do {                         \
        int rc_ = (expr);        \
        if (rc_ != HV_OK) return rc_; \
    } while (0)
