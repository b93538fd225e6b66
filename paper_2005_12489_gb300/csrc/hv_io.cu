// Layer files: a built layer (sorted objects, keys, R-trees, learned models)
// written to and restored from a binary file, so a layer is indexed once and
// reloaded without rebuilding (HiVision keeps its indexes as files, Sec. 4).
//
// Format (native little-endian): a header, then records {u32 tag, u32 0,
// u64 bytes, payload}, ending with tag kEnd.  Device arrays are streamed
// through a pinned staging buffer.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "hv_device.cuh"
#include "hv_internal.h"
#include "hv_learned.cuh"

namespace hv {

namespace {

constexpr char kMagic[8] = {'H', 'V', 'L', 'A', 'Y', 'E', 'R', '\0'};
constexpr uint32_t kVersion = 3;
constexpr uint64_t kStage = 64ull << 20;

enum Tag : uint32_t {
    kEnd = 0, kObj, kKeys, kTree, kTreeNodes, kPolyEdges, kPolyEdgeOff, kMbrObj, kMbrIds, kMbrKeys,
    kMbrTree, kMbrTreeNodes, kLearned0 = 100, kLearned1 = 200
};
// learned sub-tags (added to kLearned0 / kLearned1)
enum LTag : uint32_t {
    kLScalars = 1, kLKb, kLPa, kLPc, kLPinv, kLEps, kLRadix, kLMlp, kLEmb, kLSideTree, kLSideNodes, kLSideObj,
    kLSideIds, kLUse
};

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t kind;
    uint32_t indexes;
    int32_t piece_extent;
    uint64_t n_obj;
    uint64_t n_poly;
    int4 mbr;
    uint64_t n_src;
};

struct LScalars {
    uint32_t n_seg, P;
    int32_t hidden, halo;
    int64_t eps, eps_linear, eps_mlp;
    double mean_err, train_ms;
    uint64_t n_obj, n_outliers;
    double mean_err_linear, mean_window, mean_window_linear;
    uint32_t pieces_mlp, reserved;
};

struct Writer {
    FILE* f;
    void* stage = nullptr;
    bool ok = true;
    int put(uint32_t tag, const void* p, uint64_t bytes, bool device) {
        uint32_t h[2] = {tag, 0};
        ok = ok && fwrite(h, 4, 2, f) == 2 && fwrite(&bytes, 8, 1, f) == 1;
        for (uint64_t o = 0; ok && o < bytes; o += kStage) {
            uint64_t b = bytes - o < kStage ? bytes - o : kStage;
            const void* src = (const uint8_t*)p + o;
            if (device) {
                if (cudaMemcpy(stage, src, b, cudaMemcpyDefault) != cudaSuccess) { ok = false; break; }
                src = stage;
            }
            ok = fwrite(src, 1, b, f) == b;
        }
        if (!ok) { set_error("layer file write failed"); return HV_EINVAL; }
        return HV_OK;
    }
};

int put_tree(Writer& w, uint32_t tag_view, uint32_t tag_nodes, const Tree& t) {
    TreeView v = t.view;
    v.nodes = nullptr;
    HV_TRY(w.put(tag_view, &v, sizeof(v), false));
    return w.put(tag_nodes, t.nodes, t.nodes_bytes, true);
}

int put_learned(Writer& w, uint32_t base, const Learned& l) {
    const LearnedView& v = l.view;
    if (!v.ready) return HV_OK;
    LScalars s{v.n_seg, v.P, v.hidden, v.halo, v.eps, v.eps_linear, v.eps_mlp, v.mean_err, l.train_ms,
               v.n_obj, l.n_outliers, v.mean_err_linear, v.mean_window, v.mean_window_linear, v.pieces_mlp, 0};
    HV_TRY(w.put(base + kLScalars, &s, sizeof(s), false));
    if (v.n_obj == 0) return HV_OK;
    HV_TRY(w.put(base + kLKb, v.seg_k0, (uint64_t)v.n_seg * 8, true));
    HV_TRY(w.put(base + kLPa, v.seg_a, (uint64_t)v.n_seg * 4, true));
    HV_TRY(w.put(base + kLPc, v.seg_b, (uint64_t)v.n_seg * 4, true));
    HV_TRY(w.put(base + kLPinv, v.pinv, (uint64_t)v.n_seg * 4, true));
    HV_TRY(w.put(base + kLEps, v.eps_piece, (uint64_t)v.n_seg * 4, true));
    HV_TRY(w.put(base + kLRadix, v.radix, ((1u << kRadixBits) + 2) * 4, true));
    HV_TRY(w.put(base + kLUse, v.use_mlp, v.n_seg, true));
    if (v.hidden) {
        HV_TRY(w.put(base + kLMlp, v.mlp, kLearnNW * 2, true));
        HV_TRY(w.put(base + kLEmb, v.emb, (uint64_t)v.n_seg * 8, true));
    }
    if (l.n_outliers) {
        HV_TRY(put_tree(w, base + kLSideTree, base + kLSideNodes, l.outlier_tree));
        HV_TRY(w.put(base + kLSideObj, v.outlier_obj, l.n_outliers * 16, true));
        HV_TRY(w.put(base + kLSideIds, v.outlier_ids, l.n_outliers * 4, true));
    }
    return HV_OK;
}

struct Reader {
    FILE* f;
    Ctx* c;
    void* stage = nullptr;
    uint32_t tag = 0;
    uint64_t bytes = 0;
    bool next() {
        uint32_t h[2];
        if (fread(h, 4, 2, f) != 2 || fread(&bytes, 8, 1, f) != 1) return false;
        tag = h[0];
        return true;
    }
    int host(void* dst, uint64_t expect) {
        if (bytes != expect) { set_error("layer file: record %u has %llu bytes, expected %llu", tag,
                                         (unsigned long long)bytes, (unsigned long long)expect); return HV_EINVAL; }
        if (fread(dst, 1, bytes, f) != bytes) { set_error("layer file truncated"); return HV_EINVAL; }
        return HV_OK;
    }
    // allocate device memory for the record and fill it
    int device(void** dst, std::vector<std::pair<void*, uint64_t>>* track) {
        HV_TRY(dev_alloc(c, dst, bytes));
        if (track) track->push_back({*dst, bytes ? bytes : 16});
        for (uint64_t o = 0; o < bytes; o += kStage) {
            uint64_t b = bytes - o < kStage ? bytes - o : kStage;
            if (fread(stage, 1, b, f) != b) { set_error("layer file truncated"); return HV_EINVAL; }
            HV_CUDA(cudaMemcpy((uint8_t*)*dst + o, stage, b, cudaMemcpyHostToDevice));
        }
        return HV_OK;
    }
};

}  // namespace

// defined in hv_api.cu
void free_layer_public(Layer* L);

}  // namespace hv

using namespace hv;

extern "C" {

int hv_layer_save(hv_layer* layer, const char* path) {
    if (!layer || !path) { set_error("hv_layer_save: NULL argument"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    if (!(L->indexes & HV_INDEX_RTREE)) { set_error("hv_layer_save: build the index first"); return HV_ESTATE; }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    HV_CUDA(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) { set_error("hv_layer_save: cannot open %s", path); return HV_EINVAL; }
    Writer w{f};
    if (cudaMallocHost(&w.stage, kStage) != cudaSuccess) { fclose(f); set_error("hv_layer_save: pinned staging failed"); return HV_ECUDA; }
    Header h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.kind = L->kind;
    h.indexes = L->indexes;
    h.n_obj = L->n_obj;
    h.n_poly = L->n_poly;
    h.mbr = L->mbr;
    h.n_src = L->n_src;
    h.piece_extent = L->piece_extent;
    int rc = fwrite(&h, sizeof(h), 1, f) == 1 ? HV_OK : HV_EINVAL;
    if (rc == HV_OK && L->n_obj) rc = w.put(kObj, L->obj, L->obj_bytes, true);
    if (rc == HV_OK && L->n_obj) rc = w.put(kKeys, L->keys, L->n_obj * 8, true);
    if (rc == HV_OK) rc = put_tree(w, kTree, kTreeNodes, L->tree);
    if (rc == HV_OK && L->kind == HV_LAYER_POLYGONS) {
        if (L->n_src) rc = w.put(kPolyEdges, L->poly_edges, L->n_src * 16, true);
        if (rc == HV_OK) rc = w.put(kPolyEdgeOff, L->poly_edge_off, (L->n_poly + 1) * 8, true);
        if (rc == HV_OK && L->n_poly) rc = w.put(kMbrObj, L->mbr_obj, L->n_poly * 16, true);
        if (rc == HV_OK && L->n_poly) rc = w.put(kMbrIds, L->mbr_ids, L->n_poly * 4, true);
        if (rc == HV_OK && L->n_poly) rc = w.put(kMbrKeys, L->mbr_keys, L->n_poly * 8, true);
        if (rc == HV_OK) rc = put_tree(w, kMbrTree, kMbrTreeNodes, L->mbr_tree);
    }
    if (rc == HV_OK && (L->indexes & HV_INDEX_LEARNED)) {
        rc = put_learned(w, kLearned0, L->learned);
        if (rc == HV_OK && L->kind == HV_LAYER_POLYGONS) rc = put_learned(w, kLearned1, L->mbr_learned);
    }
    if (rc == HV_OK) rc = w.put(kEnd, nullptr, 0, false);
    cudaFreeHost(w.stage);
    if (fclose(f) != 0 && rc == HV_OK) { set_error("hv_layer_save: close failed"); rc = HV_EINVAL; }
    return rc;
}

int hv_layer_load_file(hv_ctx* ctx, const char* path, hv_layer** out) {
    if (!ctx || !path || !out) { set_error("hv_layer_load_file: NULL argument"); return HV_EINVAL; }
    *out = nullptr;
    Ctx* c = (Ctx*)ctx;
    HV_CUDA(cudaSetDevice(c->device));
    FILE* f = fopen(path, "rb");
    if (!f) { set_error("hv_layer_load_file: cannot open %s", path); return HV_EINVAL; }
    Header h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion ||
        h.kind > HV_LAYER_POLYGONS) {
        fclose(f);
        set_error("hv_layer_load_file: %s is not a version-%u layer file", path, kVersion);
        return HV_EINVAL;
    }
    Layer* L = new Layer();
    L->ctx = c;
    L->kind = (int)h.kind;
    L->n_obj = h.n_obj;
    L->n_poly = h.n_poly;
    L->mbr = h.mbr;
    L->n_src = h.n_src;
    L->piece_extent = h.piece_extent;
    Reader r{f, c};
    int rc = cudaMallocHost(&r.stage, kStage) == cudaSuccess ? HV_OK : HV_ECUDA;
    LScalars ls[2];
    memset(ls, 0, sizeof(ls));
    while (rc == HV_OK) {
        if (!r.next()) { set_error("hv_layer_load_file: truncated"); rc = HV_EINVAL; break; }
        if (r.tag == kEnd) break;
        void* d = nullptr;
        switch (r.tag) {
            case kObj: rc = r.device(&L->obj, nullptr); L->obj_bytes = r.bytes; break;
            case kKeys: rc = r.device((void**)&L->keys, nullptr); break;
            case kTree: rc = r.host(&L->tree.view, sizeof(TreeView)); break;
            case kTreeNodes:
                rc = r.device((void**)&L->tree.nodes, nullptr);
                L->tree.nodes_bytes = r.bytes;
                L->tree.n_nodes = r.bytes / 512;
                L->tree.view.nodes = L->tree.nodes;
                break;
            case kPolyEdges: rc = r.device((void**)&L->poly_edges, nullptr); break;
            case kPolyEdgeOff: rc = r.device((void**)&L->poly_edge_off, nullptr); break;
            case kMbrObj: rc = r.device((void**)&L->mbr_obj, nullptr); break;
            case kMbrIds: rc = r.device((void**)&L->mbr_ids, nullptr); break;
            case kMbrKeys: rc = r.device((void**)&L->mbr_keys, nullptr); break;
            case kMbrTree: rc = r.host(&L->mbr_tree.view, sizeof(TreeView)); break;
            case kMbrTreeNodes:
                rc = r.device((void**)&L->mbr_tree.nodes, nullptr);
                L->mbr_tree.nodes_bytes = r.bytes;
                L->mbr_tree.n_nodes = r.bytes / 512;
                L->mbr_tree.view.nodes = L->mbr_tree.nodes;
                break;
            default: {
                uint32_t which = r.tag >= kLearned1 ? 1 : 0;
                uint32_t sub = r.tag - (which ? kLearned1 : kLearned0);
                if (r.tag < kLearned0 || sub > kLUse || sub == 0) {
                    set_error("hv_layer_load_file: unknown record %u", r.tag);
                    rc = HV_EINVAL;
                    break;
                }
                Learned& l = which ? L->mbr_learned : L->learned;
                LearnedView& v = l.view;
                auto* tr = &l.allocs;
                switch (sub) {
                    case kLScalars: rc = r.host(&ls[which], sizeof(LScalars)); break;
                    case kLKb: rc = r.device(&d, tr); v.seg_k0 = (const uint64_t*)d; break;
                    case kLPa: rc = r.device(&d, tr); v.seg_a = (const float*)d; break;
                    case kLPc: rc = r.device(&d, tr); v.seg_b = (const float*)d; break;
                    case kLPinv: rc = r.device(&d, tr); v.pinv = (const float*)d; break;
                    case kLEps: rc = r.device(&d, tr); v.eps_piece = (const uint32_t*)d; break;
                    case kLRadix: rc = r.device(&d, tr); v.radix = (const uint32_t*)d; break;
                    case kLMlp: rc = r.device(&d, tr); v.mlp = (const uint16_t*)d; break;
                    case kLEmb: rc = r.device(&d, tr); v.emb = (const uint16_t*)d; break;
                    case kLSideTree: rc = r.host(&l.outlier_tree.view, sizeof(TreeView)); break;
                    case kLSideNodes:
                        rc = r.device((void**)&l.outlier_tree.nodes, nullptr);
                        l.outlier_tree.nodes_bytes = r.bytes;
                        l.outlier_tree.n_nodes = r.bytes / 512;
                        l.outlier_tree.view.nodes = l.outlier_tree.nodes;
                        break;
                    case kLSideObj: rc = r.device(&d, tr); v.outlier_obj = (const int4*)d; break;
                    case kLSideIds: rc = r.device(&d, tr); v.outlier_ids = (const uint32_t*)d; break;
                    case kLUse: rc = r.device(&d, tr); v.use_mlp = (const uint8_t*)d; break;
                }
            }
        }
    }
    if (r.stage) cudaFreeHost(r.stage);
    fclose(f);
    if (rc == HV_OK && L->kind == HV_LAYER_POLYGONS && !L->poly_edge_off) {
        set_error("hv_layer_load_file: polygon records missing");
        rc = HV_EINVAL;
    }
    if (rc == HV_OK) {
        L->indexes = HV_INDEX_RTREE;
        for (int which = 0; which < 2; which++) {
            Learned& l = which ? L->mbr_learned : L->learned;
            if (!(h.indexes & HV_INDEX_LEARNED) || (which == 1 && L->kind != HV_LAYER_POLYGONS)) continue;
            LearnedView& v = l.view;
            v.keys = which ? L->mbr_keys : L->keys;
            v.n_seg = ls[which].n_seg;
            v.P = ls[which].P;
            v.hidden = ls[which].hidden;
            v.halo = ls[which].halo;
            v.eps = ls[which].eps;
            v.eps_linear = ls[which].eps_linear;
            v.eps_mlp = ls[which].eps_mlp;
            v.mean_err = ls[which].mean_err;
            v.mean_err_linear = ls[which].mean_err_linear;
            v.mean_window = ls[which].mean_window;
            v.mean_window_linear = ls[which].mean_window_linear;
            v.pieces_mlp = ls[which].pieces_mlp;
            v.n_obj = ls[which].n_obj;
            l.train_ms = ls[which].train_ms;
            l.n_outliers = ls[which].n_outliers;
            v.outliers = l.outlier_tree.view;
            v.ready = true;
        }
        if (h.indexes & HV_INDEX_LEARNED) L->indexes |= HV_INDEX_LEARNED;
        rc = dev_alloc(c, (void**)&L->status, 16);
        if (rc == HV_OK && cudaMemset(L->status, 0, 16) != cudaSuccess) rc = HV_ECUDA;
    }
    if (rc != HV_OK) {
        free_layer_public(L);
        return rc;
    }
    *out = (hv_layer*)L;
    return HV_OK;
}

}  // extern "C"
