// hv_render_tiles_static: tile rendering for callers that cannot allocate
// device memory.
//
// hv_render_tiles stages host requests (and host outputs) through device
// buffers that the library allocates on demand with cudaMalloc.  Some callers
// cannot allow that: hosts whose device memory is owned by another allocator
// or pool, and latency-critical paths where the device synchronisation that
// cudaMalloc / cudaFree may imply is unacceptable.  This entry point uses no
// allocation at all: device requests are read in place, host requests are
// staged in a fixed file-scope device array, and the caller provides the
// output buffer.
#include <mutex>

#include "hv_internal.h"

namespace hv {

namespace {

constexpr uint32_t kStaticMaxTiles = 4096;   // 64 KiB of requests
constexpr int kMaxDevices = 64;

// The staging area, present on every device that loads the library until the
// process exits.  Host code must not use this symbol as an address: on the
// host it names a host-side stand-in.  Its device address comes from
// cudaGetSymbolAddress (per device, with that device current).
static __device__ __align__(256) hv_tile_req g_static_reqs[kStaticMaxTiles];

std::mutex g_static_mu;
hv_tile_req* g_static_addr[kMaxDevices] = {};

// Device address of the staging area on `device` (the current device).
int static_area(int device, hv_tile_req** out) {
    if (device < 0 || device >= kMaxDevices) { set_error("device %d out of range", device); return HV_EINVAL; }
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_reqs);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static request area failed: %s", cudaGetErrorString(e));
            return HV_ECUDA;
        }
        g_static_addr[device] = (hv_tile_req*)p;
    }
    *out = g_static_addr[device];
    return HV_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace hv

using namespace hv;

extern "C" {

int hv_render_tiles_static(hv_layer* layer, const hv_tile_req* reqs, uint32_t n, int mode, int index_kind,
                           const hv_style* style, void* out, uint64_t out_bytes, void* stream) {
    if (!layer) { set_error("hv_render_tiles_static: NULL layer"); return HV_EINVAL; }
    Layer* L = (Layer*)layer;
    uint64_t tb = hv_tile_bytes(mode);
    if (tb == 0) { set_error("hv_render_tiles_static: unknown mode %d", mode); return HV_EINVAL; }
    if (index_kind != HV_INDEX_RTREE && index_kind != HV_INDEX_LEARNED) {
        set_error("hv_render_tiles_static: index_kind must be HV_INDEX_RTREE or HV_INDEX_LEARNED");
        return HV_EINVAL;
    }
    if (!(L->indexes & index_kind)) { set_error("hv_render_tiles_static: index not built"); return HV_ESTATE; }
    if (n == 0) return HV_OK;
    if (n > kStaticMaxTiles) {
        set_error("hv_render_tiles_static: %u tiles exceed the static limit of %u per call", n, kStaticMaxTiles);
        return HV_EINVAL;
    }
    if (!reqs || !out) { set_error("hv_render_tiles_static: NULL reqs or out"); return HV_EINVAL; }
    if (out_bytes < (uint64_t)n * tb) { set_error("hv_render_tiles_static: out_bytes too small"); return HV_EINVAL; }
    if (((uintptr_t)out & 15u) != 0) { set_error("hv_render_tiles_static: out must be 16-byte aligned"); return HV_EINVAL; }
    HV_CUDA(cudaSetDevice(L->ctx->device));
    if (!on_device(out)) { set_error("hv_render_tiles_static: out must be device memory"); return HV_EINVAL; }
    bool dev_reqs = on_device(reqs);
    if (!dev_reqs) {
        for (uint32_t k = 0; k < n; k++) {
            const hv_tile_req& q = reqs[k];
            if (q.z > 19 || q.x >= (1u << q.z) || q.y >= (1u << q.z) || q.r16 < 1 || q.r16 > 1024) {
                set_error("hv_render_tiles_static: request %u out of range", k);
                return HV_ERANGE;
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    // device requests need no staging: the kernel reads (and checks) them
    if (dev_reqs) return launch_render(L, reqs, n, mode, index_kind, style, (uint8_t*)out, st);
    hv_tile_req* area = nullptr;
    HV_TRY(static_area(L->ctx->device, &area));
    HV_CUDA(cudaMemcpyAsync(area, reqs, (uint64_t)n * sizeof(hv_tile_req), cudaMemcpyHostToDevice, st));
    return launch_render(L, area, n, mode, index_kind, style, (uint8_t*)out, st);
}

}  // extern "C"
