// Serving loop (placeholder until the server lands).
#include "hv_internal.h"

using namespace hv;

extern "C" {

int hv_server_start(hv_ctx*, hv_layer* const*, uint32_t, const hv_server_opts*, hv_server** out) {
    if (out) *out = nullptr;
    set_error("server not available in this build");
    return HV_ESTATE;
}
int hv_server_submit(hv_server*, const hv_tile_req*, uint64_t) { return HV_ESTATE; }
int hv_server_poll(hv_server*, hv_done*, uint32_t, uint32_t* n) { if (n) *n = 0; return HV_ESTATE; }
int hv_server_stop(hv_server*) { return HV_ESTATE; }
int hv_layer_save(hv_layer*, const char*) { set_error("not available"); return HV_ESTATE; }
int hv_layer_load_file(hv_ctx*, const char*, hv_layer** out) { if (out) *out = nullptr; set_error("not available"); return HV_ESTATE; }

}
