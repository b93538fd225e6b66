// Learned Hilbert-position index (placeholder until the learned build lands).
#include "hv_internal.h"

namespace hv {

int build_learned(Layer* L, const hv_build_opts* opts) {
    (void)L;
    (void)opts;
    set_error("learned index not available in this build");
    return HV_ESTATE;
}

void free_learned(Ctx* c, Learned* l) {
    for (auto& a : l->allocs) dev_free(c, a.first, a.second);
    l->allocs.clear();
    free_tree(c, &l->outlier_tree);
    l->view = LearnedView();
}

}  // namespace hv
