// Tensor-core form (tcgen05/TMEM) of exact Gaussian KDE — see the implementation below.
#include "internal.h"

namespace stagkde {

bool tc_supported(int64_t) { return false; }
int tc_prepare_points(stag_kde *, const float *) { return fail(STAG_KDE_EUNSUPPORTED, "tensor-core form not built"); }
int tc_query(stag_kde *, const float *, int64_t, double *, cudaStream_t, int *) {
    return fail(STAG_KDE_EUNSUPPORTED, "tensor-core form not built");
}
void tc_free(stag_kde *) {}

}  // namespace stagkde
