#include "internal.h"
namespace corr {
corr_status launch_xengine_tc(const Handle &, const void *, const float2 *, bool, cudaStream_t) {
    return CORR_EUNSUPPORTED;
}
}  // namespace corr
