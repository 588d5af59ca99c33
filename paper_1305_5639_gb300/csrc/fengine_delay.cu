// F-engine instantiations with delay compensation (see fengine_kernel.cuh).
#include "fengine_kernel.cuh"

namespace corr {

corr_status fengine_run_delay(int mode, const FShape &f, const void *volt, const float *scale, void *out,
                              double *power, cudaStream_t st) {
    return launch_feature<kDelay>(mode, f, volt, scale, out, power, st);
}

}  // namespace corr
