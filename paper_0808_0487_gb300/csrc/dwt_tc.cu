// dwt_tc.cu -- split-BF16 tensor-core form of the p = 2 transform (placeholder
// until the tcgen05 kernels land).
#include "dwt_internal.cuh"

namespace dwt {

int run_tc_transform(dwt_plan_s*, const float*, float*, int, long long, long long, int, cudaStream_t) {
    set_error("the split-BF16 tensor-core form is not built yet");
    return DWT_EUNSUPPORTED;
}

}  // namespace dwt
