// Tensor-core variant of the fused kernel (blur as a banded Toeplitz MMA).
#include "bf_internal.cuh"

namespace bf {

int launch_tc(const bf_plan_s &, const float *, float *, int, int, int, int, cudaStream_t) {
    return BF_ERR_UNSUPPORTED;
}

}  // namespace bf
