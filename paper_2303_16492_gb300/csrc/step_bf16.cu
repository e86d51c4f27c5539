// Fused cluster step: FP32 cores, BF16 fibers, tensor cores on two BF16 pieces.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(float, __nv_bfloat16, 2, false)
}  // namespace trsgd
