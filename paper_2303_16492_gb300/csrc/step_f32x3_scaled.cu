// Fused cluster step: FP32 cores and fibers, tensor cores on three BF16 pieces per operand, scaled variant compiled in.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(float, float, 3, true)
}  // namespace trsgd
