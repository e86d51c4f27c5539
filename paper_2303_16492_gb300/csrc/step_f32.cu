// Fused cluster step: FP32 cores and fibers, FMA units.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(float, float, 0, false)
}  // namespace trsgd
