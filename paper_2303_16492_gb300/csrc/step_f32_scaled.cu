// Fused cluster step: FP32 cores and fibers, FMA units, scaled variant compiled in.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(float, float, 0, true)
}  // namespace trsgd
