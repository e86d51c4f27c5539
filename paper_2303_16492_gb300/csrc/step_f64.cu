// Fused cluster step: FP64 cores and fibers, FMA units.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(double, double, 0, false)
}  // namespace trsgd
