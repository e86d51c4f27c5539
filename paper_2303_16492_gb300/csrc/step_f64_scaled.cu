// Fused cluster step: FP64 cores and fibers, FMA units, scaled variant compiled in.
#include "step_kernel.cuh"

namespace trsgd {
TRSGD_STEP_INSTANTIATE(double, double, 0, true)
}  // namespace trsgd
