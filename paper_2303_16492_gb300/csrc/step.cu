// Dispatch of the fused cluster step (step_kernel.cuh) to its instantiations,
// and the device-resident iteration counter.  The kernel variants are
// compiled in step_f64.cu, step_f32.cu, step_f32x3.cu and step_bf16.cu.
#include "internal.h"

namespace trsgd {

// RMAX: register length of one chain row; the smallest of 4, 8, 12, 16 that
// holds every rank of the problem.  Pieces: lay.tcp (FP32 cores only; the
// BF16-mixed mode always runs on two pieces).
#define TRSGD_DISPATCH_RS(FN, T, XT, NPC, SC, ...)                 \
  do {                                                             \
    if (rmax <= 4) return FN<T, XT, 4, NPC, SC>(__VA_ARGS__);      \
    if (rmax <= 8) return FN<T, XT, 8, NPC, SC>(__VA_ARGS__);      \
    if (rmax <= 12) return FN<T, XT, 12, NPC, SC>(__VA_ARGS__);    \
    return FN<T, XT, 16, NPC, SC>(__VA_ARGS__);                    \
  } while (0)

// the scaled variant's code only in the kernels of launches that hold a
// scaled problem (its Gram buffers in the layout)
#define TRSGD_DISPATCH_R(FN, T, XT, NPC, ...)                                        \
  do {                                                                               \
    if (lay.QH > 0) TRSGD_DISPATCH_RS(FN, T, XT, NPC, true, __VA_ARGS__);            \
    TRSGD_DISPATCH_RS(FN, T, XT, NPC, false, __VA_ARGS__);                           \
  } while (0)

#define TRSGD_DISPATCH(FN, ...)                                                      \
  do {                                                                               \
    if (core_dtype == 0) TRSGD_DISPATCH_R(FN, double, double, 0, __VA_ARGS__);       \
    if (x_dtype == 2) TRSGD_DISPATCH_R(FN, float, __nv_bfloat16, 2, __VA_ARGS__);    \
    if (lay.tcp == 3) TRSGD_DISPATCH_R(FN, float, float, 3, __VA_ARGS__);            \
    TRSGD_DISPATCH_R(FN, float, float, 0, __VA_ARGS__);                              \
  } while (0)

cudaError_t step_kernel_prepare(int core_dtype, int x_dtype, int rmax, const StepLayout &lay) {
  TRSGD_DISPATCH(step_prepare_t, lay);
}

cudaError_t launch_step(int core_dtype, int x_dtype, int rmax, const ProbDesc *descs, int nprob,
                        const StepLayout &lay, int threads, long long t0, int nsteps,
                        const long long *t_dev, cudaStream_t s) {
  TRSGD_DISPATCH(step_launch_t, descs, nprob, lay, threads, t0, nsteps, t_dev, s);
}

// *t += T, after the step launch that read *t has finished (same stream)
__global__ void advance_counter_kernel(long long *t, long long T, int set) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t = set ? T : *t + T;
}

cudaError_t launch_advance_counter(long long *t, long long T, int set, cudaStream_t s) {
  advance_counter_kernel<<<1, 32, 0, s>>>(t, T, set);
  return cudaGetLastError();
}

int step_max_smem() { return 232448; }

}  // namespace trsgd
