// Relative error that allocates nothing: trsgd_rel_error_static.
//
// Same quantity as trsgd_rel_error, RSE = ||TR(G) - X_ref||_F / ||X_ref||_F,
// for callers that cannot call cudaMalloc.  Its only scratch, one pair of
// partial sums per tile of 64 columns of X_[1], lives in a file-scope
// __device__ array of fixed size (kMaxTiles pairs); every GPU that loads the
// library holds that array until the process exits.  The partial sums are
// reduced in a fixed order by a second kernel, so the result does not depend
// on the schedule.
#include <mutex>

#include "blocks.cuh"
#include "internal.h"
#include "trsgd.h"

namespace trsgd {

static constexpr int kMaxTiles = 65536;   // 1 MiB of scratch: up to 4,194,304 columns of X_[1]
static constexpr int kTileCols = 64;
static constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_relerr_scratch[2 * kMaxTiles];

struct StaticArgs {
  int N, I[kMaxOrder], R[kMaxOrder];
  const void *cores[kMaxOrder];
  const void *Xref;
  long long J1;
  int TI;
};

// One tile of kTileCols columns of X_[1] per CTA: the subchain rows by the
// slice chain, then X_[1](:, tile) = G_{1(2)} Z^T, compared with X_ref; the
// CTA's two sums go to partials[2 * tile], partials[2 * tile + 1].
template <typename T, int RMAX>
__global__ void __launch_bounds__(256) relerr_tiles_kernel(StaticArgs a, double *partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N;
  const int Q = a.R[0] * a.R[1];
  T *zt = reinterpret_cast<T *>(smem);            // [Q][kTileCols]
  T *gt = zt + (size_t)Q * kTileCols;             // [Q][TI]
  const T *cores_c[kMaxOrder];
  int R[kMaxOrder], order[kMaxOrder];
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) {
    cores_c[k] = static_cast<const T *>(a.cores[k]);
    R[k] = a.R[k];
    order[k] = (k + 1 < N) ? k + 1 : 0;
  }
  const long long jbase = (long long)blockIdx.x * kTileCols;
  const int jb = (int)min((long long)kTileCols, a.J1 - jbase);
  const int R0 = R[0], R1 = R[1];
  for (int e = threadIdx.x; e < jb * R1; e += blockDim.x) {
    const int jl = e / R1, rp = e % R1;
    long long rem = jbase + jl;
    int sidx[kMaxOrder];
#pragma unroll
    for (int s = 0; s < kMaxOrder; ++s) {
      if (s < N - 1) {
        const int d = a.I[order[s]];
        sidx[s] = (int)(rem % d);
        rem /= d;
      } else {
        sidx[s] = 0;
      }
    }
    T row[RMAX];
    chain_row<RMAX, T>(cores_c, R, N, order, sidx, N - 1, rp, row);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R0) zt[(size_t)(r + rp * R0) * kTileCols + jl] = row[r];
  }
  double sd = 0.0, sr = 0.0;
  const int I0 = a.I[0];
  const T *G0 = cores_c[0];
  const T *Xr = static_cast<const T *>(a.Xref);
  for (int i0 = 0; i0 < I0; i0 += a.TI) {
    const int ti = min(a.TI, I0 - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < ti * Q; e += blockDim.x) {
      const int ii = e / Q, q = e % Q;
      gt[(size_t)q * a.TI + ii] = G0[(size_t)(i0 + ii) * Q + q];
    }
    __syncthreads();
    gemm_tn<4, 2, T>(jb, ti, Q, zt, kTileCols, gt, a.TI, nullptr, [&](int jl, int ii, T v) {
      const long long pos = (long long)(i0 + ii) + (jbase + jl) * (long long)I0;
      const double r = (double)Xr[pos];
      const double d = (double)v - r;
      sd += d * d;
      sr += r * r;
    });
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = sd;
    red[1][w] = sr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      A += red[0][k];
      B += red[1][k];
    }
    partials[2 * blockIdx.x] = A;
    partials[2 * blockIdx.x + 1] = B;
  }
}

// Fixed-order reduction of the per-tile sums: thread t adds tiles t, t+256, ...
// in increasing order, then thread 0 adds the 256 thread sums in order.
__global__ void __launch_bounds__(256) relerr_finish_kernel(const double *partials, int ntiles, double *out) {
  __shared__ double sd[256], sr[256];
  double A = 0.0, B = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    A += partials[2 * t];
    B += partials[2 * t + 1];
  }
  sd[threadIdx.x] = A;
  sr[threadIdx.x] = B;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      a += sd[t];
      b += sr[t];
    }
    out[0] = b > 0.0 ? sqrt(a / b) : sqrt(a);
  }
}

// *too_big is set (and nothing launched) when the tiles of G_{1(2)} and of the
// subchain rows do not fit in shared memory; other failures are CUDA errors.
template <typename T, int RMAX>
static cudaError_t relerr_static_t(StaticArgs a, double *scratch, int ntiles, double *out, cudaStream_t s,
                                   bool *too_big) {
  const int Q = a.R[0] * a.R[1];
  a.TI = kTileCols;
  size_t smem = (size_t)Q * (kTileCols + a.TI) * sizeof(T);
  while (smem > 200 * 1024 && a.TI > 8) {
    a.TI /= 2;
    smem = (size_t)Q * (kTileCols + a.TI) * sizeof(T);
  }
  *too_big = smem > 200 * 1024;
  if (*too_big) return cudaSuccess;
  auto k = relerr_tiles_kernel<T, RMAX>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ntiles, 256, smem, s>>>(a, scratch);
  relerr_finish_kernel<<<1, 256, 0, s>>>(scratch, ntiles, out);
  return cudaGetLastError();
}

// Device address of the scratch array, looked up once per device (with that
// device current) and reused for the life of the process: a device reset
// (cudaDeviceReset) unloads the module, and the cached address is then stale.
static double *scratch_for_current_device(cudaError_t *err) {
  static std::mutex mu;
  static double *addr[kMaxDevices] = {};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_relerr_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = static_cast<double *>(p);
  }
  return addr[dev];
}

}  // namespace trsgd

extern "C" trsgd_status trsgd_rel_error_static(int32_t N, const int64_t *I, const int64_t *R, int32_t dtype,
                                               const void *const *cores_dev, const void *Xref_dev,
                                               double *out_dev, void *stream) {
  using namespace trsgd;
  if (N < 2 || N > TRSGD_MAX_ORDER || !I || !R || !cores_dev || !Xref_dev || !out_dev) return TRSGD_EINVAL;
  if (dtype != TRSGD_DTYPE_F64 && dtype != TRSGD_DTYPE_F32) return TRSGD_EUNSUPPORTED;
  StaticArgs a = {};
  a.N = N;
  long long J1 = 1;
  int rmax = 1;
  for (int k = 0; k < N; ++k) {
    if (I[k] < 1 || R[k] < 1 || I[k] > (1LL << 30) || !cores_dev[k]) return TRSGD_EINVAL;
    if (R[k] > 16) return TRSGD_EUNSUPPORTED;
    a.I[k] = (int)I[k];
    a.R[k] = (int)R[k];
    a.cores[k] = cores_dev[k];
    rmax = R[k] > rmax ? (int)R[k] : rmax;
    // beyond the fixed scratch: prod_{k>1} I_k > 4,194,304 (checked before each
    // product, so the running product stays far inside 64 bits)
    if (k > 0) {
      if (J1 > (long long)kMaxTiles * kTileCols / I[k]) return TRSGD_EINVAL;
      J1 *= I[k];
    }
  }
  const long long ntiles = (J1 + kTileCols - 1) / kTileCols;
  if (ntiles > kMaxTiles) return TRSGD_EINVAL;
  a.Xref = Xref_dev;
  a.J1 = J1;
  cudaError_t e = cudaSuccess;
  double *scratch = scratch_for_current_device(&e);
  if (!scratch) return TRSGD_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool too_big = false;
  if (dtype == TRSGD_DTYPE_F64) {
    if (rmax <= 4) e = relerr_static_t<double, 4>(a, scratch, (int)ntiles, out_dev, s, &too_big);
    else if (rmax <= 8) e = relerr_static_t<double, 8>(a, scratch, (int)ntiles, out_dev, s, &too_big);
    else e = relerr_static_t<double, 16>(a, scratch, (int)ntiles, out_dev, s, &too_big);
  } else {
    if (rmax <= 4) e = relerr_static_t<float, 4>(a, scratch, (int)ntiles, out_dev, s, &too_big);
    else if (rmax <= 8) e = relerr_static_t<float, 8>(a, scratch, (int)ntiles, out_dev, s, &too_big);
    else e = relerr_static_t<float, 16>(a, scratch, (int)ntiles, out_dev, s, &too_big);
  }
  if (too_big) return TRSGD_EUNSUPPORTED;
  return e == cudaSuccess ? TRSGD_OK : TRSGD_ECUDA;
}
