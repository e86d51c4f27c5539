// Set-up and evaluation kernels: mode-major copies of X, Euclidean sampling
// tables, full reconstruction TR({G_n}) and the relative error (RSE).
#include "blocks.cuh"
#include "internal.h"
#include "tables.cuh"

namespace trsgd {

template <typename S, typename D> __device__ __forceinline__ D cvt(S v) { return (D)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<float, __nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 v) {
  return v;
}

// X viewed as (A, In, B) with A = prod_{k<n} I_k fastest, B = prod_{k>n} I_k.
// Row col = b + a*B of the mode-n copy holds the fiber X(a, :, b)
// (Definition of the mode-n unfolding: i_{n+1} fastest, then i_1..i_{n-1}).
template <typename S, typename D>
__global__ void mode_copy_transpose(const S *__restrict__ X, D *__restrict__ out, long long A,
                                    long long In, long long B, long long ld, long long tilesI,
                                    long long tilesA) {
  __shared__ D tile[32][33];
  const long long id = blockIdx.x;
  const long long ti = id % tilesI, ta = (id / tilesI) % tilesA, b = id / (tilesI * tilesA);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  // read: a fastest in X (coalesced along a)
  for (int r = ty; r < 32; r += 8) {
    const long long i = ti * 32 + r, a = ta * 32 + tx;
    if (i < In && a < A) tile[r][tx] = cvt<S, D>(X[a + i * A + b * A * In]);
  }
  __syncthreads();
  // write: i fastest in the copy (coalesced along i)
  for (int r = ty; r < 32; r += 8) {
    const long long a = ta * 32 + r, i = ti * 32 + tx;
    if (i < In && a < A) out[(b + a * B) * ld + i] = tile[tx][r];
  }
}

template <typename S, typename D>
__global__ void mode_copy_rows(const S *__restrict__ X, D *__restrict__ out, long long In,
                               long long B, long long ld) {
  const long long total = In * B;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / In, i = e % In;
    out[b * ld + i] = cvt<S, D>(X[e]);
  }
}

template <typename S, typename D>
static cudaError_t mode_copy_t(const void *X, void *out, long long A, long long In, long long B,
                               long long ld, cudaStream_t s) {
  if (A == 1) {
    const long long total = In * B;
    long long blocks = (total + 255) / 256;
    if (blocks > (1LL << 20)) blocks = 1LL << 20;
    mode_copy_rows<S, D><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const S *>(X),
                                                        static_cast<D *>(out), In, B, ld);
  } else {
    const long long tI = (In + 31) / 32, tA = (A + 31) / 32;
    const long long blocks = tI * tA * B;
    mode_copy_transpose<S, D><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<const S *>(X), static_cast<D *>(out), A, In, B, ld, tI, tA);
  }
  return cudaGetLastError();
}

cudaError_t launch_mode_copy(int src_dtype, int dst_dtype, const void *X, void *out, long long A,
                             long long In, long long B, long long ld, cudaStream_t s) {
  if (src_dtype == 0 && dst_dtype == 0) return mode_copy_t<double, double>(X, out, A, In, B, ld, s);
  if (src_dtype == 1 && dst_dtype == 1) return mode_copy_t<float, float>(X, out, A, In, B, ld, s);
  if (src_dtype == 1 && dst_dtype == 2) return mode_copy_t<float, __nv_bfloat16>(X, out, A, In, B, ld, s);
  if (src_dtype == 2 && dst_dtype == 2)
    return mode_copy_t<__nv_bfloat16, __nv_bfloat16>(X, out, A, In, B, ld, s);
  return cudaErrorInvalidValue;
}

// Euclidean distribution of one core (Lemma euc_est): slice norms as
// left-to-right FP64 sums in column order, the core norm as the left-to-right
// sum of slice norms, p = norm_i / total, integer weights round(p * 2^52)
// and their inclusive prefix sums.  One CTA.
template <typename T>
__global__ void euclid_table_kernel(const T *__restrict__ G, int I, int Q, double *snorm,
                                    double *prob, unsigned long long *cdf, int *status) {
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double v = (double)G[(size_t)i * Q + q];
      s = __dadd_rn(s, __dmul_rn(v, v));
    }
    snorm[i] = s;
  }
  __syncthreads();
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < I; ++i) s = __dadd_rn(s, snorm[i]);
    tot = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    const double p = __ddiv_rn(snorm[i], tot);
    prob[i] = p;
    cdf[i] = __double2ull_rn(__dmul_rn(p, 4503599627370496.0));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < I; ++i) {
      run += cdf[i];
      cdf[i] = run;
    }
    if (!(tot > 0.0) && status) atomicCAS(status, 0, kStatusNumeric);
  }
}

cudaError_t launch_euclid_table(int core_dtype, const void *G, int I, int Q, double *snorm,
                                double *prob, unsigned long long *cdf, cudaStream_t s) {
  if (core_dtype == 0)
    euclid_table_kernel<double><<<1, 256, 0, s>>>(static_cast<const double *>(G), I, Q, snorm, prob, cdf, nullptr);
  else
    euclid_table_kernel<float><<<1, 256, 0, s>>>(static_cast<const float *>(G), I, Q, snorm, prob, cdf, nullptr);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(512) leverage_init_kernel(const T *G, int I, int Q, double *prob,
                                                            unsigned long long *cdf, int *status) {
  extern __shared__ __align__(128) unsigned char smem[];
  leverage_table_cta<T>(G, I, Q, smem, prob, cdf, status);
}

cudaError_t launch_leverage_table(int core_dtype, const void *G, int I, int Q, double *prob,
                                  unsigned long long *cdf, int *status, cudaStream_t s) {
  const size_t bytes = leverage_scratch_bytes(I, Q, core_dtype == 0 ? 8 : 4);
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (core_dtype == 0) {
    e = cudaFuncSetAttribute(leverage_init_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      leverage_init_kernel<double><<<1, 512, bytes, s>>>(static_cast<const double *>(G), I, Q, prob, cdf, status);
  } else {
    e = cudaFuncSetAttribute(leverage_init_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      leverage_init_kernel<float><<<1, 512, bytes, s>>>(static_cast<const float *>(G), I, Q, prob, cdf, status);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// ---------------------------------------------------------------------------
// Reconstruction X_[1] = G_{1(2)} (G^{!=1}_{[2]})^T, one tile of JT columns of
// X_[1] per CTA; optional comparison with X_ref (sum of squared differences
// and of X_ref^2 in FP64).  Column j of X_[1] is the multi-index of
// (i_2, ..., i_N), so X(i, j) sits at i + j*I_1 in the i_1-fastest layout.
// ---------------------------------------------------------------------------
struct ReconArgs {
  int N, I[kMaxOrder], R[kMaxOrder];
  const void *cores[kMaxOrder];
  void *X;
  const void *Xref;
  double *sums;       // [2]: sum (x - x_ref)^2, sum x_ref^2 (or null)
  double *partials;   // [2 * blocks]: the same two sums per CTA, reduced in a fixed order
  long long J1;
  int JT, TI;
};

template <typename T, int RMAX>
__global__ void __launch_bounds__(256) reconstruct_kernel(ReconArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N;
  const int Q = a.R[0] * a.R[1];
  T *zt = reinterpret_cast<T *>(smem);                     // [Q][JT]
  T *gt = zt + (size_t)Q * a.JT;                           // [Q][TI]
  const T *cores_c[kMaxOrder];
  int R[kMaxOrder], order[kMaxOrder];
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) {
    cores_c[k] = static_cast<const T *>(a.cores[k]);
    R[k] = a.R[k];
    order[k] = (k + 1 < N) ? k + 1 : 0;
  }
  const long long jbase = (long long)blockIdx.x * a.JT;
  const int jb = (int)min((long long)a.JT, a.J1 - jbase);
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
      if (r < R0) zt[(size_t)(r + rp * R0) * a.JT + jl] = row[r];
  }
  double sd = 0.0, sr = 0.0;
  const int I0 = a.I[0];
  const T *G0 = cores_c[0];
  T *X = static_cast<T *>(a.X);
  const T *Xr = static_cast<const T *>(a.Xref);
  for (int i0 = 0; i0 < I0; i0 += a.TI) {
    const int ti = min(a.TI, I0 - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < ti * Q; e += blockDim.x) {
      const int ii = e / Q, q = e % Q;
      gt[(size_t)q * a.TI + ii] = G0[(size_t)(i0 + ii) * Q + q];
    }
    __syncthreads();
    gemm_tn<4, 2, T>(jb, ti, Q, zt, a.JT, gt, a.TI, nullptr, [&](int jl, int ii, T v) {
      const long long pos = (long long)(i0 + ii) + (jbase + jl) * (long long)I0;
      if (X) X[pos] = v;
      if (Xr) {
        const double r = (double)Xr[pos];
        const double d = (double)v - r;
        sd += d * d;
        sr += r * r;
      }
    });
  }
  if (a.sums) {
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sd; red[1][w] = sr; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double A = 0.0, B = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { A += red[0][k]; B += red[1][k]; }
      a.partials[2 * blockIdx.x] = A;
      a.partials[2 * blockIdx.x + 1] = B;
    }
  }
}

// Fixed-order sum of the per-CTA pairs: thread t adds CTAs t, t + 256, ... in
// increasing order, then thread 0 adds the 256 thread sums in order (the
// result does not depend on the schedule of the CTAs).
__global__ void __launch_bounds__(256) reconstruct_sums_kernel(const double *partials, long long nblocks,
                                                              double *sums) {
  __shared__ double sd[256], sr[256];
  double A = 0.0, B = 0.0;
  for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) {
    A += partials[2 * b];
    B += partials[2 * b + 1];
  }
  sd[threadIdx.x] = A;
  sr[threadIdx.x] = B;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      x += sd[t];
      y += sr[t];
    }
    sums[0] = x;
    sums[1] = y;
  }
}

// Column tile JT (= TI) of the reconstruction: 64, halved while the two
// shared-memory tiles exceed 200 KB.
static int recon_tile(int Q, size_t esize) {
  int jt = 64;
  while ((size_t)Q * 2 * jt * esize > 200 * 1024 && jt > 8) jt /= 2;
  return jt;
}

template <typename T, int RMAX>
static cudaError_t recon_t(ReconArgs a, cudaStream_t s) {
  const int Q = a.R[0] * a.R[1];
  a.JT = a.TI = recon_tile(Q, sizeof(T));
  const size_t smem = (size_t)Q * (a.JT + a.TI) * sizeof(T);
  auto k = reconstruct_kernel<T, RMAX>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = (a.J1 + a.JT - 1) / a.JT;
  k<<<(unsigned)blocks, 256, smem, s>>>(a);
  if (a.sums) reconstruct_sums_kernel<<<1, 256, 0, s>>>(a.partials, blocks, a.sums);
  return cudaGetLastError();
}

long long reconstruct_partials(int dtype, int N, const int *I, const int *R) {
  long long J1 = 1;
  for (int k = 1; k < N; ++k) J1 *= I[k];
  const int jt = recon_tile(R[0] * R[1], dtype == 0 ? 8 : 4);
  return 2 * ((J1 + jt - 1) / jt);
}

cudaError_t launch_reconstruct(int dtype, int N, const int *I, const int *R, const void *const *cores,
                               void *X, const void *Xref, double *sums, double *partials, cudaStream_t s) {
  ReconArgs a = {};
  a.N = N;
  int rmax = 1;
  long long J1 = 1;
  for (int k = 0; k < N; ++k) {
    a.I[k] = I[k];
    a.R[k] = R[k];
    a.cores[k] = cores[k];
    rmax = R[k] > rmax ? R[k] : rmax;
    if (k > 0) J1 *= I[k];
  }
  a.X = X;
  a.Xref = Xref;
  a.sums = sums;
  a.partials = partials;
  if (sums && !partials) return cudaErrorInvalidValue;
  a.J1 = J1;
  a.JT = 64;
  a.TI = 64;
  if (dtype == 0) {
    if (rmax <= 4) return recon_t<double, 4>(a, s);
    if (rmax <= 8) return recon_t<double, 8>(a, s);
    if (rmax <= 16) return recon_t<double, 16>(a, s);
    return recon_t<double, 32>(a, s);
  }
  if (dtype == 1) {
    if (rmax <= 4) return recon_t<float, 4>(a, s);
    if (rmax <= 8) return recon_t<float, 8>(a, s);
    if (rmax <= 16) return recon_t<float, 16>(a, s);
    return recon_t<float, 32>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace trsgd
