// Optimal sampling distribution (Theorem variance, Eq. optimal_prob):
//   q(col) proportional to ||R_[n](:, col)||_2 ||G^{!=n}_{[2]}(col, :)||_2 over
//   all J_n columns of X_[n], R_[n] = G_{n(2)} (G^{!=n}_{[2]})^T - X_[n].
// It needs the full residual of mode n every step (the paper calls it
// impractical); these kernels evaluate it exactly, then draw |F| full column
// indices with the integer-CDF sampler on the OPT Philox stream and decode
// them into slice indices (Definition of the mode-n unfolding).
//   1. opt_weights_kernel: per tile of 64 columns, subchain rows by the slice
//      chain, residual columns G_n Z^T - X_[n](:, tile) (FP32/FP64 SIMT), and
//      a(col) in FP64.
//   2. block sums -> total (fixed order) -> q = a / total, integer weights
//      round(q 2^52), inclusive prefix sums (three-level scan).
//   3. opt_sample_kernel: draws, binary search, decode, p_F = q(col).
// An exact fit (all a = 0) falls back to the uniform distribution.
#include "blocks.cuh"
#include "internal.h"

namespace trsgd {

static constexpr int kOptCols = 64;
static constexpr int kScanBlock = 1024;

struct OptArgs {
  int N, n;
  int I[kMaxOrder], R[kMaxOrder];
  const void *cores[kMaxOrder];
  const void *xmode;     // mode-major copy of X for mode n
  long long ldx;
  long long Jn;
  double *a;             // [Jn]
  int TI;
};

template <typename T, typename XT, int RMAX>
__global__ void __launch_bounds__(256) opt_weights_kernel(OptArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = p.N, n = p.n, L = N - 1;
  const int Rn = p.R[n], Rn1 = p.R[(n + 1) % N], Q = Rn * Rn1, In = p.I[n];
  T *zt = reinterpret_cast<T *>(smem);                 // [Q][kOptCols]
  T *gt = zt + (size_t)Q * kOptCols;                   // [Q][TI]
  double *colsq = reinterpret_cast<double *>(gt + (size_t)Q * p.TI);   // [kOptCols]
  double *znrm = colsq + kOptCols;                     // [kOptCols]
  double *dsq = znrm + kOptCols;                       // [kOptCols][TI] squared residuals of a row chunk
  const T *cores_c[kMaxOrder];
  int R[kMaxOrder], order[kMaxOrder];
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) {
    cores_c[k] = static_cast<const T *>(p.cores[k]);
    R[k] = p.R[k];
    order[k] = (k < L) ? (n + 1 + k) % N : 0;
  }
  const long long cbase = (long long)blockIdx.x * kOptCols;
  const int jb = (int)min((long long)kOptCols, p.Jn - cbase);
  for (int e = threadIdx.x; e < jb * Rn1; e += blockDim.x) {
    const int jl = e / Rn1, rp = e % Rn1;
    long long rem = cbase + jl;
    int sidx[kMaxOrder];
#pragma unroll
    for (int s = 0; s < kMaxOrder; ++s) {
      if (s < L) {
        const int d = p.I[order[s]];
        sidx[s] = (int)(rem % d);
        rem /= d;
      } else {
        sidx[s] = 0;
      }
    }
    T row[RMAX];
    chain_row<RMAX, T>(cores_c, R, N, order, sidx, L, rp, row);
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < Rn) zt[(size_t)(r + rp * Rn) * kOptCols + jl] = row[r];
  }
  for (int jl = threadIdx.x; jl < kOptCols; jl += blockDim.x) colsq[jl] = 0.0;
  __syncthreads();
  for (int jl = threadIdx.x; jl < jb; jl += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double v = (double)zt[(size_t)q * kOptCols + jl];
      s += v * v;
    }
    znrm[jl] = s;
  }
  const T *Gn = cores_c[n];
  const XT *X = static_cast<const XT *>(p.xmode);
  for (int i0 = 0; i0 < In; i0 += p.TI) {
    const int ti = min(p.TI, In - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < ti * Q; e += blockDim.x) {
      const int ii = e / Q, q = e % Q;
      gt[(size_t)q * p.TI + ii] = Gn[(size_t)(i0 + ii) * Q + q];
    }
    __syncthreads();
    gemm_tn<4, 2, T>(jb, ti, Q, zt, kOptCols, gt, p.TI, nullptr, [&](int jl, int ii, T v) {
      const double x = (double)to_compute(X[(cbase + jl) * p.ldx + i0 + ii]);
      const double d = (double)v - x;
      dsq[(size_t)jl * p.TI + ii] = d * d;
    });
    __syncthreads();
    // column sums in increasing row order, one thread per column (deterministic)
    for (int jl = threadIdx.x; jl < jb; jl += blockDim.x) {
      double s = colsq[jl];
      for (int ii = 0; ii < ti; ++ii) s += dsq[(size_t)jl * p.TI + ii];
      colsq[jl] = s;
    }
  }
  __syncthreads();
  for (int jl = threadIdx.x; jl < jb; jl += blockDim.x) p.a[cbase + jl] = sqrt(colsq[jl]) * sqrt(znrm[jl]);
}

// Fixed-order sum of a per block of kScanBlock entries.
__global__ void __launch_bounds__(256) opt_block_sums(const double *a, long long n, double *bsum) {
  __shared__ double part[256];
  const long long base = (long long)blockIdx.x * kScanBlock;
  double s = 0.0;
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
    if (base + i < n) s += a[base + i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
    bsum[blockIdx.x] = t;
  }
}

// total = sum of the block sums in order; uniform fallback flag when total == 0.
__global__ void opt_total(const double *bsum, int nb, double *total) {
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += bsum[b];
    total[0] = t;
  }
}

// q = a / total (or 1/J_n on an exact fit), integer weights, per-block
// inclusive scan (sequential within the block by thread 0 after the parallel
// conversion; integer addition is exact, so any order gives the same sums).
__global__ void __launch_bounds__(256) opt_scan_local(const double *a, long long n, long long Jn, const double *total,
                                                      double *q, unsigned long long *cdf, unsigned long long *btot) {
  __shared__ unsigned long long w[kScanBlock];
  const long long base = (long long)blockIdx.x * kScanBlock;
  const double tot = total[0];
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x) {
    unsigned long long wi = 0;
    if (base + i < n) {
      const double qi = tot > 0.0 ? __ddiv_rn(a[base + i], tot) : __ddiv_rn(1.0, (double)Jn);
      q[base + i] = qi;
      wi = __double2ull_rn(__dmul_rn(qi, 4503599627370496.0));
    }
    w[i] = wi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < kScanBlock; ++i) {
      run += w[i];
      w[i] = run;
    }
    btot[blockIdx.x] = run;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
    if (base + i < n) cdf[base + i] = w[i];
}

__global__ void opt_scan_blocks(unsigned long long *btot, int nb) {
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int b = 0; b < nb; ++b) {
      const unsigned long long v = btot[b];
      btot[b] = run;   // exclusive offsets
      run += v;
    }
  }
}

__global__ void __launch_bounds__(256) opt_scan_add(unsigned long long *cdf, long long n, const unsigned long long *boff) {
  const long long base = (long long)blockIdx.x * kScanBlock;
  const unsigned long long o = boff[blockIdx.x];
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
    if (base + i < n) cdf[base + i] += o;
}

// |F| draws on the OPT stream (slot 0): column = smallest c with
// mulhi64(u, W) < cdf[c]; decoded into (i_{n+1}, ..., i_{n-1}) with i_{n+1}
// fastest; idx[j][n] = -1; pF[j] = q[column].
__global__ void opt_sample_kernel(int N, int n, const int *I, unsigned long long seed, long long t, int J, long long Jn,
                                  const unsigned long long *cdf, const double *q, int *idx, double *pF) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const uint64_t u = draw_u64(seed, t, kStreamOpt, 0, (uint32_t)j);
  const uint64_t W = __ldcg(cdf + Jn - 1);
  const uint64_t target = mulhi64(u, W);
  long long lo = 0, hi = Jn - 1;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if ((uint64_t)__ldcg(cdf + mid) > target) hi = mid; else lo = mid + 1;
  }
  long long rem = lo;
  for (int s = 0; s < N - 1; ++s) {
    const int k = (n + 1 + s) % N;
    idx[(size_t)j * N + k] = (int)(rem % I[k]);
    rem /= I[k];
  }
  idx[(size_t)j * N + n] = -1;
  pF[j] = __ldcg(q + lo);
}

template <typename T, typename XT, int RMAX>
static cudaError_t opt_weights_t(OptArgs p, cudaStream_t s) {
  const int Q = p.R[p.n] * p.R[(p.n + 1) % p.N];
  p.TI = 64;
  auto bytes = [&](int ti) {
    return (size_t)Q * (kOptCols + ti) * sizeof(T) + (2 + (size_t)ti) * kOptCols * sizeof(double);
  };
  size_t smem = bytes(p.TI);
  while (smem > 200 * 1024 && p.TI > 8) {
    p.TI /= 2;
    smem = bytes(p.TI);
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto k = opt_weights_kernel<T, XT, RMAX>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = (p.Jn + kOptCols - 1) / kOptCols;
  k<<<(unsigned)blocks, 256, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_optimal_sampling(int core_dtype, int x_dtype, int N, int n, const int *I, const int *R,
                                    const void *const *cores, const void *xmode, long long ldx,
                                    unsigned long long seed, long long t, int J, OptBuffers &b, cudaStream_t s) {
  OptArgs p = {};
  p.N = N;
  p.n = n;
  long long Jn = 1;
  int rmax = 1;
  for (int k = 0; k < N; ++k) {
    p.I[k] = I[k];
    p.R[k] = R[k];
    p.cores[k] = cores[k];
    if (k != n) Jn *= I[k];
    rmax = R[k] > rmax ? R[k] : rmax;
  }
  p.xmode = xmode;
  p.ldx = ldx;
  p.Jn = Jn;
  p.a = b.a;
  cudaError_t e;
  if (core_dtype == 0) {
    e = rmax <= 8 ? opt_weights_t<double, double, 8>(p, s) : opt_weights_t<double, double, 16>(p, s);
  } else if (x_dtype == 2) {
    e = rmax <= 8 ? opt_weights_t<float, __nv_bfloat16, 8>(p, s) : opt_weights_t<float, __nv_bfloat16, 16>(p, s);
  } else {
    e = rmax <= 8 ? opt_weights_t<float, float, 8>(p, s) : opt_weights_t<float, float, 16>(p, s);
  }
  if (e != cudaSuccess) return e;
  const int nb = (int)((Jn + kScanBlock - 1) / kScanBlock);
  opt_block_sums<<<nb, 256, 0, s>>>(b.a, Jn, b.bsum);
  opt_total<<<1, 32, 0, s>>>(b.bsum, nb, b.total);
  opt_scan_local<<<nb, 256, 0, s>>>(b.a, Jn, Jn, b.total, b.q, b.cdf, b.btot);
  opt_scan_blocks<<<1, 32, 0, s>>>(b.btot, nb);
  opt_scan_add<<<nb, 256, 0, s>>>(b.cdf, Jn, b.btot);
  opt_sample_kernel<<<(J + 127) / 128, 128, 0, s>>>(N, n, b.dims, seed, t, J, Jn, b.cdf, b.q, b.idx, b.pf);
  return cudaGetLastError();
}

}  // namespace trsgd
