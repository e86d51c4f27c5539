// Sampling tables of the non-uniform distributions (Sec. 3.2), computed by one
// CTA: probabilities p_k(i) in FP64 and the inclusive prefix sums of the
// integer weights round(p_k(i) * 2^52) used by the sampler.
#pragma once

#include "blocks.cuh"

namespace trsgd {

// In-place lower Cholesky of the m x m matrix A (leading dim ld) by one CTA.
// Returns false at the first non-positive or non-finite pivot (the same
// decision in every thread).
template <typename T>
__device__ __noinline__ bool cholesky_cta_t(T *A, int m, int ld) {
  A = smem_ptr(A);   // dynamic shared memory
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    const T d = A[k * ld + k];
    if (!(d > T(0)) || !isfinite(d)) return false;
    const T l = sqrt(d);
    __syncthreads();
    if (tid == 0) A[k * ld + k] = l;
    for (int i = k + 1 + tid; i < m; i += NT) A[i * ld + k] = A[i * ld + k] / l;
    __syncthreads();
    const int r = m - k - 1;
    for (int e = tid; e < r * r; e += NT) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j <= i) A[i * ld + j] = fma(-A[i * ld + k], A[j * ld + k], A[i * ld + j]);
    }
  }
  __syncthreads();
  return true;
}

// Inclusive prefix sums of w[0..n) in place, by warp 0 (the other threads
// return at once; callers put barriers around it).  Integer sums: exact in
// any order.  Lane l scans the segment [l s, (l + 1) s), s = ceil(n / 32), then
// adds the exclusive scan of the segment totals.
__device__ __forceinline__ void scan_u64_warp0(unsigned long long *w, int n) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x, seg = (n + 31) / 32;
  const int a = min(n, lane * seg), b = min(n, a + seg);
  unsigned long long run = 0;
  for (int i = a; i < b; ++i) {
    run += w[i];
    w[i] = run;
  }
  unsigned long long incl = run;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const unsigned long long off = incl - run;
  for (int i = a; i < b; ++i) w[i] += off;
}

// prob[i] = p[i] (given) and cdf = inclusive prefix sums of round(p * 2^52).
// scratch: In unsigned long long entries of shared memory.
__device__ __forceinline__ void write_cdf_cta(const double *p, int In, double *prob,
                                              unsigned long long *cdf, unsigned long long *wsc) {
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int i = tid; i < In; i += NT) {
    prob[i] = p[i];
    wsc[i] = __double2ull_rn(__dmul_rn(p[i], 4503599627370496.0));  // * 2^52, exact scaling
  }
  __syncthreads();
  scan_u64_warp0(wsc, In);
  __syncthreads();
  for (int i = tid; i < In; i += NT) cdf[i] = wsc[i];
  __syncthreads();
}

// Bytes of shared scratch leverage_table_cta needs.
__host__ __device__ inline size_t leverage_scratch_bytes(int I, int Q, size_t elem) {
  const int I4 = (I + 3) & ~3, Q4 = (Q + 3) & ~3;
  const int m = I > Q ? Q : I, m4 = (m + 3) & ~3;
  size_t b = (size_t)I4 * (Q4 + 4) * elem;            // A
  b = (b + 127) / 128 * 128 + (size_t)m * m4 * elem;  // Gram / factor
  b = (b + 127) / 128 * 128 + (size_t)I * 16;         // leverage scores + CDF scratch
  return b + 128;
}

// Leverage-based distribution of one core (Lemma lev_est, Definition of the
// leverage scores): p(i) = l_i(A) / rank(A), A = G_{(2)} (I x Q).
//   I > Q: l_i = || L^{-1} a_i^T ||^2 with A^T A = L L^T;
//   I <= Q: A A^T = L L^T exists (full row rank), so every l_i = 1.
// Gram and factor in the core precision, l_i accumulated in FP64.  If the
// factorisation fails (a core numerically rank-deficient in that precision),
// it is retried with a ridge shift delta = 1e-7 tr(M)/m * 10^a, a = 0..6, on
// the diagonal; the resulting ridge leverage scores are normalised by their
// sum, so the table stays exactly the distribution that is sampled (and the
// weights 1/p stay unbiased).  If every shift fails, TRSGD_ENUMERIC is
// latched and the table is left unchanged.  `smem` holds
// leverage_scratch_bytes(I, Q, sizeof(T)).
template <typename T>
__device__ void leverage_table_cta(const T *G, int I, int Q, unsigned char *smem, double *prob,
                                   unsigned long long *cdf, int *status) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int I4 = (I + 3) & ~3, Q4 = (Q + 3) & ~3;
  const int lda = Q4 + 4;                 // row stride of A: multiple of 4, rows start 16-byte aligned
  const bool tall = I > Q;
  const int m = tall ? Q : I, m4 = (m + 3) & ~3;
  T *As = reinterpret_cast<T *>(smem);
  size_t off = ((size_t)I4 * lda * sizeof(T) + 127) / 128 * 128;
  T *M = reinterpret_cast<T *>(smem + off);
  off = (off + (size_t)m * m4 * sizeof(T) + 127) / 128 * 128;
  double *lev = reinterpret_cast<double *>(smem + off);
  unsigned long long *wsc = reinterpret_cast<unsigned long long *>(lev + I);
  for (int e = tid; e < I4 * lda; e += NT) {
    const int i = e / lda, q = e - i * lda;
    As[e] = (i < I && q < Q) ? ld_l2(G + (size_t)i * Q + q) : T(0);
  }
  __syncthreads();
  bool ok = false, ridge = false;
  for (int attempt = 0; attempt < 8 && !ok; ++attempt) {
    if (tall)   // M = A^T A, contraction over the rows i (zero rows pad I to I4)
      gemm_s<4, true, true, T>(Q, Q, I, As, lda, As, lda, nullptr, [=](int a, int b, T v) { M[a * m4 + b] = v; });
    else        // M = A A^T, contraction over the columns q (zero columns pad Q to Q4)
      gemm_s<4, false, false, T>(I, I, Q, As, lda, As, lda, nullptr, [=](int a, int b, T v) { M[a * m4 + b] = v; });
    __syncthreads();
    if (attempt > 0) {   // ridge shift (every thread forms the same trace)
      double tr = 0.0;
      for (int k = 0; k < m; ++k) tr += (double)M[k * m4 + k];
      const T delta = (T)(1e-7 * tr / m * pow(10.0, (double)(attempt - 1)));
      __syncthreads();
      for (int k = tid; k < m; k += NT) M[k * m4 + k] += delta;
      ridge = true;
    }
    ok = cholesky_cta_t<T>(M, m, m4);
  }
  if (!ok) {
    if (tid == 0 && status) atomicCAS(status, 0, 4);
    __syncthreads();
    return;
  }
  if (tall) {
    // per row: solve L y = a_i^T in place (thread per row), l_i = ||y||^2
    for (int i = tid; i < I; i += NT) {
      T *y = As + (size_t)i * lda;
      double s2 = 0.0;
      for (int k = 0; k < m; ++k) {
        T acc = y[k];
        for (int j = 0; j < k; ++j) acc = fma(-M[k * m4 + j], y[j], acc);
        acc = acc / M[k * m4 + k];
        y[k] = acc;
        s2 += (double)acc * (double)acc;
      }
      lev[i] = __ddiv_rn(s2, (double)m);
    }
  } else {
    for (int i = tid; i < I; i += NT) lev[i] = __ddiv_rn(1.0, (double)I);
  }
  __syncthreads();
  if (ridge) {   // ridge scores sum to less than the rank: normalise by their sum
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < I; ++i) tot = __dadd_rn(tot, lev[i]);
      wsc[0] = (unsigned long long)__double_as_longlong(tot);
    }
    __syncthreads();
    const double tot = __longlong_as_double((long long)wsc[0]);
    __syncthreads();
    for (int i = tid; i < I; i += NT) lev[i] = __ddiv_rn(lev[i], tot);
    __syncthreads();
  }
  write_cdf_cta(lev, I, prob, cdf, wsc);
}

}  // namespace trsgd
