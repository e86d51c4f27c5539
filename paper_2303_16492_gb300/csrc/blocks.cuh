// Device building blocks shared by the step, reconstruction and error kernels.
#pragma once

#include "common.cuh"

namespace trsgd {

// C[m][n] = sum_k A[k*lda + m] * B[k*ldb + n] * (bscale ? bscale[k] : 1)
// over m < M, n < N, k < K, both operands k-major in shared memory.  Each
// warp owns TM consecutive rows m and 32*TN columns n (lane l owns columns
// n0 + l + 32*tn, so a warp's B reads are conflict-free and its A reads are
// broadcasts).  epi(m, n, value) is called once per valid output.
template <int TM, int TN, typename T, typename Epi>
__device__ __forceinline__ void gemm_tn(int M, int N, int K, const T *__restrict__ A, int lda,
                                        const T *__restrict__ B, int ldb,
                                        const double *__restrict__ bscale, Epi &&epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int tiles_m = (M + TM - 1) / TM;
  const int tiles_n = (N + 32 * TN - 1) / (32 * TN);
  for (int tile = warp; tile < tiles_m * tiles_n; tile += nwarps) {
    const int m0 = (tile / tiles_n) * TM;
    const int n0 = (tile % tiles_n) * (32 * TN) + lane;
    bool mv[TM], nv[TN];
#pragma unroll
    for (int a = 0; a < TM; ++a) mv[a] = (m0 + a) < M;
#pragma unroll
    for (int b = 0; b < TN; ++b) nv[b] = (n0 + 32 * b) < N;
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
    for (int k = 0; k < K; ++k) {
      T av[TM], bv[TN];
      const T *Ak = A + (size_t)k * lda + m0;
      const T *Bk = B + (size_t)k * ldb + n0;
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = mv[a] ? Ak[a] : T(0);
      const T s = bscale ? (T)bscale[k] : T(1);
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = nv[b] ? Bk[32 * b] * s : T(0);
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b)
        if (mv[a] && nv[b]) epi(m0 + a, n0 + 32 * b, acc[a][b]);
  }
}

// Row rp of the slice chain P = G_{k_0}(i_0) G_{k_1}(i_1) ... G_{k_{L-1}}(i_{L-1})
// (slices-Hadamard products of Algorithm 2 for one sample).  `order[s]` is the
// core of factor s, `idx[s]` its slice index.  Slice G_k(i) is column-major
// R_k x R_{k+1} at cores[k] + i*R_k*R_{k+1}.  On return row[0..R_{k_{L-1}+1})
// holds row rp of P (rp < R_{k_0}).  Core reads go through L2 only.
template <int RMAX, typename T>
__device__ __forceinline__ void chain_row(const T *const *cores, const int *R, int N,
                                          const int *order, const int *idx, int L, int rp,
                                          T (&row)[RMAX]) {
  int k = order[0];
  int Ra = R[k], Rb = R[(k + 1) % N];
  const T *S = cores[k] + (size_t)idx[0] * Ra * Rb;
#pragma unroll
  for (int b = 0; b < RMAX; ++b) row[b] = (b < Rb) ? ld_l2(S + rp + (size_t)b * Ra) : T(0);
  for (int s = 1; s < L; ++s) {
    k = order[s];
    Ra = R[k];
    Rb = R[(k + 1) % N];
    S = cores[k] + (size_t)idx[s] * Ra * Rb;
    T nrow[RMAX];
#pragma unroll
    for (int b = 0; b < RMAX; ++b) {
      T acc = T(0);
      if (b < Rb) {
#pragma unroll
        for (int a = 0; a < RMAX; ++a)
          if (a < Ra) acc = fma(row[a], ld_l2(S + a + (size_t)b * Ra), acc);
      }
      nrow[b] = acc;
    }
#pragma unroll
    for (int b = 0; b < RMAX; ++b) row[b] = nrow[b];
  }
}

}  // namespace trsgd
