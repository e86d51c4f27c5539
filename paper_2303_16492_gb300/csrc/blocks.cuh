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
// BYCORE: `idx` is indexed by core (idx[k]) instead of by factor.
template <int RMAX, typename T, bool BYCORE = false>
__device__ __forceinline__ void chain_row(const T *const *cores, const int *R, int N,
                                          const int *order, const int *idx, int L, int rp,
                                          T (&row)[RMAX]) {
  int k = order[0];
  int Ra = R[k], Rb = R[(k + 1) % N];
  const T *S = cores[k] + (size_t)idx[BYCORE ? k : 0] * Ra * Rb;
#pragma unroll
  for (int b = 0; b < RMAX; ++b) row[b] = (b < Rb) ? ld_l2(S + rp + (size_t)b * Ra) : T(0);
  for (int s = 1; s < L; ++s) {
    k = order[s];
    Ra = R[k];
    Rb = R[(k + 1) % N];
    S = cores[k] + (size_t)idx[BYCORE ? k : s] * Ra * Rb;
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

namespace trsgd {

// Load 4 consecutive elements (16-byte aligned for float, 32-byte for double).
template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = reinterpret_cast<const double2 *>(p)[0];
    const double2 y = reinterpret_cast<const double2 *>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

// Small shared-memory GEMM, C(m, n) = sum_{k < K4} A(m, k) B(k, n) * s_k, out of
// line so that its registers are not shared with the caller's live state.
//   A(m, k) = A[k*lda + m] (AKM) or A[m*lda + k];  B(k, n) = B[k*ldb + n] (BKN)
//   or B[n*ldb + k].  K4 = K rounded up to 4: rows/columns k in [K, K4) of
//   both operands must hold zeros.
// Warp tile: 4 rows m (warp-uniform, broadcast reads) x 32*TN columns n; lane
// l owns n = n0 + l + 32*b (BKN: contiguous per warp; n-major B: conflict-free
// 16-byte reads when ldb = 4 mod 32).  Every pointer/stride used with a
// 4-wide load is 4-element aligned.  epi(m, n, v) once per valid output.
// A, B and bscale (or null) point into dynamic shared memory.
template <int TN, bool AKM, bool BKN, typename T, typename Epi>
__device__ __noinline__ void gemm_s(int M, int N, int K, const T *__restrict__ A, int lda,
                                    const T *__restrict__ B, int ldb, const T *__restrict__ bscale,
                                    Epi epi) {
  A = smem_ptr(A);   // operands in dynamic shared memory
  B = smem_ptr(B);
  if (bscale) bscale = smem_ptr(bscale);
  constexpr int TM = 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int K4 = (K + 3) & ~3;
  const int tiles_m = (M + TM - 1) / TM;
  const int tiles_n = (N + 32 * TN - 1) / (32 * TN);
  for (int tile = warp; tile < tiles_m * tiles_n; tile += nwarps) {
    const int m0 = (tile / tiles_n) * TM;
    const int n0 = (tile % tiles_n) * (32 * TN) + lane;
    bool nv[TN];
#pragma unroll
    for (int b = 0; b < TN; ++b) nv[b] = (n0 + 32 * b) < N;
    int mr[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) mr[a] = min(m0 + a, M - 1);   // clamp: rows past M are discarded
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
    for (int k = 0; k < K4; k += 4) {
      T av[4][TM], bv[4][TN];   // [k offset][m or n]
      if constexpr (AKM) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          if (m0 + TM <= M) {
            T t4[4];
            ld4(A + (size_t)(k + kk) * lda + m0, t4);
#pragma unroll
            for (int a = 0; a < TM; ++a) av[kk][a] = t4[a];
          } else {
#pragma unroll
            for (int a = 0; a < TM; ++a) av[kk][a] = A[(size_t)(k + kk) * lda + mr[a]];
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          T t4[4];
          ld4(A + (size_t)mr[a] * lda + k, t4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) av[kk][a] = t4[kk];
        }
      }
      if constexpr (BKN) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[kk][b] = nv[b] ? B[(size_t)(k + kk) * ldb + n0 + 32 * b] : T(0);
      } else {
#pragma unroll
        for (int b = 0; b < TN; ++b) {
          T t4[4] = {T(0), T(0), T(0), T(0)};
          if (nv[b]) ld4(B + (size_t)(n0 + 32 * b) * ldb + k, t4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) bv[kk][b] = t4[kk];
        }
      }
      if (bscale) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const T sc = bscale[k + kk];
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[kk][b] *= sc;
        }
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[kk][a], bv[kk][b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b)
        if (m0 + a < M && nv[b]) epi(m0 + a, n0 + 32 * b, acc[a][b]);
  }
}

}  // namespace trsgd
