// The scaled variant's Gram solve (Sec. 3.3): factorisation of the damped
// preconditioner h = Z_H^T D_H Z_H / (|H| J_n) + eta^t I and the triangular
// solves p = -g h^{-1}.  The scalar is double for FP64 cores and double-float
// (df64.cuh) for float cores; the gs_* overloads below hide the difference.
#pragma once

#include "df64.cuh"

namespace trsgd {

template <typename T> struct GramScalar { using type = df64; };
template <> struct GramScalar<double> { using type = double; };

__device__ __forceinline__ double gs_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double gs_fnms(double a, double b, double c) { return fma(-a, b, c); }   // c - a b
__device__ __forceinline__ double gs_div(double a, double b) { return a / b; }
__device__ __forceinline__ double gs_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double gs_add(double a, double b) { return a + b; }
__device__ __forceinline__ bool gs_pos(double a) { return a > 0.0 && isfinite(a); }
__device__ __forceinline__ double gs_to_double(double a) { return a; }
__device__ __forceinline__ void gs_from_double(double d, double &out) { out = d; }
__device__ __forceinline__ void gs_one(double &out) { out = 1.0; }
__device__ __forceinline__ double gs_shfl(double a, int src) { return __shfl_sync(0xffffffffu, a, src); }
__device__ __forceinline__ double gs_ldcg(const double *p) { return __ldcg(p); }

__device__ __forceinline__ df64 gs_mul(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 gs_fnms(df64 a, df64 b, df64 c) { return df_fnms_fast(a, b, c); }
__device__ __forceinline__ df64 gs_div(df64 a, df64 b) { return df_div(a, b); }
__device__ __forceinline__ df64 gs_sqrt(df64 a) { return df_sqrt(a); }
__device__ __forceinline__ df64 gs_add(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ bool gs_pos(df64 a) { return a.hi > 0.f && isfinite(a.hi); }
__device__ __forceinline__ double gs_to_double(df64 a) { return df_to_double(a); }
__device__ __forceinline__ void gs_from_double(double d, df64 &out) { out = df_from_double(d); }
__device__ __forceinline__ void gs_one(df64 &out) { out = df64{1.f, 0.f}; }
__device__ __forceinline__ df64 gs_shfl(df64 a, int src) {
  return df64{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}
__device__ __forceinline__ df64 gs_ldcg(const df64 *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return df64{v.x, v.y};
}

template <typename V> __device__ __forceinline__ V gs_zero() {
  V z;
  gs_from_double(0.0, z);
  return z;
}

// Cholesky factorisation of the damped Q x Q Gram matrix by one CTA, entries
// held in registers.  The lower triangle is cut into 4 x 4 blocks; thread t
// owns block t (and t + blockDim.x when NBS = 2) of the row-major packed
// block triangle.  A (symmetric, row-major, leading dim lda) is only read, so
// a failed attempt restarts from it with a larger `extra` on the diagonal.
//
// Square-root-free right-looking elimination: at pivot k the owners of
// column k publish it (unscaled) into one half of a double buffer, one
// barrier, then every entry with i >= j > k becomes a_ij - a_ik (a_jk / a_kk)
// (4 + 4 column values and 16 updates per thread).  The owner of a_{k+1,k+1}
// stores its reciprocal for the next pivot.  Afterwards L_ij = a_ij / sqrt(a_jj).
//
// Writes L column-major (out[j * Q + i], i >= j) and 1 / L_jj (out[Q * Q + j])
// to global memory; colbuf holds 2 * Q and pinv Q scalars of shared memory.
// Returns false at the first non-positive or non-finite pivot, the same
// decision in every thread, right after a barrier; returns true after a
// final barrier, so colbuf and pinv are free again in both cases.
// Needs (Q/4)(Q/4 + 1)/2 <= NBS * blockDim.x.
template <typename V, int NBS>
__device__ __noinline__ bool gram_factor_reg(const V *A, int Q, int lda, double extra, V *colbuf, V *pinv,
                                             V *out) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int Qb = (Q + 3) >> 2, nblk = Qb * (Qb + 1) / 2;
  V one, ex;
  gs_one(one);
  gs_from_double(extra, ex);
  int bi[NBS], bj[NBS];
  bool own[NBS];
  V a[NBS][4][4];
#pragma unroll
  for (int s = 0; s < NBS; ++s) {
    const int b = tid + s * NT;
    own[s] = b < nblk;
    int r = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while (r > 0 && r * (r + 1) / 2 > b) --r;
    while ((r + 1) * (r + 2) / 2 <= b) ++r;
    bi[s] = own[s] ? r : 0;
    bj[s] = own[s] ? b - r * (r + 1) / 2 : 0;
#pragma unroll
    for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * bi[s] + r4, j = 4 * bj[s] + u;
        a[s][r4][u] = gs_zero<V>();
        if (own[s] && j <= i && i < Q) {
          a[s][r4][u] = A[(size_t)i * lda + j];
          if (i == j) a[s][r4][u] = gs_add(a[s][r4][u], ex);
        }
      }
  }
  if (tid == 0) pinv[0] = gs_div(one, a[0][0][0]);
  for (int k = 0; k < Q; ++k) {
    const int kb = k >> 2, ku = k & 3;
    V *cb = colbuf + (k & 1) * Q;
#pragma unroll
    for (int s = 0; s < NBS; ++s)
      if (own[s] && bj[s] == kb)
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
          const int i = 4 * bi[s] + r4;
          V v = a[s][r4][0];
#pragma unroll
          for (int u = 1; u < 4; ++u)
            if (u == ku) v = a[s][r4][u];
          if (i >= k && i < Q) cb[i] = v;
        }
    __syncthreads();
    if (!gs_pos(cb[k])) {   // same value, same decision in every thread
      __syncthreads();
      return false;
    }
    const V invd = pinv[k];
#pragma unroll
    for (int s = 0; s < NBS; ++s) {
      if (!own[s] || 4 * bj[s] + 3 <= k) continue;   // no column right of k in this block
      V ci[4], tj[4];
#pragma unroll
      for (int r4 = 0; r4 < 4; ++r4) ci[r4] = cb[min(4 * bi[s] + r4, Q - 1)];
#pragma unroll
      for (int u = 0; u < 4; ++u) tj[u] = gs_mul(cb[min(4 * bj[s] + u, Q - 1)], invd);
#pragma unroll
      for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * bi[s] + r4, j = 4 * bj[s] + u;
          const V nv = gs_fnms(ci[r4], tj[u], a[s][r4][u]);
          if (j > k && j <= i && i < Q) a[s][r4][u] = nv;
        }
      const int k1 = k + 1;
      if (k1 < Q && bi[s] == (k1 >> 2) && bj[s] == (k1 >> 2)) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u == (k1 & 3)) pinv[k1] = gs_div(one, a[s][u][u]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NBS; ++s) {
    if (!own[s]) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * bj[s] + u;
      if (j >= Q) continue;
      const V rs = gs_sqrt(pinv[j]);   // 1 / sqrt(a_jj)
#pragma unroll
      for (int r4 = 0; r4 < 4; ++r4) {
        const int i = 4 * bi[s] + r4;
        if (j <= i && i < Q) out[(size_t)j * Q + i] = gs_mul(a[s][r4][u], rs);
      }
    }
  }
  for (int j = tid; j < Q; j += NT) out[(size_t)Q * Q + j] = gs_sqrt(pinv[j]);
  __syncthreads();   // colbuf and pinv may be reused by the caller
  return true;
}

}  // namespace trsgd
