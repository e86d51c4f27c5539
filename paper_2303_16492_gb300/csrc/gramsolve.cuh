// The scaled variant's Gram solve (Sec. 3.3): factorisation of the damped
// preconditioner h = Z_H^T D_H Z_H / (|H| J_n) + eta^t I and the triangular
// solves p = -g h^{-1}.  The scalar is double for FP64 cores and double-float
// (df64.cuh) for float cores; the gs_* overloads below hide the difference.
#pragma once

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace trsgd {

template <typename T> struct GramScalar { using type = df64; };
template <> struct GramScalar<double> { using type = double; };

__device__ __forceinline__ double gs_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double gs_fnms(double a, double b, double c) { return fma(-a, b, c); }   // c - a b
__device__ __forceinline__ double gs_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ double gs_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double gs_add(double a, double b) { return a + b; }
__device__ __forceinline__ double gs_neg(double a) { return -a; }
__device__ __forceinline__ bool gs_pos(double a) { return a > 0.0 && isfinite(a); }
__device__ __forceinline__ double gs_to_double(double a) { return a; }
__device__ __forceinline__ void gs_from_double(double d, double &out) { out = d; }
__device__ __forceinline__ void gs_one(double &out) { out = 1.0; }
__device__ __forceinline__ double gs_ldcg(const double *p) { return __ldcg(p); }

__device__ __forceinline__ df64 gs_mul(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 gs_fnms(df64 a, df64 b, df64 c) { return df_fnms_fast(a, b, c); }
__device__ __forceinline__ df64 gs_rcp(df64 a) { return df_rcp(a); }
__device__ __forceinline__ df64 gs_sqrt(df64 a) { return df_sqrt(a); }
__device__ __forceinline__ df64 gs_add(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 gs_neg(df64 a) { return df_neg(a); }
__device__ __forceinline__ bool gs_pos(df64 a) { return a.hi > 0.f && isfinite(a.hi); }
__device__ __forceinline__ double gs_to_double(df64 a) { return df_to_double(a); }
__device__ __forceinline__ void gs_from_double(double d, df64 &out) { out = df_from_double(d); }
__device__ __forceinline__ void gs_one(df64 &out) { out = df64{1.f, 0.f}; }
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
// owns block t (and t + blockDim.x when NBS = 2) of the column-major packed
// block triangle, so that the blocks of a panel and those right of it are
// contiguous runs of threads (few, full warps).  A (symmetric, row-major, leading dim lda) is only read, so
// a failed attempt restarts from it with a larger `extra` on the diagonal.
//
// Square-root-free right-looking elimination, one block column (4 pivots)
// at a time: (1) the owner of the diagonal block eliminates it in registers
// (pivots d_u, 1/d_u and the multipliers l_{j,u} = a_{j,u} / d_u) and
// publishes them; (2) the owners of the blocks below it eliminate their rows
// against those multipliers and publish the results w_{i,u}; (3) every block
// right of the column takes the rank-4 update a_ij - sum_u w_iu (w_ju / d_u).
// Each entry sees the same operations in the same order as pivot-by-pivot
// elimination, with two barriers per 4 pivots; the published values are
// double-buffered by block-column parity, the rows w_i stored block-innermost
// (entry (r, v) of block row b at (4 r + v) ceil(Q/4) + b) so that a warp's
// consecutive blocks read consecutive words.  Afterwards L_ij = a_ij / sqrt(a_jj).
//
// Writes L column-major (out[j * Q + i], i >= j) and 1 / L_jj (out[Q * Q + j])
// to global memory; colbuf holds 32 ceil(Q/4) + 64 <= 8 Q + 96 and pinv Q
// scalars of shared memory.  Returns false at the first non-positive or non-finite pivot, the
// same decision in every thread, right after a barrier; returns true after a
// final barrier, so colbuf and pinv are free again in both cases.
// Needs (Q/4)(Q/4 + 1)/2 <= NBS * blockDim.x.
template <typename V, int NBS>
__device__ __noinline__ bool gram_factor_reg(const V *A, int Q, int lda, double extra, V *colbuf, V *pinv,
                                             V *out) {
  A = smem_ptr(A);
  colbuf = smem_ptr(colbuf);
  pinv = smem_ptr(pinv);
  const int tid = threadIdx.x, NT = blockDim.x;
  const int Qb = (Q + 3) >> 2, nblk = Qb * (Qb + 1) / 2;
  // a launch shape with too few threads for the block triangle would leave
  // diagonal blocks without an owner: fail (uniformly) instead of factoring
  // with stale pivots
  if (nblk > NBS * NT) return false;
  V one, ex;
  gs_one(one);
  gs_from_double(extra, ex);
  const V zero = gs_zero<V>();
  int bi[NBS], bj[NBS];
  bool own[NBS];
  V a[NBS][4][4];
#pragma unroll
  for (int s = 0; s < NBS; ++s) {
    const int b = tid + s * NT;
    own[s] = b < nblk;
    int c = 0, off = 0;   // block column c holds blocks off .. off + Qb - c - 1
    while (c < Qb && off + (Qb - c) <= b) off += Qb - c++;
    bi[s] = own[s] ? c + (b - off) : 0;
    bj[s] = own[s] ? c : 0;
#pragma unroll
    for (int r4 = 0; r4 < 4; ++r4)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * bi[s] + r4, j = 4 * bj[s] + u;
        a[s][r4][u] = zero;
        if (own[s] && j <= i && i < Q) {
          a[s][r4][u] = A[(size_t)i * lda + j];
          if (i == j) a[s][r4][u] = gs_add(a[s][r4][u], ex);
        }
      }
  }
  for (int kb = 0; kb < Qb; ++kb) {
    V *W = colbuf + (kb & 1) * 16 * Qb;               // w_{4b+r,v} at (4 r + v) Qb + b
    V *P = colbuf + 32 * Qb + (kb & 1) * 32;          // d[4], 1/d[4], l[j][u] at 8 + 4 j + u, flag at 24
    // (1) the diagonal block
#pragma unroll
    for (int s = 0; s < NBS; ++s) {
      if (!own[s] || bi[s] != kb || bj[s] != kb) continue;
      bool okb = true;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = 4 * kb + u;
        V inv = one, lj[4];
        if (k < Q) {
          const V d = a[s][u][u];
          if (!gs_pos(d)) okb = false;
          inv = gs_rcp(d);
          pinv[k] = inv;
          P[u] = d;
        } else {
          P[u] = one;
        }
        P[4 + u] = inv;
#pragma unroll
        for (int j = 0; j < 4; ++j) lj[j] = (j > u && k < Q) ? gs_mul(a[s][j][u], inv) : zero;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j > u && j <= i) a[s][i][j] = gs_fnms(a[s][i][u], lj[j], a[s][i][j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) P[8 + 4 * j + u] = lj[j];
      }
      P[24] = okb ? one : zero;
    }
    __syncthreads();
    if (!gs_pos(P[24])) {   // same value, same decision in every thread
      __syncthreads();
      return false;
    }
    // (2) the blocks below it: w_{i,u} = a_{i,u} - sum_{v<u} w_{i,v} l_{u,v}
#pragma unroll
    for (int s = 0; s < NBS; ++s) {
      if (!own[s] || bj[s] != kb || bi[s] <= kb) continue;
#pragma unroll
      for (int r4 = 0; r4 < 4; ++r4) {
#pragma unroll
        for (int u = 1; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < u; ++v) a[s][r4][u] = gs_fnms(a[s][r4][v], P[8 + 4 * u + v], a[s][r4][u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) W[(4 * r4 + u) * Qb + bi[s]] = a[s][r4][u];
      }
    }
    __syncthreads();
    // (3) the blocks right of it: rank-4 update with the published rows
#pragma unroll
    for (int s = 0; s < NBS; ++s) {
      if (!own[s] || bj[s] <= kb) continue;
      V tj[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) tj[u][v] = gs_mul(W[(4 * u + v) * Qb + bj[s]], P[4 + v]);
#pragma unroll
      for (int r4 = 0; r4 < 4; ++r4) {
        V wi[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) wi[v] = W[(4 * r4 + v) * Qb + bi[s]];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) a[s][r4][u] = gs_fnms(wi[v], tj[u][v], a[s][r4][u]);
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


// Inverse of the b-th diagonal block of L (a forward substitution per column,
// the columns independent): one warp, lane j computing column j,
//   X_jj = 1 / L_jj,  X_ij = -(1 / L_ii) sum_{j <= k < i} L_ik X_kj  (i > j),
// zero above the diagonal.  L is read column-major at pitch ldl (entry (q, k)
// at Lc[k ldl + q]) with 1 / L_qq at ivc[q]; block b's entry (i, j) goes to
// Dc[b kGsB (kGsB + 1) + j (kGsB + 1) + i] (odd pitch: a column and a row are
// both free of bank conflicts).  Each lane reads back only its own column.
template <typename V>
__device__ __noinline__ void gram_block_inverse(const V *Lc, int ldl, const V *ivc, int Q, int b, V *Dc) {
  const int j = threadIdx.x & 31, q0 = kGsB * b, nbk = min(kGsB, Q - q0);
  if (j >= nbk) return;
  Lc = smem_ptr(Lc);
  ivc = smem_ptr(ivc);
  Dc = smem_ptr(Dc);
  V *X = Dc + b * kGsB * (kGsB + 1) + j * (kGsB + 1);
  const V zero = gs_zero<V>();
  for (int i = 0; i < nbk; ++i) {
    const V *Li = Lc + q0 + i;   // L(q0 + i, q0 + k) at Li[(q0 + k) ldl]
    V a0 = zero, a1 = zero, a2 = zero, a3 = zero;   // - sum L_ik X_kj in four parts
    int k = j;
    for (; k + 3 < i; k += 4) {
      a0 = gs_fnms(Li[(q0 + k) * ldl], X[k], a0);
      a1 = gs_fnms(Li[(q0 + k + 1) * ldl], X[k + 1], a1);
      a2 = gs_fnms(Li[(q0 + k + 2) * ldl], X[k + 2], a2);
      a3 = gs_fnms(Li[(q0 + k + 3) * ldl], X[k + 3], a3);
    }
    for (; k < i; ++k) a0 = gs_fnms(Li[(q0 + k) * ldl], X[k], a0);
    const V s = gs_add(gs_add(a0, a1), gs_add(a2, a3));
    X[i] = i < j ? zero : (i == j ? ivc[q0 + i] : gs_mul(s, ivc[q0 + i]));
  }
}

// One warp solves h x = -g^T for one row g of the gradient, with h = L L^T
// factored by gram_factor_reg, block by block with the inverted diagonal
// blocks D_b^{-1} of gram_block_inverse:
//   forward   y_b = D_b^{-1} (-g_b - sum_{c<b} L_bc y_c),
//   backward  x_b = D_b^{-T} (y_b - sum_{c>b} L_cb^T x_c),
// lane l holding entry kGsB b + l of each block.  Every sum is a dot product
// with independent terms, so a sweep has nb sequential steps instead of Q.
// `row` (shared memory, Q entries) holds g on entry and x on return (x = 0
// when ok is false); buf is this warp's Q + kGsB entries of shared memory.
template <typename T, typename V>
__device__ __noinline__ void gram_solve_row(const V *Lc, int ldl, const V *Dc, int Q, bool ok, T *row, V *buf) {
  const int lane = threadIdx.x & 31, nb = (Q + kGsB - 1) / kGsB;
  const V zero = gs_zero<V>();
  Lc = smem_ptr(Lc);
  Dc = smem_ptr(Dc);
  row = smem_ptr(row);
  buf = smem_ptr(buf);
  V *ys = buf, *rs = buf + Q;
  if (!ok) {
    for (int q = lane; q < Q; q += 32) row[q] = T(0);
    return;
  }
  for (int b = 0; b < nb; ++b) {   // forward
    const int q0 = kGsB * b, nbk = min(kGsB, Q - q0), q = q0 + lane, qc = min(q, Q - 1);
    V a0, a1 = zero, a2 = zero, a3 = zero;
    gs_from_double(q < Q ? -(double)row[qc] : 0.0, a0);
    for (int k = 0; k < q0; k += 4) {   // q0 is a multiple of 4
      a0 = gs_fnms(Lc[k * ldl + qc], ys[k], a0);
      a1 = gs_fnms(Lc[(k + 1) * ldl + qc], ys[k + 1], a1);
      a2 = gs_fnms(Lc[(k + 2) * ldl + qc], ys[k + 2], a2);
      a3 = gs_fnms(Lc[(k + 3) * ldl + qc], ys[k + 3], a3);
    }
    rs[lane] = gs_add(gs_add(a0, a1), gs_add(a2, a3));
    __syncwarp();
    const V *Db = Dc + b * kGsB * (kGsB + 1);   // entry (i, j) at Db[j (kGsB + 1) + i]
    const int lc = min(lane, nbk - 1);
    a0 = a1 = a2 = a3 = zero;                     // - sum_j D(l, j) r_j
    int j = 0;
    for (; j + 3 < nbk; j += 4) {
      a0 = gs_fnms(Db[j * (kGsB + 1) + lc], rs[j], a0);
      a1 = gs_fnms(Db[(j + 1) * (kGsB + 1) + lc], rs[j + 1], a1);
      a2 = gs_fnms(Db[(j + 2) * (kGsB + 1) + lc], rs[j + 2], a2);
      a3 = gs_fnms(Db[(j + 3) * (kGsB + 1) + lc], rs[j + 3], a3);
    }
    for (; j < nbk; ++j) a0 = gs_fnms(Db[j * (kGsB + 1) + lc], rs[j], a0);
    const V y = gs_neg(gs_add(gs_add(a0, a1), gs_add(a2, a3)));
    __syncwarp();
    if (q < Q) ys[q] = y;
    __syncwarp();
  }
  for (int b = nb - 1; b >= 0; --b) {   // backward; ys[k] holds x_k for k beyond block b
    const int q0 = kGsB * b, nbk = min(kGsB, Q - q0), q = q0 + lane, qc = min(q, Q - 1);
    V a0 = q < Q ? ys[qc] : zero, a1 = zero, a2 = zero, a3 = zero;
    const V *Lr = Lc + (size_t)qc * ldl;        // L(k, q) at Lr[k]
    int k = q0 + nbk;
    for (; k + 3 < Q; k += 4) {
      a0 = gs_fnms(Lr[k], ys[k], a0);
      a1 = gs_fnms(Lr[k + 1], ys[k + 1], a1);
      a2 = gs_fnms(Lr[k + 2], ys[k + 2], a2);
      a3 = gs_fnms(Lr[k + 3], ys[k + 3], a3);
    }
    for (; k < Q; ++k) a0 = gs_fnms(Lr[k], ys[k], a0);
    rs[lane] = gs_add(gs_add(a0, a1), gs_add(a2, a3));
    __syncwarp();
    const V *Db = Dc + b * kGsB * (kGsB + 1) + min(lane, nbk - 1) * (kGsB + 1);   // D(j, l) at Db[j]
    a0 = a1 = a2 = a3 = zero;                     // - sum_j D(j, l) r_j
    int j = 0;
    for (; j + 3 < nbk; j += 4) {
      a0 = gs_fnms(Db[j], rs[j], a0);
      a1 = gs_fnms(Db[j + 1], rs[j + 1], a1);
      a2 = gs_fnms(Db[j + 2], rs[j + 2], a2);
      a3 = gs_fnms(Db[j + 3], rs[j + 3], a3);
    }
    for (; j < nbk; ++j) a0 = gs_fnms(Db[j], rs[j], a0);
    const V x = gs_neg(gs_add(gs_add(a0, a1), gs_add(a2, a3)));
    __syncwarp();
    if (q < Q) ys[q] = x;
    __syncwarp();
  }
  for (int q = lane; q < Q; q += 32) row[q] = (T)gs_to_double(ys[q]);
}

}  // namespace trsgd
