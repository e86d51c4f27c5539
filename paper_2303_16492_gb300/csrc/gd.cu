// Full-gradient iterations of the methods the paper compares against (Sec. 3):
// TR-GD, G_{n(2)} <- G_{n(2)} - alpha grad_n with the gradient of Eq. gradient,
//   grad_n = G_{n(2)} Gamma_n - M_n,   Gamma_n = Z^T Z,   M_n = X_[n] Z,
//   Z = G^{!=n}_{[2]} (J_n x R_n R_{n+1}),
// and TR-ScaledGD (Eq. scaled_gd), grad_n (Gamma_n + damping I)^{-1}.  Every
// core takes its step from the same iterate: M_n and Gamma_n of all modes are
// formed first, then the cores are updated.
//
// Per mode: gd_subchain_kernel writes Z row by row (the slice chain of each
// column j, i_{n+1} fastest, as the mode-major copy of X orders its fibers);
// gd_atz_kernel forms column-chunk partials of A^T Z over the J_n rows, with
// A the mode-major copy of X (M_n) or Z itself (Gamma_n); gd_reduce_kernel
// sums the partials in fixed chunk order (FP64), so the result does not
// depend on scheduling.  gd_factor_kernel factors Gamma_n + damping I in FP64
// (the damping grows as for the scaled step when the factorisation fails);
// gd_update_kernel updates one row of G_{n(2)} per warp.
#include "blocks.cuh"
#include "internal.h"
#include "tables.cuh"

#include <algorithm>

namespace trsgd {

namespace {

constexpr int kGdRMax = 16;
constexpr int kAtzThreads = 256, kAtzRows = 32;

// Z(j, r + r' R_n) = P_j(r', r), P_j = G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}),
// column j = i_{n+1} + I_{n+1} (i_{n+2} + ...); one thread per (j, r').
template <typename T>
__global__ void gd_subchain_kernel(GdArgs a, int n, T *Z) {
  const int N = a.N, L = N - 1, Rn = a.R[n], Rn1 = a.R[(n + 1) % N], Q = Rn * Rn1;
  const long long Jn = a.J[n];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Jn * Rn1) return;
  const long long j = e / Rn1;
  const int rp = (int)(e - j * Rn1);
  int order[kMaxOrder], idx[kMaxOrder];
  long long rest = j;
  for (int s = 0; s < kMaxOrder; ++s) {
    order[s] = 0;
    idx[s] = 0;
    if (s < L) {
      const int k = (n + 1 + s) % N;
      order[s] = k;
      idx[s] = (int)(rest % a.I[k]);
      rest /= a.I[k];
    }
  }
  const T *cores[kMaxOrder];
  for (int k = 0; k < kMaxOrder; ++k) cores[k] = static_cast<const T *>(a.cores[k]);
  T row[kGdRMax];
  chain_row<kGdRMax, T>(cores, a.R, N, order, idx, L, rp, row);
  T *zr = Z + (size_t)j * Q + (size_t)rp * Rn;
  for (int r = 0; r < kGdRMax; ++r)
    if (r < Rn) zr[r] = row[r];
}

// part[c][p][q] = sum over the rows j of chunk c of A[j][p] Z[j][q]
// (p < P, q < Q).  CTA (row block, chunk): 32 values of p and every q; each
// thread keeps 4 x ceil(Q/32) accumulators; A and Z rows staged 32 at a time.
template <typename T>
__global__ void __launch_bounds__(kAtzThreads) gd_atz_kernel(const T *A, long long lda, int P, const T *Z, int Q,
                                                              long long J, long long chunk, T *part) {
  constexpr int kAtzTile = sizeof(T) == 4 ? 32 : 16;   // rows of A and Z staged at a time
  __shared__ T As[kAtzTile][kAtzRows];
  __shared__ T Zs[kAtzTile][256];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int p0 = blockIdx.x * kAtzRows;
  const long long j0 = (long long)blockIdx.y * chunk, j1 = min(J, j0 + chunk);
  const int QM = (Q + 31) >> 5;
  T acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[u][m] = T(0);
  for (long long jt = j0; jt < j1; jt += kAtzTile) {
    const int tj = (int)min((long long)kAtzTile, j1 - jt);
    for (int e = tid; e < kAtzTile * kAtzRows; e += kAtzThreads) {
      const int jj = e / kAtzRows, pp = e - jj * kAtzRows;
      As[jj][pp] = (jj < tj && p0 + pp < P) ? A[(size_t)(jt + jj) * lda + p0 + pp] : T(0);
    }
    for (int e = tid; e < kAtzTile * Q; e += kAtzThreads) {
      const int jj = e / Q, q = e - jj * Q;
      Zs[jj][q] = jj < tj ? Z[(size_t)(jt + jj) * Q + q] : T(0);
    }
    __syncthreads();
    for (int jj = 0; jj < tj; ++jj) {
      T av[4], zv[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = As[jj][ty * 4 + u];
#pragma unroll
      for (int m = 0; m < 8; ++m) zv[m] = (m < QM && tx + 32 * m < Q) ? Zs[jj][tx + 32 * m] : T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[u][m] = fma(av[u], zv[m], acc[u][m]);
    }
    __syncthreads();
  }
  T *out = part + (size_t)blockIdx.y * P * Q;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty * 4 + u;
    if (p >= P) continue;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int q = tx + 32 * m;
      if (m < QM && q < Q) out[(size_t)p * Q + q] = acc[u][m];
    }
  }
}

// out[p][q] = sum_c part[c][p][q] in increasing c, accumulated in FP64
template <typename T, typename O>
__global__ void gd_reduce_kernel(const T *part, int nchunk, long long PQ, O *out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PQ) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += (double)part[(size_t)c * PQ + e];
  out[e] = (O)s;
}

// FP64 Cholesky of Gamma + damping I (Q <= 128) into fac (row-major, lower),
// the damping grown by 1e-12 tr/Q * 10^m, m = 0..6, on failure.
__global__ void gd_factor_kernel(const double *Gam, int Q, double damping, double *fac, int *status) {
  extern __shared__ double F[];
  const int tid = threadIdx.x, NT = blockDim.x;
  double tr = 0.0;
  for (int k = 0; k < Q; ++k) tr += Gam[(size_t)k * Q + k];
  bool ok = false;
  for (int m = -1; m < 7 && !ok; ++m) {
    const double d = damping + (m < 0 ? 0.0 : 1e-12 * tr / Q * pow(10.0, (double)m));
    for (int e = tid; e < Q * Q; e += NT) F[e] = Gam[e] + ((e / Q == e % Q) ? d : 0.0);
    ok = cholesky_cta_t<double>(F, Q, Q);
  }
  if (!ok) {
    if (tid == 0) latch_status(status, kStatusNumeric);
    return;
  }
  for (int e = tid; e < Q * Q; e += NT) fac[e] = F[e];
}

// One warp per row i of G_{n(2)}: g = G(i, :) Gamma - M(i, :); scaled: solve
// x (Gamma + damping I) = g with the factor (forward and backward sweeps);
// G(i, :) -= alpha x.  Lanes own the columns q = lane + 32 m.
template <typename T>
__global__ void gd_update_kernel(T *G, int In, int Q, const double *Gam, const T *M, const double *fac, int scaled,
                                 double alpha, int *status) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= In) return;
  T *row = G + (size_t)warp * Q;
  double g[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) g[m] = 0.0;
  for (int a = 0; a < Q; ++a) {
    const double ga = (double)row[a];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int q = lane + 32 * m;
      if (q < Q) g[m] = fma(ga, Gam[(size_t)a * Q + q], g[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int q = lane + 32 * m;
    if (q < Q) g[m] -= (double)M[(size_t)warp * Q + q];
  }
  if (scaled) {
    // x L L^T = g  <=>  L L^T x^T = g^T: forward L y = g, backward L^T x = y
    for (int k = 0; k < Q; ++k) {
      double yk = 0.0;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const double v = __shfl_sync(0xffffffffu, g[m], k & 31);
        if ((k >> 5) == m) yk = v;
      }
      yk /= fac[(size_t)k * Q + k];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int q = lane + 32 * m;
        if (q > k && q < Q) g[m] -= fac[(size_t)q * Q + k] * yk;
        if (q == k) g[m] = yk;
      }
    }
    for (int k = Q - 1; k >= 0; --k) {
      double xk = 0.0;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const double v = __shfl_sync(0xffffffffu, g[m], k & 31);
        if ((k >> 5) == m) xk = v;
      }
      xk /= fac[(size_t)k * Q + k];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int q = lane + 32 * m;
        if (q < k) g[m] -= fac[(size_t)k * Q + q] * xk;
        if (q == k) g[m] = xk;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int q = lane + 32 * m;
    if (q < Q) {
      const T nv = (T)((double)row[q] - alpha * g[m]);
      if (!isfinite((double)nv)) latch_status(status, kStatusNumeric);
      row[q] = nv;
    }
  }
}

template <typename T>
cudaError_t gd_iteration_t(const GdArgs &a, int scaled, double alpha, double damping, GdBuffers &b, int *status,
                           cudaStream_t s) {
  const int N = a.N;
  for (int n = 0; n < N; ++n) {
    const int Rn = a.R[n], Rn1 = a.R[(n + 1) % N], Q = Rn * Rn1, In = a.I[n];
    const long long Jn = a.J[n];
    T *Z = static_cast<T *>(b.Z);
    const long long nz = Jn * Rn1;
    gd_subchain_kernel<T><<<(unsigned)((nz + 255) / 256), 256, 0, s>>>(a, n, Z);
    // M_n = X_[n] Z = (mode-major copy)^T Z, then Gamma_n = Z^T Z
    for (int which = 0; which < 2; ++which) {
      const int P = which == 0 ? In : Q;
      const T *A = which == 0 ? static_cast<const T *>(a.xmode[n]) : Z;
      const long long lda = which == 0 ? a.ldx[n] : Q;
      const int rb = (P + kAtzRows - 1) / kAtzRows;
      int nchunk = (int)std::max(1LL, std::min((long long)std::max(1, 608 / rb), (Jn + 63) / 64));
      nchunk = std::min(nchunk, b.max_chunks);
      const long long chunk = (Jn + nchunk - 1) / nchunk;
      nchunk = (int)((Jn + chunk - 1) / chunk);
      gd_atz_kernel<T><<<dim3((unsigned)rb, (unsigned)nchunk), kAtzThreads, 0, s>>>(
          A, lda, P, Z, Q, Jn, chunk, static_cast<T *>(b.part));
      const long long PQ = (long long)P * Q;
      if (which == 0)
        gd_reduce_kernel<T, T><<<(unsigned)((PQ + 255) / 256), 256, 0, s>>>(
            static_cast<const T *>(b.part), nchunk, PQ, static_cast<T *>(b.M[n]));
      else
        gd_reduce_kernel<T, double><<<(unsigned)((PQ + 255) / 256), 256, 0, s>>>(
            static_cast<const T *>(b.part), nchunk, PQ, b.Gam[n]);
    }
  }
  for (int n = 0; n < N; ++n) {
    const int Q = a.R[n] * a.R[(n + 1) % N], In = a.I[n];
    if (scaled)
      gd_factor_kernel<<<1, 256, (size_t)Q * Q * sizeof(double), s>>>(b.Gam[n], Q, damping, b.fac, status);
    gd_update_kernel<T><<<(unsigned)((In + 7) / 8), 256, 0, s>>>(static_cast<T *>(a.cores[n]), In, Q, b.Gam[n],
                                                                  static_cast<const T *>(b.M[n]), b.fac, scaled,
                                                                  alpha, status);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t gd_prepare() {
  return cudaFuncSetAttribute(gd_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8);
}

cudaError_t launch_gd_iteration(int core_dtype, const GdArgs &a, int scaled, double alpha, double damping,
                                GdBuffers &b, int *status, cudaStream_t s) {
  return core_dtype == 0 ? gd_iteration_t<double>(a, scaled, alpha, damping, b, status, s)
                         : gd_iteration_t<float>(a, scaled, alpha, damping, b, status, s);
}

}  // namespace trsgd
