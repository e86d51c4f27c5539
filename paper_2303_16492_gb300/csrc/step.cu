// Fused TR-BRSGD / TR-ScaledBRSGD step: one thread-block cluster per problem.
//
// One launch runs `nsteps` iterations t0 .. t0+nsteps-1 of every problem
// (Algorithm 3 with Algorithm 2).  The CTAs of a cluster split the |F|
// samples of each step; everything a step needs stays on chip:
//
//   A  draws (Philox, Algorithm 2), p_F, weights 1/(|F| J_n p_F), the fiber
//      gather by TMA bulk copies from the mode-major copy of X, and the
//      sampled subchain rows Z (slice chain, one thread per row of P_j).
//   S  (scaled variant) partial Gram Z^T D Z, reduced over the cluster in
//      FP64 into CTA 0, which factors h + eta^t I (Cholesky, FP64).
//   B  per chunk of G_n rows: residual E = G_n Z^T - X_S (Eq. S_gradient),
//      weighted in place over the fibers;
//   C  partial gradient E D Z of this CTA's samples;
//   R  cluster reduction of the partials through distributed shared memory
//      in a fixed CTA order (deterministic), then the step rule (fixed alpha
//      or AdaGrad) on the rows this CTA owns, written to G_n in HBM.
//   Scaled: p = -g h^{-1} per owned row by two FP64 triangular solves
//      against CTA 0's factor (Eq. scaledsg_direction, damped form).
//   Euclidean distribution: slice norms of the updated rows and CTA 0's
//      integer CDF of core n for the next iteration (Lemma euc_est).
//
// Cluster barriers (barrier.cluster, release/acquire) separate the phases;
// cores and distribution tables are read through L2 only because other CTAs
// of the cluster rewrite them between steps.  The only spin-wait (the TMA
// mbarrier) is bounded and latches TRSGD_ETIMEOUT.
#include "blocks.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace trsgd {

static constexpr long long kWaitLimit = 1LL << 22;
static constexpr int kMaxThreads = 512;

__host__ __device__ inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// In-place lower Cholesky of the Q x Q matrix A (leading dim ld) by one CTA;
// the strict upper triangle is left untouched.  Returns false at the first
// non-positive or non-finite pivot (the same decision in every thread).
template <typename Dummy = void>
__device__ bool cholesky_cta(double *A, int Q, int ld) {
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int k = 0; k < Q; ++k) {
    __syncthreads();
    const double d = A[k * ld + k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double l = sqrt(d);
    __syncthreads();
    if (tid == 0) A[k * ld + k] = l;
    for (int i = k + 1 + tid; i < Q; i += NT) A[i * ld + k] = A[i * ld + k] / l;
    __syncthreads();
    const int m = Q - k - 1;
    for (int e = tid; e < m * m; e += NT) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) A[i * ld + j] = fma(-A[i * ld + k], A[j * ld + k], A[i * ld + j]);
    }
  }
  __syncthreads();
  return true;
}

template <typename T, typename XT, int RMAX>
__global__ void __launch_bounds__(kMaxThreads)
    step_cluster_kernel(const ProbDesc *__restrict__ descs, StepLayout lay, long long t0, int nsteps) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = lay.C;
  const int c = (int)cluster.block_rank();
  const int pidx = blockIdx.x / C;
  const ProbDesc &D = descs[pidx];

  extern __shared__ __align__(128) unsigned char smem[];
  int *idx_s = reinterpret_cast<int *>(smem + lay.off_idx);
  long long *col_s = reinterpret_cast<long long *>(smem + lay.off_col);
  double *w_s = reinterpret_cast<double *>(smem + lay.off_w);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.off_bar);
  XT *xs = reinterpret_cast<XT *>(smem + lay.off_x);
  T *zs = reinterpret_cast<T *>(smem + lay.off_z);
  T *zt = reinterpret_cast<T *>(smem + lay.off_zt);
  T *reg = reinterpret_cast<T *>(smem + lay.off_reg);
  double *h64 = reinterpret_cast<double *>(smem + lay.off_h64);
  double *hdiag = reinterpret_cast<double *>(smem + lay.off_hdiag);
  T *gown = reinterpret_cast<T *>(smem + lay.off_gown);
  double *misc = reinterpret_cast<double *>(smem + lay.off_misc);

  const int tid = threadIdx.x, NT = blockDim.x;
  const int N = D.N, J = D.J;
  int I[kMaxOrder], R[kMaxOrder];
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) { I[k] = D.I[k]; R[k] = D.R[k]; }
  const T *cores_c[kMaxOrder];
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) cores_c[k] = static_cast<const T *>(D.cores[k]);
  const bool scaled = D.variant == 1;
  const bool rec = D.dbg && pidx == 0;
  const int ldq = lay.ldq;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;

  for (int s = 0; s < nsteps; ++s) {
    const long long t = t0 + s;
    const int n = draw_mode(D.seed, t, N);
    const int In = I[n], Rn = R[n], Rn1 = R[(n + 1) % N], Q = Rn * Rn1;
    const int L = N - 1;
    int order[kMaxOrder];
    double Jn = 1.0;
#pragma unroll
    for (int q = 0; q < kMaxOrder; ++q) order[q] = (q < L) ? (n + 1 + q) % N : 0;
    for (int k = 0; k < N; ++k)
      if (k != n) Jn *= (double)I[k];
    const int j0 = (int)((long long)J * c / C), j1 = (int)((long long)J * (c + 1) / C);
    const int jb = j1 - j0;
    T *Gn = static_cast<T *>(D.cores[n]);
    T *accn = static_cast<T *>(D.acc[n]);

    // ---- A1: slice indices (Algorithm 2) -----------------------------------
    for (int e = tid; e < jb * L; e += NT) {
      const int jl = e / L, sp = e % L, k = order[sp];
      const uint64_t u = draw_u64(D.seed, t, kStreamF, k, (uint32_t)(j0 + jl));
      int i;
      if (D.dist == 0) {
        i = (int)mulhi64(u, (uint64_t)I[k]);
      } else {
        const unsigned long long *cdf = D.cdf[k];
        const uint64_t W = __ldcg(cdf + I[k] - 1);
        i = cdf_search(cdf, I[k], mulhi64(u, W));
      }
      idx_s[jl * kMaxOrder + k] = i;
    }
    __syncthreads();

    // ---- A2: p_F (product in ring order), weights, fiber column -------------
    for (int jl = tid; jl < jb; jl += NT) {
      double pF = 1.0;
      long long col = 0, st = 1;
      for (int sp = 0; sp < L; ++sp) {
        const int k = order[sp], i = idx_s[jl * kMaxOrder + k];
        const double pk = (D.dist == 0) ? __ddiv_rn(1.0, (double)I[k]) : __ldcg(D.prob[k] + i);
        pF = __dmul_rn(pF, pk);
        col += (long long)i * st;
        st *= I[k];
      }
      w_s[jl] = __ddiv_rn(1.0, __dmul_rn(__dmul_rn((double)J, Jn), pF));
      col_s[jl] = col;
      if (rec) {
        D.dbg_pf[j0 + jl] = pF;
        for (int k = 0; k < N; ++k)
          D.dbg_idx[(size_t)(j0 + jl) * N + k] = (k == n) ? -1 : idx_s[jl * kMaxOrder + k];
      }
    }
    if (rec && c == 0 && tid == 0) *D.dbg_n = n;
    __syncthreads();

    // ---- A3: fiber gather, one TMA bulk copy per sample -------------------
    const uint32_t fbytes = (uint32_t)round_up((size_t)In * sizeof(XT), 16);
    if (tid == 0 && jb > 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, (uint32_t)jb * fbytes);
      const XT *base = static_cast<const XT *>(D.xmode[n]);
      const long long ldg = D.ldx[n];
      for (int jl = 0; jl < jb; ++jl)
        tma_load_1d(xs + (size_t)jl * lay.ldxs, base + col_s[jl] * ldg, fbytes, bar);
    }

    // ---- A4: sampled subchain rows, Z(j, r + r' R_n) = P_j(r', r) ----------
    for (int e = tid; e < jb * Rn1; e += NT) {
      const int jl = e / Rn1, rp = e % Rn1;
      int sidx[kMaxOrder];
#pragma unroll
      for (int q = 0; q < kMaxOrder; ++q) sidx[q] = (q < L) ? idx_s[jl * kMaxOrder + order[q]] : 0;
      T row[RMAX];
      chain_row<RMAX, T>(cores_c, R, N, order, sidx, L, rp, row);
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        if (r < Rn) {
          const int q = r + rp * Rn;
          zs[(size_t)jl * ldq + q] = row[r];
          zt[(size_t)q * lay.ldjb + jl] = row[r];
          if (rec) static_cast<T *>(D.dbg_z)[(size_t)(j0 + jl) * Q + q] = row[r];
        }
      }
    }
    if (jb > 0) {
      if (!mbar_wait_bounded(bar, phase, kWaitLimit)) {
        latch_status(D.status, kStatusTimeout);
        mbar_wait_bounded(bar, phase, kWaitLimit);
      }
      phase ^= 1u;
    }
    __syncthreads();

    // ---- S: preconditioner h = Z^T D Z / (|F| J_n) + eta^t I (FP64 solve) ---
    if (scaled) {
      const int QH = lay.QH;
      gemm_tn<8, 4, T>(Q, Q, jb, zs, ldq, zs, ldq, w_s,
                       [&](int a, int b, T v) { reg[(size_t)a * ldq + b] = v; });
      cluster.sync();
      double *h0 = cluster.map_shared_rank(h64, 0);
      double *hd0 = cluster.map_shared_rank(hdiag, 0);
      const int q0 = Q * c / C, q1 = Q * (c + 1) / C;
      for (int e = tid; e < (q1 - q0) * Q; e += NT) {
        const int a = q0 + e / Q, b = e % Q;
        double v = 0.0;
        for (int cc = 0; cc < C; ++cc) v += (double)cluster.map_shared_rank(reg, cc)[(size_t)a * ldq + b];
        if (a == b) {
          v += D.damping;
          hd0[a] = v;
        }
        h0[a * QH + b] = v;
        if (rec) D.dbg_h[a * Q + b] = v;
      }
      cluster.sync();
      if (c == 0) {
        // factor, growing the damping on failure (1e-12 tr(h)/Q * 10^m, m = 0..6)
        __shared__ double tr_s;
        if (tid == 0) {
          double tr = 0.0;
          for (int q = 0; q < Q; ++q) tr += hdiag[q] - D.damping;
          tr_s = tr;
        }
        __syncthreads();
        bool ok = cholesky_cta(h64, Q, QH);
        double extra = 0.0;
        for (int m = 0; m < 7 && !ok; ++m) {
          extra = 1e-12 * tr_s / Q * pow(10.0, (double)m);
          __syncthreads();
          for (int e = tid; e < Q * Q; e += NT) {
            const int a = e / Q, b = e % Q;
            if (a == b) h64[a * QH + a] = hdiag[a] + extra;
            else if (a > b) h64[a * QH + b] = h64[b * QH + a];
          }
          ok = cholesky_cta(h64, Q, QH);
        }
        if (tid == 0) {
          misc[0] = ok ? 1.0 : 0.0;
          if (!ok) latch_status(D.status, kStatusNumeric);
        }
        if (rec && ok && extra > 0.0)
          for (int q = tid; q < Q; q += NT) D.dbg_h[q * Q + q] = hdiag[q] + extra;
      }
    }

    // ---- B/C/R: per chunk of rows of G_n ------------------------------------
    int own_rows = 0;
    for (int i0 = 0; i0 < In; i0 += lay.TI) {
      const int ti = min(lay.TI, In - i0);
      for (int e = tid; e < ti * Q; e += NT) {
        const int ii = e / Q, q = e % Q;
        reg[(size_t)q * lay.ldti + ii] = ld_l2(Gn + (size_t)(i0 + ii) * Q + q);
      }
      __syncthreads();
      // residual, weighted in place: X_s <- w_j (G Z^T - X_S)
      gemm_tn<8, 4, T>(jb, ti, Q, zt, lay.ldjb, reg, lay.ldti, nullptr, [&](int jl, int ii, T v) {
        T *xp = reinterpret_cast<T *>(xs) + (size_t)jl * lay.ldxs + i0 + ii;
        const T e = v - *xp;
        if (rec) static_cast<T *>(D.dbg_e)[(size_t)(j0 + jl) * In + i0 + ii] = e;
        *xp = e * (T)w_s[jl];
      });
      __syncthreads();
      // partial gradient of this CTA's samples
      gemm_tn<8, 4, T>(ti, Q, jb, reinterpret_cast<T *>(xs) + i0, lay.ldxs, zs, ldq, nullptr,
                       [&](int ii, int q, T v) { reg[(size_t)ii * ldq + q] = v; });
      cluster.sync();
      const int r0 = ti * c / C, r1 = ti * (c + 1) / C;
      for (int e = tid; e < (r1 - r0) * Q; e += NT) {
        const int ii = r0 + e / Q, q = e % Q;
        T g = T(0);
        for (int cc = 0; cc < C; ++cc) g += cluster.map_shared_rank(reg, cc)[(size_t)ii * ldq + q];
        const size_t gi = (size_t)(i0 + ii) * Q + q;
        if (rec) static_cast<T *>(D.dbg_g)[gi] = g;
        if (scaled) {
          gown[(size_t)(own_rows + ii - r0) * ldq + q] = g;
        } else {
          const T p = -g;
          T delta;
          if (D.rule == 0) {
            delta = (T)D.alpha * p;
          } else {
            const T a = ld_l2(accn + gi) + p * p;
            accn[gi] = a;
            const double base = D.b + (double)a;
            const double sc = base > 0.0 ? (D.eps == 0.0 ? D.eta / sqrt(base)
                                                         : D.eta * pow(base, -(0.5 + D.eps)))
                                         : 0.0;
            delta = (T)sc * p;
          }
          const T nv = ld_l2(Gn + gi) + delta;
          if (!isfinite((double)nv)) latch_status(D.status, kStatusNumeric);
          Gn[gi] = nv;
          if (rec) static_cast<T *>(D.dbg_p)[gi] = p;
        }
      }
      if (!scaled && D.dist == 2) {
        __syncthreads();
        for (int ii = r0 + tid; ii < r1; ii += NT) {
          const T *row = Gn + (size_t)(i0 + ii) * Q;
          double sn = 0.0;
          for (int q = 0; q < Q; ++q) {
            const double v = (double)ld_l2(row + q);
            sn = __dadd_rn(sn, __dmul_rn(v, v));
          }
          D.snorm[n][i0 + ii] = sn;
        }
      }
      own_rows += r1 - r0;
      cluster.sync();
    }

    // ---- scaled direction p = -g h^{-1} on the owned rows, then the update --
    if (scaled) {
      const int QH = lay.QH;
      const double *L0 = cluster.map_shared_rank(h64, 0);
      const bool ok = *cluster.map_shared_rank(misc, 0) != 0.0;
      const int warp = tid >> 5, lane = tid & 31, nw = NT >> 5;
      const int r0 = In * c / C;   // single chunk: owned rows [r0, r0 + own_rows)
      constexpr int QM = 4;        // Q <= 128 = 32 * QM
      for (int rr = warp; rr < own_rows; rr += nw) {
        const int i = r0 + rr;
        double y[QM];
#pragma unroll
        for (int m = 0; m < QM; ++m) {
          const int q = lane + 32 * m;
          y[m] = (q < Q) ? -(double)gown[(size_t)rr * ldq + q] : 0.0;
        }
        if (ok) {
          for (int k = 0; k < Q; ++k) {        // L y = -g^T
            double yk = 0.0;
#pragma unroll
            for (int m = 0; m < QM; ++m)
              if ((k >> 5) == m && lane == (k & 31)) yk = y[m] / L0[k * QH + k];
            yk = __shfl_sync(0xffffffffu, yk, k & 31);
#pragma unroll
            for (int m = 0; m < QM; ++m) {
              const int q = lane + 32 * m;
              if (q == k) y[m] = yk;
              else if (q > k && q < Q) y[m] = fma(-L0[q * QH + k], yk, y[m]);
            }
          }
          for (int k = Q - 1; k >= 0; --k) {   // L^T x = y
            double xk = 0.0;
#pragma unroll
            for (int m = 0; m < QM; ++m)
              if ((k >> 5) == m && lane == (k & 31)) xk = y[m] / L0[k * QH + k];
            xk = __shfl_sync(0xffffffffu, xk, k & 31);
#pragma unroll
            for (int m = 0; m < QM; ++m) {
              const int q = lane + 32 * m;
              if (q == k) y[m] = xk;
              else if (q < k) y[m] = fma(-L0[k * QH + q], xk, y[m]);
            }
          }
        } else {
#pragma unroll
          for (int m = 0; m < QM; ++m) y[m] = 0.0;
        }
#pragma unroll
        for (int m = 0; m < QM; ++m) {
          const int q = lane + 32 * m;
          if (q >= Q) continue;
          const size_t gi = (size_t)i * Q + q;
          const T p = (T)y[m];
          T delta;
          if (D.rule == 0) {
            delta = (T)D.alpha * p;
          } else {
            const T a = ld_l2(accn + gi) + p * p;
            accn[gi] = a;
            const double base = D.b + (double)a;
            const double sc = base > 0.0 ? (D.eps == 0.0 ? D.eta / sqrt(base)
                                                         : D.eta * pow(base, -(0.5 + D.eps)))
                                         : 0.0;
            delta = (T)sc * p;
          }
          const T nv = ld_l2(Gn + gi) + delta;
          if (!isfinite((double)nv)) latch_status(D.status, kStatusNumeric);
          Gn[gi] = nv;
          if (rec) static_cast<T *>(D.dbg_p)[gi] = p;
        }
      }
      if (D.dist == 2) {
        __syncthreads();
        for (int rr = tid; rr < own_rows; rr += NT) {
          const T *row = Gn + (size_t)(r0 + rr) * Q;
          double sn = 0.0;
          for (int q = 0; q < Q; ++q) {
            const double v = (double)ld_l2(row + q);
            sn = __dadd_rn(sn, __dmul_rn(v, v));
          }
          D.snorm[n][r0 + rr] = sn;
        }
      }
      cluster.sync();
    }

    // ---- Euclidean table of core n for the next iteration (CTA 0) ---------
    if (D.dist == 2) {
      if (c == 0) {
        const double *sn = D.snorm[n];
        if (tid == 0) {
          double tot = 0.0;
          for (int i = 0; i < In; ++i) tot = __dadd_rn(tot, __ldcg(sn + i));
          misc[1] = tot;
          if (!(tot > 0.0)) latch_status(D.status, kStatusNumeric);
        }
        __syncthreads();
        const double tot = misc[1];
        unsigned long long *cdf = D.cdf[n];
        for (int i = tid; i < In; i += NT) {
          const double p = __ddiv_rn(__ldcg(sn + i), tot);
          D.prob[n][i] = p;
          cdf[i] = __double2ull_rn(__dmul_rn(p, 4503599627370496.0));  // * 2^52, exact
        }
        __syncthreads();
        if (tid == 0) {
          unsigned long long run = 0;
          for (int i = 0; i < In; ++i) {
            run += __ldcg(cdf + i);
            cdf[i] = run;
          }
        }
      }
      cluster.sync();
    }
  }
}

template <typename T, typename XT, int RMAX>
static cudaError_t prepare_one(const StepLayout &lay) {
  auto k = step_cluster_kernel<T, XT, RMAX>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename T, typename XT, int RMAX>
static cudaError_t launch_one(const ProbDesc *descs, int nprob, const StepLayout &lay, int threads,
                              long long t0, int nsteps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(lay.C * nprob), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = lay.total;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)lay.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_cluster_kernel<T, XT, RMAX>, descs, lay, t0, nsteps);
}

#define TRSGD_DISPATCH(FN, ...)                                                        \
  do {                                                                                 \
    if (core_dtype == 0) {                                                             \
      if (rmax <= 4) return FN<double, double, 4>(__VA_ARGS__);                        \
      if (rmax <= 8) return FN<double, double, 8>(__VA_ARGS__);                        \
      return FN<double, double, 16>(__VA_ARGS__);                                      \
    } else {                                                                           \
      if (rmax <= 4) return FN<float, float, 4>(__VA_ARGS__);                          \
      if (rmax <= 8) return FN<float, float, 8>(__VA_ARGS__);                          \
      return FN<float, float, 16>(__VA_ARGS__);                                        \
    }                                                                                  \
  } while (0)

cudaError_t step_kernel_prepare(int core_dtype, int x_dtype, int rmax, const StepLayout &lay) {
  (void)x_dtype;
  TRSGD_DISPATCH(prepare_one, lay);
}

cudaError_t launch_step(int core_dtype, int x_dtype, int rmax, const ProbDesc *descs, int nprob,
                        const StepLayout &lay, int threads, long long t0, int nsteps,
                        cudaStream_t s) {
  (void)x_dtype;
  TRSGD_DISPATCH(launch_one, descs, nprob, lay, threads, t0, nsteps, s);
}

int step_max_smem() { return 232448; }

}  // namespace trsgd
