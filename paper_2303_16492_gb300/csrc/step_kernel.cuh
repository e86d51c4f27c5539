// Fused TR-BRSGD / TR-ScaledBRSGD step: one thread-block cluster per problem.
//
// One launch runs `nsteps` iterations t0 .. t0+nsteps-1 of every problem
// (Algorithm 3 with Algorithm 2).  The CTAs of a cluster split the |F|
// samples of each step; everything a step needs stays on chip:
//
//   A1 slice indices (Philox, Algorithm 2) of this CTA's samples, one thread
//      per (sample, factor) for uniform sampling and for the leverage /
//      Euclidean tables staged in shared memory;
//   A2 p_F (product in ring order), weights 1/(|F| J_n p_F), fiber columns;
//   A3 the mode-n fibers of X from its mode-major copy, by 16-byte
//      asynchronous copies (fibers of 1 KB or more: TMA bulk copies completing
//      on an mbarrier), waited for after A4;
//   A4 per group of samples whose slices fit: the sampled slices G_k(i_k)
//      staged in shared memory (one cp.async group per factor), then the
//      sampled subchain rows Z(j, r + r' R_n) = P_j(r', r),
//      P_j = G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}), factor by factor;
//   S  (scaled variant) partial Gram Z^T D Z, reduced over the cluster into
//      CTA 0, which factors h + eta^t I (blocked square-root-free Cholesky
//      in the Gram-solve scalar: FP64, or double-float for float cores;
//      damping grown on failure) and writes the factor to global memory.  In
//      the scaled variant CTA 0 takes no samples, so the factorisation
//      overlaps the other CTAs' B and C;
//   B  per chunk of G_n rows: residual E = G_n Z^T - X_S (Eq. S_gradient),
//      weighted by 1/(|F| J_n p_F);
//   C  partial gradient (E D) Z of this CTA's samples.  B and C run on the
//      tensor cores (tcgen05, accumulators in TMEM) with every operand held
//      as BF16 pieces (three for FP32, two for BF16-mixed), else on the FMA
//      units;
//   R  reduction of the partials over the cluster through distributed shared
//      memory, each element summed in a fixed order (owner c pulls CTAs
//      c+1, c+2, ... mod C: deterministic), then the step rule (fixed alpha
//      or AdaGrad) on the rows this CTA owns, written to G_n in HBM;
//   scaled: p = -g h^{-1} on the owned rows by two blocked triangular solves
//      against CTA 0's factor, whose 32 x 32 diagonal blocks every CTA
//      inverts first (Eq. scaledsg_direction, damped form);
//   Euclidean / leverage distribution: CTA 0 rebuilds the table of core n for
//      the next iteration (Lemma euc_est, Lemma lev_est).
//
// With uniform sampling the draws of iteration t+1 depend on no core: once
// the last chunk of iteration t has consumed the fibers, the upper half of
// each CTA issues A1-A3 of t+1 (named barrier 1) while the lower half
// reduces and updates; both meet at the closing cluster barrier.
//
// The template argument SC compiles the scaled variant in; launches without
// a scaled problem use the instantiation without it (fewer registers).
//
// Cluster barriers (barrier.cluster, release/acquire) separate the phases.
// Cores and sampling tables are read through L2 only (ld.global.cg /
// cp.async.cg) because other CTAs of the cluster rewrite them between steps.
// The spin-waits (the fiber TMA and the MMA completion mbarriers) are
// bounded and latch TRSGD_ETIMEOUT.
#pragma once

#include "blocks.cuh"
#include "internal.h"
#include "tables.cuh"
#include "df64.cuh"
#include "gramsolve.cuh"

#include <type_traits>

namespace cg = cooperative_groups;

namespace trsgd {

static constexpr long long kWaitLimit = 1LL << 22;
static constexpr int kMaxThreads = 512;
static constexpr uint32_t kTmaFiberBytes = 1024;   // fibers at least this long go through TMA

__host__ __device__ inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Eight consecutive values as P BF16 pieces, 8 per 16 bytes: piece k is the
// BF16 rounding (to nearest) of what pieces 0..k-1 left, so that the pieces
// sum to the value up to the last piece's rounding (P = 3: 24 significant bits).
template <int P, int PA>
__device__ __forceinline__ void bf16_split8(const float (&v)[8], uint4 (&w)[PA]) {
  uint32_t u[PA][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float a = v[2 * j], b = v[2 * j + 1];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      const float2 hf = __bfloat1622float2(h);
      a -= hf.x;
      b -= hf.y;
      u[k][j] = *reinterpret_cast<const uint32_t *>(&h);
    }
  }
#pragma unroll
  for (int k = 0; k < P; ++k) w[k] = make_uint4(u[k][0], u[k][1], u[k][2], u[k][3]);
}

// The same split for four consecutive values (8 bytes per piece) and for one
// value (2 bytes per piece).
template <int P>
__device__ __forceinline__ void bf16_split4(const float (&v)[4], uint2 (&w)[P]) {
  uint32_t u[P][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float a = v[2 * j], b = v[2 * j + 1];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      const float2 hf = __bfloat1622float2(h);
      a -= hf.x;
      b -= hf.y;
      u[k][j] = *reinterpret_cast<const uint32_t *>(&h);
    }
  }
#pragma unroll
  for (int k = 0; k < P; ++k) w[k] = make_uint2(u[k][0], u[k][1]);
}
template <int P>
__device__ __forceinline__ void bf16_split1(float a, __nv_bfloat16 (&w)[P]) {
#pragma unroll
  for (int k = 0; k < P; ++k) {
    w[k] = __float2bfloat16_rn(a);
    a -= __bfloat162float(w[k]);
  }
}

// Commit this thread's outstanding cp.async copies as one group; wait until at
// most n of its most recent groups are still in flight (n >= 6: 6).
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
  }
}

// Split cluster barrier (all threads of every CTA arrive once, then wait once).
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Smallest i in [0, n) with target < cdf[i], cdf in shared memory (the same
// search as cdf_search on the global table).
__device__ __forceinline__ int cdf_search_smem(const unsigned long long *cdf, int n, uint64_t target) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

// sum_{a < LEN} p[a * PS] * s[a] with compile-time length and stride
template <int LEN, int PS, typename T>
__device__ __forceinline__ T dotk(const T *p, const T *s) {
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < LEN; ++a) acc = fma(p[a * PS], s[a], acc);
  return acc;
}

// One factor of the batched slice chain for a uniform (even) rank RU:
// P_{q+1} = P_q S_q per sample, written row-major [r'][b]; the first P is the
// staged slice itself (column-major).  A group of RU / CB lanes per sample:
// lane bb owns the CB output columns bb*CB .., whose entries of S_q stay in
// registers, so every loaded value of P_q serves CB outputs and a warp covers
// 32 / (RU / CB) samples.  Each output is a dot product of a row of P_q (read
// with stride RU when P_q is the column-major staged slice, FIRST) with a
// column of S_q, summed a = 0 .. RU-1 in order with fused multiply-adds.
// src, sfac and dst point into dynamic shared memory.
template <int RU, int CB, bool FIRST, typename T>
__device__ __noinline__ void chain_factor_uniform(const T *src, int sstride, const T *sfac, int qpad, T *dst,
                                                  int dstride, int jb) {
  static_assert(RU % 2 == 0 && RU % CB == 0, "even rank, whole lane groups");
  constexpr int LPS = RU / CB, G = 32 / LPS;
  src = smem_ptr(src);   // all three in dynamic shared memory
  sfac = smem_ptr(sfac);
  dst = smem_ptr(dst);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int g = lane / LPS, bb = lane - g * LPS;
  const bool lane_ok = g < G;
  const int b0 = (lane_ok ? bb : 0) * CB;
  for (int j0 = warp * G; j0 < jb; j0 += nwarps * G) {
    const int jl = j0 + g;
    const bool ok = lane_ok && jl < jb;
    const int jc = ok ? jl : 0;
    const T *P = src + (size_t)jc * sstride;
    const T *S = sfac + (size_t)jc * qpad;   // column-major RU x RU
    T col[CB][RU];
#pragma unroll
    for (int c = 0; c < CB; ++c)
#pragma unroll
      for (int a = 0; a < RU; ++a) col[c][a] = S[(b0 + c) * RU + a];
    T *Dp = dst + (size_t)jc * dstride + b0;
    if constexpr (FIRST) {
#pragma unroll 2
      for (int r = 0; r < RU; ++r) {
        T pr[RU];   // row r of the column-major P_q (stride RU)
#pragma unroll
        for (int a = 0; a < RU; ++a) pr[a] = P[r + a * RU];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          T acc = T(0);
#pragma unroll
          for (int a = 0; a < RU; ++a) acc = fma(pr[a], col[c][a], acc);
          if (ok) Dp[r * RU + c] = acc;
        }
      }
    } else {
#pragma unroll 2
      for (int r = 0; r < RU; ++r) {
        T pr[RU];   // row r of P_q
        if constexpr (sizeof(T) == 4) {
          const float2 *p2 = reinterpret_cast<const float2 *>(P + r * RU);
#pragma unroll
          for (int a2 = 0; a2 < RU / 2; ++a2) {
            const float2 v = p2[a2];
            pr[2 * a2] = v.x;
            pr[2 * a2 + 1] = v.y;
          }
        } else {
#pragma unroll
          for (int a = 0; a < RU; ++a) pr[a] = P[r * RU + a];
        }
        T acc[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          acc[c] = T(0);
#pragma unroll
          for (int a = 0; a < RU; ++a) acc[c] = fma(pr[a], col[c][a], acc[c]);
        }
        if (ok) {
#pragma unroll
          for (int c = 0; c < CB; ++c) Dp[r * RU + c] = acc[c];
        }
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T step_delta(int rule, T alpha, T eta, T b, double eps, T *accn, size_t gi, T p) {
  if (rule == 0) return alpha * p;
  const T a = ld_l2(accn + gi) + p * p;
  accn[gi] = a;
  const T base = b + a;
  if (!(base > T(0))) return T(0);
  const T sc = (eps == 0.0) ? eta / sqrt(base) : eta * pow(base, (T)(-(0.5 + eps)));
  return sc * p;
}

template <typename T, typename XT, int RMAX, int NPC, bool SC>
__global__ void __launch_bounds__(kMaxThreads)
    step_cluster_kernel(const ProbDesc *__restrict__ descs, StepLayout lay, long long t0, int nsteps,
                        const long long *__restrict__ t_dev) {
  if (t_dev) t0 += __ldcg(t_dev);   // device-resident iteration counter (graph replays)
  cg::cluster_group cluster = cg::this_cluster();
  const int C = lay.C;
  const int c = (int)cluster.block_rank();
  const int pidx = blockIdx.x / C;

  extern __shared__ __align__(128) unsigned char smem[];
  ProbDesc *desc_s = reinterpret_cast<ProbDesc *>(smem + lay.off_desc);
  int *idx_s = reinterpret_cast<int *>(smem + lay.off_idx);
  long long *col_s = reinterpret_cast<long long *>(smem + lay.off_col);
  T *wt_s = reinterpret_cast<T *>(smem + lay.off_wt);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.off_bar);
  XT *xs = reinterpret_cast<XT *>(smem + lay.off_x);
  T *zs = reinterpret_cast<T *>(smem + lay.off_z);
  T *reg = reinterpret_cast<T *>(smem + lay.off_reg);
  double *h64 = reinterpret_cast<double *>(smem + lay.off_h64);
  double *hdiag = reinterpret_cast<double *>(smem + lay.off_hdiag);
  T *gown = reinterpret_cast<T *>(smem + lay.off_gown);
  double *misc = reinterpret_cast<double *>(smem + lay.off_misc);
  double *cst = reinterpret_cast<double *>(smem + lay.off_const);   // [0,8): 1/I_k, [8,16): |F| J_n
  T *sb = reinterpret_cast<T *>(smem + lay.off_sb);                 // staged slices (aliases the tail)
  // per step: ring order of the chain factors, staged-slice offsets and pitches
  int *order = reinterpret_cast<int *>(smem + lay.off_ord);
  int *soff = order + kMaxOrder, *qpad = order + 2 * kMaxOrder;

  const int tid = threadIdx.x, NT = blockDim.x;
  {   // the problem descriptor, once per launch
    const int *src = reinterpret_cast<const int *>(descs + pidx);
    int *dst = reinterpret_cast<int *>(desc_s);
    for (int i = tid; i < (int)(sizeof(ProbDesc) / 4); i += NT) dst[i] = src[i];
  }
  // NPC > 0: the two contractions on the tensor cores with every operand held
  // as NPC BF16 pieces (2: BF16-mixed fibers; 3: FP32 accuracy); 0: FMA units
  constexpr bool kTC = NPC > 0;
  static_assert(NPC == 0 || (NPC == 2 && std::is_same<XT, __nv_bfloat16>::value) ||
                    (NPC == 3 && std::is_same<XT, float>::value && std::is_same<T, float>::value),
                "piece count and fiber type do not match");
  constexpr int EWP = NPC == 3 ? 3 : 1;   // pieces of the weighted residual
  constexpr bool kDF = std::is_same<T, float>::value;             // Gram solve in double-float
  uint64_t *bar_mma = bar + 1;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(misc + 6);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar + 2, 1);
    fence_mbar_init();
  }
  if constexpr (kTC) {
    if (tid < 32) tmem_alloc(tslot, 512);
    tc_fence_before();
  }
  __syncthreads();
  if constexpr (kTC) tc_fence_after();
  const uint32_t tbase = kTC ? *tslot : 0u;
  uint32_t mphase = 0;
  const ProbDesc &D = *desc_s;
  const int N = D.N, J = D.J;
  // dims and ranks read from the shared descriptor: small per-thread arrays
  // indexed at run time would live in local memory (L2 round trips)
  const int *I = D.I, *R = D.R;
  const bool scaled = SC && D.variant == 1;   // SC false: the scaled variant is compiled out
  const bool rec = D.dbg && pidx == 0;
  // first try of every bounded wait; a timeout is latched, then the operation
  // is drained by a second wait of the default length
  const long long wlim = D.wait_limit == 0 ? kWaitLimit : (D.wait_limit < 0 ? 0 : D.wait_limit);
  int ru = R[0];   // the common rank when all ranks are equal, else 0
  for (int k = 1; k < N; ++k)
    if (R[k] != ru) ru = 0;
  const int ldq = lay.ldq;
  const T alpha_t = (T)D.alpha, eta_t = (T)D.eta, b_t = (T)D.b;
  if (tid < N) {   // FP64 constants, once per launch (FP64 throughput is scarce)
    cst[tid] = __ddiv_rn(1.0, (double)I[tid]);
    double jn = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != tid) jn = __dmul_rn(jn, (double)I[k]);
    cst[8 + tid] = __dmul_rn((double)J, jn);
    cst[24 + tid] = __dmul_rn((double)D.JH, jn);   // |H| J_n
  }
  if (tid == 0) cst[16] = __ddiv_rn(1.0, (double)J);
  __syncthreads();
  const T wt_uni = (T)cst[16];
  uint32_t phase = 0;

  // Plain variant on the tensor cores: every core is kept in global memory as
  // its NPC BF16 pieces, in the residual's operand tile layout (per chunk of
  // 128 rows and per piece one K-major 128 x qp tile), so that a chunk's G_n
  // operand arrives by bulk copies instead of being converted every step.  The
  // pieces are rebuilt here, at the start of every launch (the cores may have
  // changed between launches), and the owners of the updated rows rewrite
  // theirs with the update.
  const bool gbulk = kTC && !scaled && D.gpc[0] != nullptr;
  uint64_t *bar_g = bar + 2;
  uint32_t gphase = 0;
  const size_t gcs = (size_t)lay.qp * 256;   // bytes of one piece of one chunk (128 x qp BF16)
  if constexpr (kTC) {
    if (gbulk) {
      const int QC = lay.qp / 8;
      for (int k = 0; k < N; ++k) {
        const int Qk = R[k] * R[(k + 1) % N], Ik = I[k];
        const float *G = static_cast<const float *>(D.cores[k]);
        unsigned char *dst = static_cast<unsigned char *>(D.gpc[k]);
        // 8 consecutive threads: the 8 rows of one 128-byte core matrix
        for (int e = c * NT + tid; e < ((Ik + 7) & ~7) * QC; e += C * NT) {
          const int rest = e >> 3, qb = rest % QC, i = (rest / QC) * 8 + (e & 7);
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int q = qb * 8 + j;
            v[j] = (i < Ik && q < Qk) ? __ldcg(G + (size_t)i * Qk + q) : 0.f;
          }
          uint4 w[NPC > 0 ? NPC : 1];
          bf16_split8<NPC>(v, w);
          unsigned char *o = dst + (size_t)(i >> 7) * NPC * gcs + kmaj_off(i & 127, qb * 8, QC);
#pragma unroll
          for (int p = 0; p < NPC; ++p) *reinterpret_cast<uint4 *>(o + p * gcs) = w[p];
        }
      }
      fence_proxy_async_global();
      cluster.sync();
    }
  }

  // sum of one element of a shared-memory buffer over the cluster's CTAs in
  // fixed CTA order 0..C-1 (deterministic); the C remote loads are issued together
  auto cluster_sum = [&](T *local, size_t off) -> T {
    T v[16];
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) v[cc] = (cc < C) ? cluster.map_shared_rank(local, cc)[off] : T(0);
    T g = T(0);
#pragma unroll
    for (int cc = 0; cc < 16; ++cc)
      if (cc < C) g += v[cc];
    return g;
  };

  // samples of this CTA (the same every iteration): CTAs cw0..C-1 share the J
  // samples (with cw0 = 1 CTA 0 factorises the scaled variant's Gram matrix
  // while the others work on them)
  const int cr = c - lay.cw0, CWk = C - lay.cw0;
  const int j0 = cr < 0 ? 0 : (int)((long long)J * cr / CWk), j1 = cr < 0 ? 0 : (int)((long long)J * (cr + 1) / CWk);
  const int jb = j1 - j0, jb4 = (jb + 3) & ~3;
  const int jbs = min(jb, lay.sbj);   // samples whose slices are staged at a time
  const int L = N - 1;
  // uniform draws depend on no core: the next iteration's draws and fiber
  // copies overlap the tail of the current one (not while recording)
  const bool pipe = D.dist == 0 && !rec;
  bool fronted = false;   // this iteration's draws and fiber copies were issued by the previous one
  long long pf_t = -1;    // >= 0: the chunk loop issues front(pf_t) once the fibers are consumed
  int cur_n = 0, cur_Q = 0, cur_jb = 0, cur_j0 = 0;
  // Draws of iteration tt (A1/A2), the per-step order/offset table and the
  // fiber copies (A3 issue; waited for after A4).  Called at the top of an
  // iteration, or, for uniform sampling, by the previous iteration once its
  // last chunk has consumed the fibers (its draws depend on no core).
  // The group is threads [gbase, gbase + gsize) (whole warps): all threads, or
  // the upper half while the lower half reduces; its barriers are named
  // barrier 1 when it is not the whole CTA.
  auto front = [&](long long tt, int gbase, int gsize) {
    const long long t = tt;
    const int tid = threadIdx.x - gbase, NT = gsize;
    auto gsync = [&]() {
      if (gsize == (int)blockDim.x) __syncthreads();
      else asm volatile("bar.sync 1, %0;" ::"r"(gsize) : "memory");
    };
    const int n = draw_mode(D.seed, t, N);
    const int In = I[n];
    auto ring = [&](int q) {
      const int k = n + 1 + q;
      return k >= N ? k - N : k;
    };
    // staged slice layout: factor s at sb + soff[s], sample jl at + jl * qpad[s];
    // written by the last thread here, read after the sampling barrier (the
    // readers of the previous iteration finished several barriers ago)
    if (tid == NT - 1) {   // the last thread: the sampling below starts at thread 0
      int off = 0;
      for (int q = 0; q < kMaxOrder; ++q) {
        const int k = q < L ? ring(q) : 0;
        const int qs = R[k] * R[k + 1 == N ? 0 : k + 1];
        order[q] = k;
        qpad[q] = (int)round_up((size_t)qs, 16 / sizeof(T));
        soff[q] = off;
        if (q < L) off += jbs * qpad[q];
      }
    }

    // ---- A1/A2: per sample, slice indices (Algorithm 2), p_F (product in ring
    // order), weight 1/(|F| J_n p_F) and fiber column -------------------------
    // Uniform sampling: first one thread per (sample, factor) draws the index,
    // then one thread per sample combines them (the draws are independent).
    const bool uni_split = D.dist == 0;
    // Leverage / Euclidean with the tables staged: the CDF and p of the L sampled
    // cores are copied to shared memory (factor sp at offset toff(sp)), then one
    // thread per (sample, factor) searches; p_F is formed per sample below.
    const bool tab_split = (D.dist == 1 || D.dist == 2) && lay.tab_ok;
    unsigned long long *tcdf = reinterpret_cast<unsigned long long *>(smem + lay.off_tab);
    int ttot = 0;
    for (int sp = 0; sp < L; ++sp) ttot += I[ring(sp)];
    double *tprob = reinterpret_cast<double *>(tcdf + ttot);
    auto toff = [&](int sp) {
      int o = 0;
      for (int q = 0; q < sp; ++q) o += I[ring(q)];
      return o;
    };
    if (tab_split) {
      for (int e = tid; e < ttot; e += NT) {
        int sp = 0, i = e;
        while (i >= I[ring(sp)]) i -= I[ring(sp++)];
        const int k = ring(sp);
        tcdf[e] = __ldcg(D.cdf[k] + i);
        tprob[e] = __ldcg(D.prob[k] + i);
      }
      gsync();
      for (int e = tid; e < L * jb; e += NT) {
        const int sp = e / jb, jl = e - sp * jb;
        const int k = ring(sp), Ik = I[k];
        const unsigned long long *cdf = tcdf + toff(sp);
        const uint64_t u = draw_u64(D.seed, t, kStreamF, k, (uint32_t)(j0 + jl));
        idx_s[jl * kMaxOrder + k] = cdf_search_smem(cdf, Ik, mulhi64(u, cdf[Ik - 1]));
      }
      gsync();
    }
    if (uni_split) {
      for (int e = tid; e < L * jb; e += NT) {
        const int sp = e / jb, jl = e - sp * jb;
        const int k = ring(sp);
        const uint64_t u = draw_u64(D.seed, t, kStreamF, k, (uint32_t)(j0 + jl));
        idx_s[jl * kMaxOrder + k] = (int)mulhi64(u, (uint64_t)I[k]);
      }
      gsync();
    }
    for (int jl = tid; jl < jb4; jl += NT) {
      if (jl >= jb) {
        wt_s[jl] = T(0);
        continue;
      }
      const bool uni = D.dist == 0;
      const bool need_pf = !uni || rec;   // uniform: every p_F = 1/J_n, weight 1/|F| (to rounding)
      double pF = 1.0;
      long long col = 0, st = 1;
      if (D.dist == 3) {   // optimal distribution: indices and p_F drawn by the sampling kernels
        for (int sp = 0; sp < L; ++sp) {
          const int k = ring(sp);
          const int i = __ldcg(D.ext_idx + (size_t)(j0 + jl) * N + k);
          idx_s[jl * kMaxOrder + k] = i;
          col += (long long)i * st;
          st *= I[k];
        }
        pF = __ldcg(D.ext_pf + j0 + jl);
      } else if (tab_split) {   // indices drawn above; p_F = prod p_k(i_k) in ring order
        for (int sp = 0; sp < L; ++sp) {
          const int k = ring(sp), i = idx_s[jl * kMaxOrder + k];
          pF = __dmul_rn(pF, tprob[toff(sp) + i]);
          col += (long long)i * st;
          st *= I[k];
        }
      } else if (uni) {   // indices drawn above; p_F = prod 1/I_k (only when recorded)
        for (int sp = 0; sp < L; ++sp) {
          const int k = ring(sp);
          if (need_pf) pF = __dmul_rn(pF, cst[k]);
          col += (long long)idx_s[jl * kMaxOrder + k] * st;
          st *= I[k];
        }
      } else {   // leverage / Euclidean: inverse-CDF draws, p_F in ring order
        uint64_t us[kMaxOrder];
#pragma unroll
        for (int sp = 0; sp < kMaxOrder; ++sp)
          us[sp] = (sp < L) ? draw_u64(D.seed, t, kStreamF, ring(sp), (uint32_t)(j0 + jl)) : 0ull;
#pragma unroll
        for (int sp = 0; sp < kMaxOrder; ++sp) {
          if (sp >= L) break;
          const int k = ring(sp), Ik = I[k];
          const unsigned long long *cdf = D.cdf[k];
          const uint64_t W = __ldcg(cdf + Ik - 1);
          const int i = cdf_search(cdf, Ik, mulhi64(us[sp], W));
          pF = __dmul_rn(pF, __ldcg(D.prob[k] + i));
          idx_s[jl * kMaxOrder + k] = i;
          col += (long long)i * st;
          st *= Ik;
        }
      }
      const double w = need_pf ? __ddiv_rn(1.0, __dmul_rn(cst[8 + n], pF)) : cst[16];
      wt_s[jl] = need_pf ? (T)w : wt_uni;
      if (kDebugChecks) {   // debug build: this sample's indices and fiber column (st = J_n here)
        for (int sp = 0; sp < L; ++sp) {
          const int k = ring(sp);
          idx_s[jl * kMaxOrder + k] =
              debug_checked(idx_s[jl * kMaxOrder + k], D.dbg_bound[k] > 0 ? D.dbg_bound[k] : I[k], D.status);
        }
        col = debug_checked(col, st, D.status);
      }
      col_s[jl] = col;
      if (rec) {
        D.dbg_pf[j0 + jl] = pF;
        for (int k = 0; k < N; ++k)
          D.dbg_idx[(size_t)(j0 + jl) * N + k] = (k == n) ? -1 : idx_s[jl * kMaxOrder + k];
      }
    }
    if (rec && c == 0 && tid == 0) *D.dbg_n = n;
    gsync();

    // ---- A3: gather the fibers into shared memory (waited for after A4) -----
    // Long fibers by bulk copies (one per fiber, issued by warp 0, completing on
    // an mbarrier); short fibers (and the slices, in A4) by 16-byte per-thread
    // asynchronous copies, which issue faster than one small bulk copy each.
    const uint32_t fbytes = (uint32_t)round_up((size_t)In * sizeof(XT), 16);
    const bool fiber_tma = fbytes >= kTmaFiberBytes;
    {
      const XT *base = static_cast<const XT *>(D.xmode[n]);
      const long long ldg = D.ldx[n];
      if (fiber_tma) {
        if (tid < 32 && jb > 0) {
          if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)jb * fbytes);
          __syncwarp();
          fence_proxy_async_smem();
          for (int jl = tid; jl < jb; jl += 32)
            tma_load_1d(xs + (size_t)jl * lay.ldxs, base + col_s[jl] * ldg, fbytes, bar);
        }
      } else {
        const int nch = (int)(fbytes / 16);
        for (int e = tid; e < jb * nch; e += NT) {
          const int jl = e / nch, ch = e - jl * nch;
          cp_async16(reinterpret_cast<char *>(xs + (size_t)jl * lay.ldxs) + 16 * ch,
                     reinterpret_cast<const char *>(base + col_s[jl] * ldg) + 16 * ch);
        }
      }
      // pad fiber rows [jb, jb4) read as zeros by the partial-gradient GEMM
      for (int e = tid; e < (jb4 - jb) * lay.ldxs; e += NT)
        xs[(size_t)(jb + e / lay.ldxs) * lay.ldxs + e % lay.ldxs] = XT(0);
    }
  };

  // The G_n pieces of the chunk of ti rows at row i0 into its operand tiles by
  // NPC bulk copies completing on bar_g (only the core-matrix rows that hold
  // rows of the chunk), and the FP32 rows [r0, r1) of the chunk this CTA
  // updates into gown (16-byte asynchronous copies, waited for before the
  // residual).  The operand tiles alias the staged slices and the chain
  // buffers: called once those are dead.
  auto g_issue = [&](int ti, int i0) {
    if constexpr (kTC) {
      const int n = cur_n, Q = cur_Q;
      const float *Gn = static_cast<const float *>(D.cores[n]);
      const int QC = lay.qp / 8;
      const uint32_t bytes = (uint32_t)(((ti + 7) & ~7) >> 3) * (uint32_t)QC * 128u;
      if (tid == 0) {
        fence_proxy_async_smem();   // earlier generic accesses of the region come first
        mbar_arrive_expect_tx(bar_g, (uint32_t)NPC * bytes);
        const unsigned char *src = static_cast<const unsigned char *>(D.gpc[n]) + (size_t)(i0 >> 7) * NPC * gcs;
#pragma unroll
        for (int p = 0; p < NPC; ++p) tma_load_1d(smem + lay.off_reg + p * gcs, src + p * gcs, bytes, bar_g);
      }
      const int r0 = ti * c / C, r1 = ti * (c + 1) / C;
      float *own = reinterpret_cast<float *>(gown);
      if ((Q & 3) == 0 && ((D.slice_tma >> n) & 1)) {
        const int nch = Q >> 2;
        for (int e = tid; e < (r1 - r0) * nch; e += NT) {
          const int ii = e / nch, ch = e - ii * nch;
          cp_async16(own + (size_t)ii * ldq + 4 * ch, Gn + (size_t)(i0 + r0 + ii) * Q + 4 * ch);
        }
      } else {
        for (int e = tid; e < (r1 - r0) * Q; e += NT) {
          const int ii = e / Q, q = e - ii * Q;
          own[(size_t)ii * ldq + q] = __ldcg(Gn + (size_t)(i0 + r0 + ii) * Q + q);
        }
      }
    }
  };

  // Tensor-core residual and partial gradient of one chunk of <= 128 rows of
  // G_n (operands as NPC BF16 pieces, FP32 accumulation in TMEM):
  //   D_R(i, jl) = G(i, :) Z(jl, :)^T  as the piece products of total order
  //                < NPC (NPC = 2: hi*hi + hi*lo + lo*hi; NPC = 3: six),
  //   Ew(i, jl)  = w_jl (D_R(i, jl) - X_S(jl, i))   (epilogue; EWP pieces),
  //   D_P(i, q)  = sum_jl Ew(i, jl) Z(jl, q)        (Z read MN-major; products
  //                of total order < EWP: Ew x Z_hi for BF16-mixed),
  // then D_P -> reg[i][q] (FP32) for the cluster reduction.
  auto tc_chunk = [&](int ti, int i0) {
    if constexpr (kTC) {
      const int n = cur_n, In = I[n], Q = cur_Q, jb = cur_jb;
      T *Gn = static_cast<T *>(D.cores[n]);
      const int QC = lay.qp / 8;
      unsigned char *gp[NPC > 0 ? NPC : 1], *zp[NPC > 0 ? NPC : 1], *ewp[EWP];
#pragma unroll
      for (int k = 0; k < NPC; ++k) {
        gp[k] = smem + lay.off_reg + (size_t)k * 128 * lay.qp * 2;
        zp[k] = smem + lay.off_zp[k];
      }
#pragma unroll
      for (int k = 0; k < EWP; ++k) ewp[k] = smem + lay.off_ew + (size_t)k * 128 * lay.jbp * 2;
      const bool g16 = (D.slice_tma >> n) & 1;   // 16-byte rows of G_n: float4 reads
      // plain variant: the rows [r0, r1) this CTA owns in the update are kept in
      // gown, so that the update reads them from shared memory
      const bool stash = !scaled;
      const int r0 = ti * c / C, r1 = ti * (c + 1) / C;
      // only the core-matrix rows that hold rows of the chunk: row i of both
      // products depends on row i of G (and of Ew) only, and rows >= ti of the
      // results are never read
      const int ti8 = (ti + 7) & ~7;
      if (gbulk) {
        if (i0 > 0) g_issue(ti, i0);   // the first chunk's copies were issued beside the Z pieces
        cp_async_wait_all();           // the owned rows
        if (!mbar_wait_bounded(bar_g, gphase, wlim)) {
          latch_status(D.status, kStatusTimeout);
          mbar_wait_bounded(bar_g, gphase, kWaitLimit);
        }
        gphase ^= 1u;
      }
      for (int e = tid; !gbulk && e < ti8 * QC; e += NT) {
        // 8 consecutive threads: the 8 rows of one core matrix, so that each
        // piece store of a warp covers 512 contiguous bytes (no bank conflicts)
        const int rest = e >> 3, qb = rest % QC, ii = (rest / QC) * 8 + (e & 7);
        const bool live = ii < ti;
        const float *grow = reinterpret_cast<const float *>(Gn) + (size_t)(i0 + (live ? ii : 0)) * Q;
        float v[8];
        if (g16) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = qb * 8 + 4 * h;
            const float4 f = (live && q < Q) ? __ldcg(reinterpret_cast<const float4 *>(grow + q))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * h] = f.x;
            v[4 * h + 1] = f.y;
            v[4 * h + 2] = f.z;
            v[4 * h + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int q = qb * 8 + j;
            v[j] = (live && q < Q) ? __ldcg(grow + q) : 0.f;
          }
        }
        uint4 w[NPC > 0 ? NPC : 1];
        bf16_split8<NPC>(v, w);
        const uint32_t o = kmaj_off(ii, qb * 8, QC);
#pragma unroll
        for (int k = 0; k < NPC; ++k) *reinterpret_cast<uint4 *>(gp[k] + o) = w[k];
        if (stash && ii >= r0 && ii < r1) {   // FP32 values of the rows this CTA updates
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (qb * 8 + j < Q) gown[(size_t)(ii - r0) * ldq + qb * 8 + j] = v[j];
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      const int NR = max(16, (jb + 15) & ~15);   // columns of D_R (samples, padded)
      const int KQ = (Q + 15) & ~15;             // contraction length of D_R
      if (tid == 0) {
        tc_fence_after();
        const uint32_t idr = umma_idesc_bf16(128, NR, 0, 0);
        const uint32_t sbo = (uint32_t)QC * 128;
        // piece products of total order < NPC, in the order (0,0), (0,1), ..
        for (int kb = 0; kb < KQ / 16; ++kb) {
          const uint32_t ko = (uint32_t)kb * 256;
#pragma unroll
          for (int a = 0; a < NPC; ++a)
#pragma unroll
            for (int b = 0; a + b < NPC; ++b)
              umma_bf16(tbase, umma_desc(smem_u32(gp[a]) + ko, 128, sbo), umma_desc(smem_u32(zp[b]) + ko, 128, sbo),
                        idr, kb > 0 || a > 0 || b > 0);
        }
        umma_commit(bar_mma);
      }
      if (!mbar_wait_bounded(bar_mma, mphase, wlim)) {
        latch_status(D.status, kStatusTimeout);
        mbar_wait_bounded(bar_mma, mphase, kWaitLimit);
      }
      mphase ^= 1u;
      tc_fence_after();
      const int warp = tid >> 5, lane = tid & 31, qd = warp & 3, wg = warp >> 2, nwg = NT >> 7;
      const int row = 32 * qd + lane;
      const int JC = NR / 8;
      T *dbg_e = rec ? static_cast<T *>(D.dbg_e) : nullptr;
      for (int c16 = wg; c16 < NR / 16; c16 += nwg) {   // 16 TMEM columns per load (NR: multiple of 16)
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(c16 * 16), v);
        if (row < ti) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c8 = 2 * c16 + h;
            float ev[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int jl = c8 * 8 + j;
              ev[j] = 0.f;
              if (jl < jb) {
                const float x = to_f32(xs[(size_t)jl * lay.ldxs + i0 + row]);
                const float e = v[8 * h + j] - x;
                if (dbg_e) dbg_e[(size_t)(cur_j0 + jl) * In + i0 + row] = e;
                ev[j] = e * wt_s[jl];
              }
            }
            uint4 w[EWP];
            bf16_split8<EWP>(ev, w);
            const uint32_t o = kmaj_off(row, c8 * 8, JC);
#pragma unroll
            for (int k = 0; k < EWP; ++k) *reinterpret_cast<uint4 *>(ewp[k] + o) = w[k];
          }
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      const int NP = (Q + 15) & ~15;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t idp = umma_idesc_bf16(128, NP, 0, 1);
        // Ew pieces x Z pieces of total order < EWP (BF16-mixed: Ew x Z_hi)
        for (int kb = 0; kb < NR / 16; ++kb) {
#pragma unroll
          for (int a = 0; a < EWP; ++a)
#pragma unroll
            for (int b = 0; a + b < EWP; ++b)
              umma_bf16(tbase + 256, umma_desc(smem_u32(ewp[a]) + (uint32_t)kb * 256, 128, (uint32_t)JC * 128),
                        umma_desc(smem_u32(zp[b]) + (uint32_t)kb * 2 * QC * 128, (uint32_t)QC * 128, 128), idp,
                        kb > 0 || a > 0 || b > 0);
        }
        umma_commit(bar_mma);
      }
      if (!mbar_wait_bounded(bar_mma, mphase, wlim)) {
        latch_status(D.status, kStatusTimeout);
        mbar_wait_bounded(bar_mma, mphase, kWaitLimit);
      }
      mphase ^= 1u;
      tc_fence_after();
      for (int c16 = wg; c16 < NP / 16; c16 += nwg) {   // NP: multiple of 16
        float v[16];
        tmem_ld16(tbase + 256 + ((uint32_t)(32 * qd) << 16) + (uint32_t)(c16 * 16), v);
        if (row < ti) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int q = c16 * 16 + j;
            if (q < Q) reg[(size_t)row * lay.ldq + q] = v[j];
          }
        }
      }
      tc_fence_before();
    }
  };

  for (int s = 0; s < nsteps; ++s) {
    const long long t = t0 + s;
    const int n = draw_mode(D.seed, t, N);
    const int In = I[n], Rn = R[n], Rn1 = R[(n + 1) % N], Q = Rn * Rn1;
    const int Q4 = (Q + 3) & ~3;
    cur_n = n;
    cur_Q = Q;
    cur_jb = jb;
    cur_j0 = j0;
    const int all_k = (1 << N) - 1;
    const bool sl_async = ((D.slice_tma | (1 << n)) & all_k) == all_k;   // every factor's slices 16-byte rows
    T *Gn = static_cast<T *>(D.cores[n]);
    T *accn = static_cast<T *>(D.acc[n]);
    const uint32_t fbytes = (uint32_t)round_up((size_t)In * sizeof(XT), 16);
    const bool fiber_tma = fbytes >= kTmaFiberBytes;
    if (!fronted) front(t, 0, NT);
    fronted = false;

    // ---- A4: sampled subchain rows, Z(j, r + r' R_n) = P_j(r', r) ----------
    if (lay.sb_ok) {
      // Per group of jbs samples: stage the sampled slices G_k(i_k), then
      // P_1 = G_{n+1}(i) (staged, column-major); P_{s+1} = P_s G_{k_s}(i_s),
      // row-major [r'][b] per sample; the last product lands in rows s0.. of Z.
      // Intermediates ping-pong between two buffers.
      T *const pb0 = reinterpret_cast<T *>(smem + lay.off_p0), *const pb1 = reinterpret_cast<T *>(smem + lay.off_p1);
      const int pst = lay.pstride;
      const int warp = tid >> 5, lane = tid & 31, nwarps = NT >> 5;
      for (int s0 = 0; s0 < jb; s0 += jbs) {
        const int jbc = min(jbs, jb - s0);
        const int *idg = idx_s + s0 * kMaxOrder;
        for (int q = 0; q < L; ++q) {
          const int k = order[q], qs = R[k] * R[(k + 1) % N];
          const T *G = static_cast<const T *>(D.cores[k]);
          if (sl_async) {
            const int nch = qs * (int)sizeof(T) / 16;
            for (int e = tid; e < jbc * nch; e += NT) {
              const int jl = e / nch, ch = e - jl * nch;
              cp_async16(reinterpret_cast<char *>(sb + soff[q] + (size_t)jl * qpad[q]) + 16 * ch,
                         reinterpret_cast<const char *>(G + (size_t)idg[jl * kMaxOrder + k] * qs) + 16 * ch);
            }
          } else {
#pragma unroll 4
            for (int e = tid; e < jbc * qs; e += NT) {
              const int jl = e / qs, off = e - jl * qs;
              sb[soff[q] + (size_t)jl * qpad[q] + off] = ld_l2(G + (size_t)idg[jl * kMaxOrder + k] * qs + off);
            }
          }
          cp_async_commit_group();   // one group per factor (the first also holds the fibers)
        }
        // factor 1 needs the slices of factors 0 and 1; later ones arrive meanwhile
        cp_async_wait_pending(L >= 2 ? L - 2 : 0);
        __syncthreads();
        for (int q = 1; q < L; ++q) {
          if (q >= 2) {
            cp_async_wait_pending(L - 1 - q);
            __syncthreads();
          }
          const int k = order[q], Ra = R[k], Rb = R[(k + 1) % N];
          const bool last = q == L - 1;
          T *dst = last ? zs + (size_t)s0 * ldq : ((q & 1) ? pb1 : pb0);
          const int dstride = last ? ldq : pst;
          const T *src = (q == 1) ? sb + soff[0] : (((q - 1) & 1) ? pb1 : pb0);
          const int sstride = (q == 1) ? qpad[0] : pst;
          const int per = Rn1 * Rb;              // entries of P_{q+1} per sample (<= 256)
          bool done = true;
          switch (ru) {
            case 4: q == 1 ? chain_factor_uniform<4, 2, true, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc)
                           : chain_factor_uniform<4, 2, false, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc); break;
            case 8: q == 1 ? chain_factor_uniform<8, 2, true, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc)
                           : chain_factor_uniform<8, 2, false, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc); break;
            case 10: q == 1 ? chain_factor_uniform<10, 2, true, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc)
                            : chain_factor_uniform<10, 2, false, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc); break;
            case 16: q == 1 ? chain_factor_uniform<16, 2, true, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc)
                            : chain_factor_uniform<16, 2, false, T>(src, sstride, sb + soff[q], qpad[q], dst, dstride, jbc); break;
            default: done = false;
          }
          if (!done) {
            // general ranks: this lane's entries it = lane + 32 u, row r' and column b
            int pofs[8], pstep[8], sofs[8], dofs[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int it = lane + 32 * u;
              const int rp = it / Rb, bb = it - rp * Rb;
              pofs[u] = (q == 1) ? rp : rp * Ra;
              pstep[u] = (q == 1) ? Rn1 : 1;
              sofs[u] = bb * Ra;
              dofs[u] = rp * Rb + bb;
            }
            for (int jl = warp; jl < jbc; jl += nwarps) {
              const T *prow = src + (size_t)jl * sstride;
              const T *S = sb + soff[q] + (size_t)jl * qpad[q];
              T *drow = dst + (size_t)jl * dstride;
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (lane + 32 * u < per) {
                  const T *pp = prow + pofs[u];
                  const T *sc = S + sofs[u];
                  const int ps = pstep[u];
                  T acc = T(0);
                  for (int a = 0; a < Ra; ++a) acc = fma(pp[a * ps], sc[a], acc);
                  drow[dofs[u]] = acc;
                }
              }
            }
          }
          __syncthreads();
        }
        if (L == 1) {   // N = 2: Z row is the single staged slice, transposed
          for (int e = tid; e < jbc * Q; e += NT) {
            const int jl = e / Q, rem = e - jl * Q, rp = rem / Rn, r = rem - rp * Rn;
            zs[(size_t)(s0 + jl) * ldq + rem] = sb[soff[0] + (size_t)jl * qpad[0] + rp + r * Rn1];
          }
          __syncthreads();   // the next group restages the slices
        }
      }
      if (rec) {
        __syncthreads();
        for (int e = tid; e < jb * Q; e += NT)
          static_cast<T *>(D.dbg_z)[(size_t)(j0 + e / Q) * Q + e % Q] = zs[(size_t)(e / Q) * ldq + e % Q];
      }
    } else {
      for (int e = tid; e < jb * Rn1; e += NT) {
        const int jl = e / Rn1, rp = e - jl * Rn1;
        T row[RMAX];
        chain_row<RMAX, T, true>(reinterpret_cast<const T *const *>(D.cores), R, N, order, idx_s + jl * kMaxOrder,
                                 L, rp, row);
        T *zrow = zs + (size_t)jl * ldq + rp * Rn;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
          if (r < Rn) {
            zrow[r] = row[r];
            if (rec) static_cast<T *>(D.dbg_z)[(size_t)(j0 + jl) * Q + rp * Rn + r] = row[r];
          }
        }
      }
    }
    // the fibers (A3)
    cp_async_wait_all();
    if (fiber_tma && jb > 0) {
      if (!mbar_wait_bounded(bar, phase, wlim)) {
        latch_status(D.status, kStatusTimeout);
        mbar_wait_bounded(bar, phase, kWaitLimit);
      }
      phase ^= 1u;
    }
    // zero padding of Z: columns [Q, Q4) of rows < jb, and rows [jb, jb4)
    if (Q4 > Q)
      for (int e = tid; e < jb * (Q4 - Q); e += NT) zs[(size_t)(e / (Q4 - Q)) * ldq + Q + e % (Q4 - Q)] = T(0);
    for (int e = tid; e < (jb4 - jb) * Q4; e += NT) zs[(size_t)(jb + e / Q4) * ldq + e % Q4] = T(0);
    __syncthreads();
    if (gbulk && c >= lay.cw0) g_issue(min(lay.TI, In), 0);   // lands while the Z pieces are formed
    if constexpr (kTC) {
      // Z as NPC BF16 pieces in the no-swizzle K-major tiles [JBP rows jl][QP cols q]
      const int QC = lay.qp / 8;
      for (int e = tid; e < lay.jbp * QC; e += NT) {
        // 8 consecutive threads: the 8 rows of one core matrix (conflict-free
        // piece stores); 16-byte reads of Z, whose rows are zero-padded to Q4
        const int rest = e >> 3, qb = rest % QC, jl = (rest / QC) * 8 + (e & 7);
        float v[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = qb * 8 + 4 * h;
          const float4 f = (jl < jb && q < Q) ? *reinterpret_cast<const float4 *>(zs + (size_t)jl * ldq + q)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
          v[4 * h] = f.x;
          v[4 * h + 1] = f.y;
          v[4 * h + 2] = f.z;
          v[4 * h + 3] = f.w;
        }
        uint4 w[NPC > 0 ? NPC : 1];
        bf16_split8<NPC>(v, w);
        const uint32_t o = kmaj_off(jl, qb * 8, QC);
#pragma unroll
        for (int k = 0; k < NPC; ++k) *reinterpret_cast<uint4 *>(smem + lay.off_zp[k] + o) = w[k];
      }
      fence_proxy_async_smem();
      __syncthreads();
    }

    // ---- S: preconditioner h = Z^T D Z / (|F| J_n) + eta^t I (FP64 solve) ---
    if (scaled) {
      const int QH = lay.QH;
      const T *gz = zs;     // rows of the Hessian batch: F itself, or an independent H
      const T *gw = wt_s;
      int gjb = jb;
      if (D.JH > 0) {
        // |H| rows drawn on their own Philox stream with the same distributions;
        // weights 1/(|H| J_n p_H) (Eq. S_hessian)
        const int JH = D.JH;
        const int h0 = (int)((long long)JH * c / C), h1 = (int)((long long)JH * (c + 1) / C);
        const int jbh = h1 - h0, jbh4 = (jbh + 3) & ~3;
        int *hidx = reinterpret_cast<int *>(smem + lay.off_hidx);
        T *hw = reinterpret_cast<T *>(smem + lay.off_hw);
        T *hz = reinterpret_cast<T *>(smem + lay.off_hz);
        for (int jl = tid; jl < jbh4; jl += NT) {
          if (jl >= jbh) {
            hw[jl] = T(0);
            continue;
          }
          double pH = 1.0;
          for (int sp = 0; sp < L; ++sp) {
            const int k = order[sp], Ik = I[k];
            const uint64_t u = draw_u64(D.seed, t, kStreamH, k, (uint32_t)(h0 + jl));
            int i;
            if (D.dist == 0) {
              i = (int)mulhi64(u, (uint64_t)Ik);
              pH = __dmul_rn(pH, cst[k]);
            } else {
              const unsigned long long *cdf = D.cdf[k];
              const uint64_t W = __ldcg(cdf + Ik - 1);
              i = cdf_search(cdf, Ik, mulhi64(u, W));
              pH = __dmul_rn(pH, __ldcg(D.prob[k] + i));
            }
            hidx[jl * kMaxOrder + k] = debug_checked(i, D.dbg_bound[k] > 0 ? D.dbg_bound[k] : Ik, D.status);
          }
          hw[jl] = (T)__ddiv_rn(1.0, __dmul_rn(cst[24 + n], pH));
        }
        __syncthreads();
        for (int e = tid; e < jbh * Rn1; e += NT) {
          const int jl = e / Rn1, rp = e - jl * Rn1;
          T row[RMAX];
          chain_row<RMAX, T, true>(reinterpret_cast<const T *const *>(D.cores), R, N, order, hidx + jl * kMaxOrder,
                                   L, rp, row);
          T *zrow = hz + (size_t)jl * ldq + rp * Rn;
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < Rn) zrow[r] = row[r];
        }
        for (int e = tid; e < jbh4 * Q4; e += NT) {
          const int jl = e / Q4, q = e - jl * Q4;
          if (jl >= jbh || q >= Q) hz[(size_t)jl * ldq + q] = T(0);
        }
        __syncthreads();
        gz = hz;
        gw = hw;
        gjb = jbh;
      }
      gemm_s<4, true, true, T>(Q, Q, gjb, gz, ldq, gz, ldq, gw,
                               [=](int a, int b, T v) { reg[(size_t)a * ldq + b] = v; });
      cluster.sync();
      const int q0 = Q * c / C, q1 = Q * (c + 1) / C;
      if constexpr (kDF) {   // FP32 cores: the Gram solve in double-float arithmetic
        df64 *h0 = reinterpret_cast<df64 *>(cluster.map_shared_rank(h64, 0));
        df64 *hd0 = reinterpret_cast<df64 *>(cluster.map_shared_rank(hdiag, 0));
        const df64 damp = df_from_double(D.damping);
        for (int e = tid; e < (q1 - q0) * Q; e += NT) {
          const int a = q0 + e / Q, b = e % Q;
          df64 v = df64{(float)cluster_sum(reg, (size_t)a * ldq + b), 0.f};
          if (a == b) {
            v = df_add(v, damp);
            hd0[a] = v;
          }
          h0[a * QH + b] = v;
          if (rec) D.dbg_h[a * Q + b] = df_to_double(v);
        }
      } else {
        double *h0 = cluster.map_shared_rank(h64, 0);
        double *hd0 = cluster.map_shared_rank(hdiag, 0);
        for (int e = tid; e < (q1 - q0) * Q; e += NT) {
          const int a = q0 + e / Q, b = e % Q;
          double v = (double)cluster_sum(reg, (size_t)a * ldq + b);
          if (a == b) {
            v += D.damping;
            hd0[a] = v;
          }
          h0[a * QH + b] = v;
          if (rec) D.dbg_h[a * Q + b] = v;
        }
      }
      cluster.sync();
      if (c == 0) {
        // factor, growing the damping on failure (1e-12 tr(h)/Q * 10^m, m = 0..6);
        // the factor and reciprocal pivots go to D.lfac for every CTA's solves
        using V = typename GramScalar<T>::type;
        const V *A = reinterpret_cast<const V *>(h64);
        const V *hd = reinterpret_cast<const V *>(hdiag);
        V *colbuf = reinterpret_cast<V *>(smem + lay.off_reg);   // reg is free here
        V *pinv = colbuf + 8 * Q + 96;   // past the factorisation's published blocks
        V *lout = static_cast<V *>(D.lfac);
        if (tid == 0) {
          double tr = 0.0;
          for (int q = 0; q < Q; ++q) tr += gs_to_double(hd[q]) - D.damping;
          misc[2] = tr;
        }
        __syncthreads();
        const double tr = misc[2];
        const int Qb = (Q + 3) >> 2;
        const bool one_block = Qb * (Qb + 1) / 2 <= NT;   // else two blocks per thread
        auto attempt = [&](double extra) {
          return one_block ? gram_factor_reg<V, 1>(A, Q, QH, extra, colbuf, pinv, lout)
                           : gram_factor_reg<V, 2>(A, Q, QH, extra, colbuf, pinv, lout);
        };
        bool ok = attempt(0.0);
        double extra = 0.0;
        for (int m = 0; m < 7 && !ok; ++m) {
          extra = 1e-12 * tr / Q * pow(10.0, (double)m);
          __syncthreads();
          ok = attempt(extra);
        }
        if (rec && ok && extra > 0.0)
          for (int q = tid; q < Q; q += NT) D.dbg_h[q * Q + q] = gs_to_double(hd[q]) + extra;
        if (tid == 0) {
          misc[0] = ok ? 1.0 : 0.0;
          if (!ok) latch_status(D.status, kStatusNumeric);
        }
      }
    }

    // ---- B/C/R: per chunk of rows of G_n ------------------------------------
    int own_rows = 0;
    T *gs = reg;   // G_n chunk [ti][ldg]; the partial gradient reuses the same region
    const int ldg = lay.ldg;
    for (int i0 = 0; i0 < In; i0 += lay.TI) {
      const int ti = min(lay.TI, In - i0);
      pf_t = (pipe && i0 + ti >= In && s + 1 < nsteps) ? t + 1 : -1;
      if (c < lay.cw0) {   // no samples on this CTA: a zero partial gradient
        for (int e = tid; e < ti * Q; e += NT) reg[(size_t)(e / Q) * ldq + e % Q] = T(0);
        if (kTC && !scaled) {   // a plain problem beside scaled ones: the update reads its rows from gown
          const int r0 = ti * c / C, r1 = ti * (c + 1) / C;
          for (int e = tid; e < (r1 - r0) * Q; e += NT)
            gown[(size_t)(e / Q) * ldq + e % Q] = ld_l2(Gn + (size_t)(i0 + r0 + e / Q) * Q + e % Q);
        }
      } else {
        if constexpr (kTC) {
          tc_chunk(ti, i0);
        } else {
          if ((Q * (int)sizeof(T)) % 16 == 0 && ((D.slice_tma >> n) & 1)) {
            const int nch = Q * (int)sizeof(T) / 16;
            for (int e = tid; e < ti * nch; e += NT) {
              const int ii = e / nch, ch = e - ii * nch;
              cp_async16(reinterpret_cast<char *>(gs + (size_t)ii * ldg) + 16 * ch,
                         reinterpret_cast<const char *>(Gn + (size_t)(i0 + ii) * Q) + 16 * ch);
            }
          } else {
#pragma unroll 4
            for (int e = tid; e < ti * Q; e += NT) {
              const int ii = e / Q, q = e - ii * Q;
              gs[(size_t)ii * ldg + q] = ld_l2(Gn + (size_t)(i0 + ii) * Q + q);
            }
          }
          if (Q4 > Q)
            for (int e = tid; e < ti * (Q4 - Q); e += NT) gs[(size_t)(e / (Q4 - Q)) * ldg + Q + e % (Q4 - Q)] = T(0);
          cp_async_wait_all();
          __syncthreads();
          // residual, weighted in place: X_s(jl, i) <- w_j (G Z^T - X_S)(i, jl)
          {
            XT *xsp = xs;
            const int ldxs = lay.ldxs;
            T *dbg_e = rec ? static_cast<T *>(D.dbg_e) : nullptr;
            const T *wt = wt_s;
            gemm_s<2, false, false, T>(ti, jb, Q, gs, ldg, zs, ldq, nullptr, [=](int ii, int jl, T v) {
              T *xp = reinterpret_cast<T *>(xsp) + (size_t)jl * ldxs + i0 + ii;
              const T e = v - *xp;
              if (dbg_e) dbg_e[(size_t)(j0 + jl) * In + i0 + ii] = e;
              *xp = e * wt[jl];
            });
          }
          __syncthreads();
          // partial gradient of this CTA's samples: Gp(i, q) = sum_jl Ew(jl, i) Z(jl, q)
          gemm_s<4, true, true, T>(ti, Q, jb, reinterpret_cast<T *>(xs) + i0, lay.ldxs, zs, ldq, nullptr,
                                   [=](int ii, int q, T v) { reg[(size_t)ii * ldq + q] = v; });
        }
      }
      // Last chunk of a pipelined iteration: every thread arrives (its partial
      // gradient released); the upper half of the CTA then issues the next
      // iteration's draws and fiber copies while the lower half waits, reduces
      // and updates; the halves meet at the closing cluster barrier.
      const bool split = pf_t >= 0;
      const int rt = split ? NT / 2 : NT;   // threads of the reduction
      if (split) {
        if constexpr (!kTC) __syncthreads();   // the SIMT gradient GEMM's reads of xs are done
        cluster_arrive_release();
        if (tid >= rt) front(pf_t, rt, NT - rt);
        cluster_wait_acquire();
        fronted = true;
      } else {
        cluster.sync();
      }
      pf_t = -1;
      const int r0 = ti * c / C, r1 = ti * (c + 1) / C;
      // reduced gradient of one owned entry -> step rule and update (or kept for
      // the solve); returns the updated entry (plain variant)
      auto own_entry = [&](int ii, int q, T g) -> T {
        const size_t gi = (size_t)(i0 + ii) * Q + q;
        if (rec) static_cast<T *>(D.dbg_g)[gi] = g;
        if (scaled) {
          gown[(size_t)(own_rows + ii - r0) * ldq + q] = g;
          return g;
        }
        const T p = -g;
        T *own = gown + (size_t)(ii - r0) * ldq + q;
        const T cur = kTC ? *own : ld_l2(Gn + gi);   // the tensor-core chunk kept the owned rows
        const T nv = cur + step_delta<T>(D.rule, alpha_t, eta_t, b_t, D.eps, accn, gi, p);
        if (!isfinite(nv)) latch_status(D.status, kStatusNumeric);
        Gn[gi] = nv;
        *own = nv;
        if (rec) static_cast<T *>(D.dbg_p)[gi] = p;
        return nv;
      };
      // the pieces of updated entries (q0, 4 values / q, one value) of row ii of
      // the chunk in the global piece tiles of core n
      unsigned char *gpn = gbulk ? static_cast<unsigned char *>(D.gpc[n]) + (size_t)(i0 >> 7) * NPC * gcs : nullptr;
      auto put_pieces4 = [&](int ii, int q0, float v0, float v1, float v2, float v3) {
        if constexpr (kTC) {
          const float v[4] = {v0, v1, v2, v3};
          uint2 w[NPC > 0 ? NPC : 1];
          bf16_split4<NPC>(v, w);
          unsigned char *o = gpn + kmaj_off(ii, q0, lay.qp / 8);
#pragma unroll
          for (int p = 0; p < NPC; ++p) *reinterpret_cast<uint2 *>(o + p * gcs) = w[p];
        }
      };
      auto put_piece1 = [&](int ii, int q, T v) {
        if constexpr (kTC) {
          __nv_bfloat16 w[NPC > 0 ? NPC : 1];
          bf16_split1<NPC>((float)v, w);
          unsigned char *o = gpn + kmaj_off(ii, q, lay.qp / 8);
#pragma unroll
          for (int p = 0; p < NPC; ++p) *reinterpret_cast<__nv_bfloat16 *>(o + p * gcs) = w[p];
        }
      };
      if constexpr (sizeof(T) == 4) {
        if ((Q & 3) == 0) {
          // 16-byte remote loads; owner c pulls from CTAs c+1, c+2, ... (mod C) and
          // sums in that fixed order (deterministic), so that the owners' requests
          // spread over all CTAs instead of all hitting CTA 0 first
          const int Qv = Q >> 2;
          for (int e = tid; tid < rt && e < (r1 - r0) * Qv; e += rt) {
            const int ii = r0 + e / Qv, q0 = (e - (e / Qv) * Qv) * 4;
            float4 v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int cc = c + 1 + u >= C ? c + 1 + u - C : c + 1 + u;
              v[u] = (u < C) ? *reinterpret_cast<const float4 *>(cluster.map_shared_rank(reg, cc) + (size_t)ii * ldq + q0)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (u < C) {
                g.x += v[u].x;
                g.y += v[u].y;
                g.z += v[u].z;
                g.w += v[u].w;
              }
            const float n0 = own_entry(ii, q0, g.x), n1 = own_entry(ii, q0 + 1, g.y);
            const float n2 = own_entry(ii, q0 + 2, g.z), n3 = own_entry(ii, q0 + 3, g.w);
            if (gbulk) put_pieces4(ii, q0, n0, n1, n2, n3);
          }
        } else {
          for (int e = tid; tid < rt && e < (r1 - r0) * Q; e += rt) {
            const int ii = r0 + e / Q, q = e % Q;
            const T nv = own_entry(ii, q, cluster_sum(reg, (size_t)ii * ldq + q));
            if (gbulk) put_piece1(ii, q, nv);
          }
        }
      } else {
        for (int e = tid; tid < rt && e < (r1 - r0) * Q; e += rt) {
          const int ii = r0 + e / Q, q = e % Q;
          own_entry(ii, q, cluster_sum(reg, (size_t)ii * ldq + q));
        }
      }
      if (!scaled && D.dist == 2) {
        __syncthreads();
        for (int ii = r0 + tid; ii < r1; ii += NT) {
          const T *row = gown + (size_t)(ii - r0) * ldq;
          double sn = 0.0;
          for (int q = 0; q < Q; ++q) {
            const double v = (double)row[q];
            sn = __dadd_rn(sn, __dmul_rn(v, v));
          }
          D.snorm[n][i0 + ii] = sn;
        }
      }
      own_rows += r1 - r0;
      if (gbulk) fence_proxy_async_global();   // the rewritten pieces before the next bulk copies
      cluster.sync();
    }

    // ---- scaled direction p = -g h^{-1} on the owned rows, then the update --
    if (scaled) {
      // every CTA copies the factor (written by CTA 0 before the chunk loop's
      // barriers) into its own shared memory at an odd pitch, so that both a
      // column (forward solve) and a row (backward solve) of L are read
      // without bank conflicts, and inverts its 32 x 32 diagonal blocks (one
      // warp each, in the reg region, free here); then one warp per owned row
      // solves L y = -g^T and L^T x = y blockwise in the Gram-solve scalar.
      using V = typename GramScalar<T>::type;
      const int ldl = Q | 1;
      V *Lc = reinterpret_cast<V *>(h64);
      V *ivc = reinterpret_cast<V *>(hdiag);
      const bool ok = *cluster.map_shared_rank(misc, 0) != 0.0;
      const int warp = tid >> 5, lane = tid & 31, nw = NT >> 5;
      // owned row number rr -> row of G_n: chunk by chunk, this CTA owned rows
      // [i0 + ti c / C, i0 + ti (c + 1) / C) of each chunk [i0, i0 + ti)
      auto own_row = [&](int rr) {
        for (int i0 = 0; i0 < In; i0 += lay.TI) {
          const int ti = min(lay.TI, In - i0), a = ti * c / C, b = ti * (c + 1) / C;
          if (rr < b - a) return i0 + a + rr;
          rr -= b - a;
        }
        return In - 1;   // not reached: rr < own_rows
      };
      constexpr int QM = 4;        // Q <= 128 = 32 * QM
      if (ok) {
        const V *Lg = static_cast<const V *>(D.lfac);
        for (int e = tid; e < Q * Q; e += NT) {
          const int k = e / Q, q = e - k * Q;
          if (q >= k) Lc[k * ldl + q] = gs_ldcg(Lg + e);
        }
        for (int q = tid; q < Q; q += NT) ivc[q] = gs_ldcg(Lg + (size_t)Q * Q + q);
      }
      __syncthreads();
      V *Dc = reinterpret_cast<V *>(reg);   // inverted diagonal blocks, then a buffer per solving warp
      const int nbq = (Q + kGsB - 1) / kGsB;
      if (ok && warp < nbq) gram_block_inverse<V>(Lc, ldl, ivc, Q, warp, Dc);
      __syncthreads();
      const int nsv = min(nw, lay.nsolve);   // solving warps, one buffer each after the blocks
      V *wbuf = Dc + gram_solve_scratch(Q, warp);
      for (int rr = warp; warp < nsv && rr < own_rows; rr += nsv) {
        const int i = own_row(rr);
        T *grow = gown + (size_t)rr * ldq;
        gram_solve_row<T, V>(Lc, ldl, Dc, Q, ok, grow, wbuf);   // g in, p out
        __syncwarp();
#pragma unroll
        for (int m = 0; m < QM; ++m) {
          const int q = lane + 32 * m;
          if (q >= Q) continue;
          const size_t gi = (size_t)i * Q + q;
          const T p = grow[q];
          const T nv = ld_l2(Gn + gi) + step_delta<T>(D.rule, alpha_t, eta_t, b_t, D.eps, accn, gi, p);
          if (!isfinite(nv)) latch_status(D.status, kStatusNumeric);
          Gn[gi] = nv;
          grow[q] = nv;
          if (rec) static_cast<T *>(D.dbg_p)[gi] = p;
        }
      }
      if (D.dist == 2) {
        __syncthreads();
        for (int rr = tid; rr < own_rows; rr += NT) {
          const T *row = gown + (size_t)rr * ldq;
          double sn = 0.0;
          for (int q = 0; q < Q; ++q) {
            const double v = (double)row[q];
            sn = __dadd_rn(sn, __dmul_rn(v, v));
          }
          D.snorm[n][own_row(rr)] = sn;
        }
      }
      cluster.sync();
    }

    // ---- leverage table of core n for the next iteration (CTA 0) ----------
    if (D.dist == 1) {
      if (c == 0) leverage_table_cta<T>(Gn, In, Q, smem + lay.off_reg, D.prob[n], D.cdf[n], D.status);
      cluster.sync();
    }

    // ---- Euclidean table of core n for the next iteration (CTA 0) ---------
    if (D.dist == 2) {
      if (c == 0) {
        double *scr = reinterpret_cast<double *>(smem + lay.off_reg);   // dead after the last barrier
        unsigned long long *wsc = reinterpret_cast<unsigned long long *>(scr + In);
        const double *sn = D.snorm[n];
        for (int i = tid; i < In; i += NT) scr[i] = __ldcg(sn + i);
        __syncthreads();
        if (tid == 0) {
          double tot = 0.0;
          for (int i = 0; i < In; ++i) tot = __dadd_rn(tot, scr[i]);
          misc[1] = tot;
          if (!(tot > 0.0)) latch_status(D.status, kStatusNumeric);
        }
        __syncthreads();
        const double tot = misc[1];
        for (int i = tid; i < In; i += NT) {
          const double p = __ddiv_rn(scr[i], tot);
          D.prob[n][i] = p;
          wsc[i] = __double2ull_rn(__dmul_rn(p, 4503599627370496.0));  // * 2^52, exact
        }
        __syncthreads();
        scan_u64_warp0(wsc, In);
        __syncthreads();
        for (int i = tid; i < In; i += NT) D.cdf[n][i] = wsc[i];
      }
      cluster.sync();
    }
  }
  if constexpr (kTC) {
    tc_fence_before();
    __syncthreads();
    if (tid < 32) tmem_dealloc(tbase, 512);
  }
}

template <typename T, typename XT, int RMAX, int NPC, bool SC>
cudaError_t step_prepare_t(const StepLayout &lay) {
  auto k = step_cluster_kernel<T, XT, RMAX, NPC, SC>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename T, typename XT, int RMAX, int NPC, bool SC>
cudaError_t step_launch_t(const ProbDesc *descs, int nprob, const StepLayout &lay, int threads, long long t0,
                          int nsteps, const long long *t_dev, cudaStream_t s) {
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
  return cudaLaunchKernelEx(&cfg, step_cluster_kernel<T, XT, RMAX, NPC, SC>, descs, lay, t0, nsteps, t_dev);
}

// One translation unit per (core type, fiber type, pieces, scaled variant
// compiled in) instantiates the four chain-row lengths, so that the variants
// compile in parallel.
#define TRSGD_STEP_INSTANTIATE_R(T, XT, R, NPC, SC)                                                      \
  template cudaError_t step_prepare_t<T, XT, R, NPC, SC>(const StepLayout &);                            \
  template cudaError_t step_launch_t<T, XT, R, NPC, SC>(const ProbDesc *, int, const StepLayout &, int, \
                                                        long long, int, const long long *, cudaStream_t);
#define TRSGD_STEP_INSTANTIATE(T, XT, NPC, SC)      \
  TRSGD_STEP_INSTANTIATE_R(T, XT, 4, NPC, SC)       \
  TRSGD_STEP_INSTANTIATE_R(T, XT, 8, NPC, SC)       \
  TRSGD_STEP_INSTANTIATE_R(T, XT, 12, NPC, SC)      \
  TRSGD_STEP_INSTANTIATE_R(T, XT, 16, NPC, SC)

}  // namespace trsgd
