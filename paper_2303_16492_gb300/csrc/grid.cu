// Whole-GPU ("grid") path of one TR-BRSGD iteration, for problems beyond the
// fused cluster kernel (large ranks R_n R_{n+1}, many samples): the
// iteration is a short sequence of kernels over all SMs, with the two big
// contractions of Eq. S_gradient on the 5th-generation tensor cores.
//
//   1. grid_prepare_kernel  G_n (FP32) -> BF16 operand pieces, zero-padded;
//   2. grid_samples_kernel  one warp per sample: slice indices (Philox,
//                           Algorithm 2, the same counters as the fused
//                           kernel), fiber column, and the sampled subchain
//                           row Z(j, r + r' R_n) = P_j(r', r) (Def. subchain)
//                           as BF16 pieces, row-major [j][q];
//   3. grid_gemm_kernel     E = G_n Z^T - X_S, weighted (residual epilogue
//                           reads the fibers straight from the mode-major
//                           copy of X);
//   4. grid_gemm_kernel     partial gradients (E D) Z over slices of the
//                           samples (split-K; Z read MN-major, no transpose);
//   5. grid_update_kernel   fixed-order sum of the partials, step rule
//                           (fixed alpha or AdaGrad), update of G_n.
//
// Precision: an operand is held as np BF16 "pieces" whose sum approximates
// the FP32 value (each piece the BF16 rounding of what the previous ones
// left).  np = 1 is the BF16-mixed mode; np = 3 (24 significant bits) with
// the six products of total piece order <= 2 reproduces an FP32 contraction
// to about 2^-24 relative per term, accumulated in FP32 in tensor memory.
#include "common.cuh"
#include "internal.h"
#include "nvtx.h"

#include <cuda_bf16.h>

#include <algorithm>

namespace trsgd {

namespace {

constexpr long long kGridWaitLimit = 1LL << 24;

__device__ __forceinline__ void bf16_pieces(float x, int np, __nv_bfloat16 (&p)[3]) {
  float r = x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p[k] = __float2bfloat16_rn(k < np ? r : 0.f);
    r -= __bfloat162float(p[k]);
  }
}

template <int N> __device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

}  // namespace

// ---- 1. G_n -> operand pieces [Ip][ldq], zero outside I_n x Q ----------------
__global__ void grid_prepare_kernel(const float *__restrict__ G, int In, int Q, int Ip, int Qp, long long ldq,
                                    int np, __nv_bfloat16 *g0, __nv_bfloat16 *g1, __nv_bfloat16 *g2) {
  const long long total = (long long)Ip * Qp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / Qp), q = (int)(e - (long long)i * Qp);
    const float v = (i < In && q < Q) ? __ldcg(G + (size_t)i * Q + q) : 0.f;
    __nv_bfloat16 p[3];
    bf16_pieces(v, np, p);
    const size_t o = (size_t)i * ldq + q;
    g0[o] = p[0];
    if (np > 1) {
      g1[o] = p[1];
      g2[o] = p[2];
    }
  }
}

// ---- 2. samples and sampled subchain rows ---------------------------------
struct GridSampleArgs {
  int N, n, J, Q, Qp, np, rec;
  int j0, j1;                           // sample range of this launch
  int stream;                           // Philox stream: F (fibers drawn) or H (Hessian batch)
  int I[kMaxOrder], R[kMaxOrder];
  unsigned long long seed;
  long long t;
  const float *cores[kMaxOrder];
  long long *col;                       // [J] fiber column of X_[n]
  __nv_bfloat16 *Z[3];                  // [Jp][ldz] row-major pieces
  long long ldz;
  int *dbg_idx;                         // [J][N] (-1 at n)
  double *dbg_pf;                       // [J]
  float *dbg_z;                         // [J][Q]
  int *dbg_n;
  int bound[kMaxOrder];                 // debug build: upper bounds of the index checks
  int *status;
};

constexpr int kGridRmax = 32;
constexpr int kSpc = 8;             // samples per CTA, one warp each
constexpr int kSmpThreads = 32 * kSpc;

// floats of one staged slice (column-major c + b R_k, as in memory), padded to
// a multiple of 4 so that every staged slice starts on a 16-byte boundary
__host__ __device__ inline int smp_mat(int rmax) { return (rmax * rmax + 3) & ~3; }
constexpr int kProwPitch = kGridRmax + 1;   // a lane's row of P between two factors (odd pitch)
// two staging buffers (this factor, the next) of kSpc slices, per warp np
// rows of Z (BF16) assembled before the row is stored, and for chains of
// more than two factors (N > 3) the lanes' rows of P between two factors
__host__ __device__ inline size_t smp_pb_floats(int N) { return N > 3 ? (size_t)kSpc * 32 * kProwPitch : 0; }
size_t grid_samples_smem(int rmax, int Qp, int np, int N) {
  return (size_t)2 * kSpc * smp_mat(rmax) * sizeof(float) + (size_t)kSpc * np * Qp * sizeof(__nv_bfloat16) +
         smp_pb_floats(N) * sizeof(float);
}

// n / d for n d < 2^32 as the high word of n * ceil(2^32 / d) (division by an
// invariant integer, Granlund and Montgomery, PLDI 1994)
struct FastDiv {
  unsigned d, m;
  __device__ explicit FastDiv(unsigned dv) : d(dv), m(0xFFFFFFFFu / dv + 1u) {}
  __device__ __forceinline__ unsigned div(unsigned n) const { return d == 1u ? n : __umulhi(n, m); }
};

// (row r' of P) S for a staged slice S (Ra x Rb, column-major): the lane's
// row of P is in registers, the columns of S are read as broadcasts (16-byte
// loads when Ra is a multiple of 4, i.e. when every column starts on a
// 16-byte boundary), each output summed c = 0 .. Ra-1 in order and handed to
// emit(r, value) as soon as it is formed.
template <typename Emit>
__device__ __forceinline__ void chain_row(const float (&prow)[kGridRmax], const float *S, int Ra, int Rb, Emit emit) {
  // the outputs in a loop (the code stays small enough for the instruction
  // cache), each inner product unrolled against the registers as four
  // interleaved partial sums (groups of four terms, modulo 4) added pairwise:
  // four independent FMA chains in flight instead of one
  if ((Ra & 3) == 0) {
    const int Ra4 = Ra >> 2;
#pragma unroll 1
    for (int r = 0; r < Rb; ++r) {
      const float4 *col = reinterpret_cast<const float4 *>(S + r * Ra);
      float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c4 = 0; c4 < kGridRmax / 4; ++c4)
        if (c4 < Ra4) {
          const float4 sv = col[c4];
          float &x = a[c4 & 3];
          x = fmaf(prow[4 * c4], sv.x, x);
          x = fmaf(prow[4 * c4 + 1], sv.y, x);
          x = fmaf(prow[4 * c4 + 2], sv.z, x);
          x = fmaf(prow[4 * c4 + 3], sv.w, x);
        }
      emit(r, (a[0] + a[1]) + (a[2] + a[3]));
    }
  } else {
#pragma unroll 1
    for (int r = 0; r < Rb; ++r) {
      const float *col = S + r * Ra;
      float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kGridRmax; ++c)
        if (c < Ra) a[(c >> 2) & 3] = fmaf(prow[c], col[c], a[(c >> 2) & 3]);
      emit(r, (a[0] + a[1]) + (a[2] + a[3]));
    }
  }
}

// kSpc samples per CTA, one warp per sample: the L = N - 1 slice indices of
// each sample (one thread per (sample, factor) draw) and its fiber column;
// the slices of every sample staged by asynchronous copies exactly as they
// lie in memory, factor by factor (the next factor's copies in flight while
// this one is multiplied); lane r' forms row r' of the subchain product
// P = G_{n+1}(i) G_{n+2}(i) ... G_{n-1}(i) (R_{n+1} x R_n) in registers, by
// L - 1 row-times-slice products (chain_row); then
// Z(j, r + r' R_n) = P(r', r) as np BF16 pieces, assembled row by row in
// shared memory (zero in the padding [Q, Qp)) and stored with 16-byte stores,
// row-major [j][q].
__global__ void __launch_bounds__(kSmpThreads, 3) grid_samples_kernel(GridSampleArgs a) {
  extern __shared__ __align__(16) float smp[];
  __shared__ int idx_s[kSpc][kMaxOrder];
  const int N = a.N, n = a.n, L = N - 1, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int jbase = a.j0 + blockIdx.x * kSpc;
  const int nj = min(kSpc, a.j1 - jbase);
  if (nj <= 0) return;
  int rmax = 1;
  for (int k = 0; k < N; ++k) rmax = max(rmax, a.R[k]);
  const int mat = smp_mat(rmax), np = a.np, Qp = a.Qp, Q = a.Q;
  float *stg[2] = {smp, smp + kSpc * mat};
  __nv_bfloat16 *zrow = reinterpret_cast<__nv_bfloat16 *>(smp + 2 * kSpc * mat) + (size_t)warp * np * Qp;
  // this lane's row of P between two factors (N > 3 only), after the Z rows
  float *pb = reinterpret_cast<float *>(reinterpret_cast<__nv_bfloat16 *>(smp + 2 * kSpc * mat) + (size_t)kSpc * np * Qp) +
              (size_t)(warp * 32 + lane) * kProwPitch;
  for (int e = tid; e < nj * L; e += kSmpThreads) {
    const int jl = e / L, sf = e - jl * L, k = (n + 1 + sf) % N;
    const uint64_t u = draw_u64(a.seed, a.t, a.stream, k, (uint32_t)(jbase + jl));
    idx_s[jl][sf] = debug_checked((int)mulhi64(u, (uint64_t)a.I[k]), a.bound[k], a.status);
  }
  __syncthreads();
  if (a.col || a.rec) {
    for (int jl = tid; jl < nj; jl += kSmpThreads) {
      const int j = jbase + jl;
      long long col = 0, st = 1;
      for (int sf = 0; sf < L; ++sf) {
        const int k = (n + 1 + sf) % N;
        col += (long long)idx_s[jl][sf] * st;
        st *= a.I[k];
      }
      if (a.col) a.col[j] = debug_checked(col, st, a.status);
      if (a.rec) {   // p_F in ring order (FP64), only for the record
        double pf = 1.0;
        for (int sf = 0; sf < L; ++sf) pf = __dmul_rn(pf, __ddiv_rn(1.0, (double)a.I[(n + 1 + sf) % N]));
        a.dbg_pf[j] = pf;
        for (int k = 0; k < N; ++k) a.dbg_idx[(size_t)j * N + k] = -1;
        for (int sf = 0; sf < L; ++sf) a.dbg_idx[(size_t)j * N + (n + 1 + sf) % N] = idx_s[jl][sf];
      }
    }
  }
  if (a.rec && blockIdx.x == 0 && tid == 0) *a.dbg_n = n;
  // slice sf of every sample, as in memory: 16-byte asynchronous copies when
  // the slices are a multiple of 4 floats long (each then starts on a 16-byte
  // boundary), else 4-byte copies; one commit group per factor
  auto stage = [&](int sf, float *dst) {
    const int k = (n + 1 + sf) % N, sz = a.R[k] * a.R[(k + 1) % N];
    const float *src = a.cores[k];
    if ((sz & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      const int q4 = sz >> 2;
      const FastDiv dq((unsigned)q4);
      for (int e = tid; e < nj * q4; e += kSmpThreads) {
        const int jl = (int)dq.div((unsigned)e), el = e - jl * q4;
        cp_async16(dst + jl * mat + 4 * el, src + (size_t)idx_s[jl][sf] * sz + 4 * el);
      }
    } else {
      const FastDiv dsz((unsigned)sz);
      for (int e = tid; e < nj * sz; e += kSmpThreads) {
        const int jl = (int)dsz.div((unsigned)e), el = e - jl * sz;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst + jl * mat + el)),
                     "l"(src + (size_t)idx_s[jl][sf] * sz + el)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  stage(0, stg[0]);
  if (L > 1) stage(1, stg[1]);
  else asm volatile("cp.async.commit_group;" ::: "memory");   // an empty group keeps the count
  const int jl = warp;
  const bool live = jl < nj;
  const int Rn1 = a.R[(n + 1) % N], Rn = a.R[n];
  float prow[kGridRmax];
  asm volatile("cp.async.wait_group 1;" ::: "memory");
  __syncthreads();
  {   // row r' = lane of the first slice G_{n+1}(i) (R_{n+1} x R_{n+2}, column-major)
    const int rc = a.R[(n + 2) % N];
    const float *S0 = stg[0] + jl * mat;
#pragma unroll
    for (int c = 0; c < kGridRmax; ++c) prow[c] = (live && lane < Rn1 && c < rc) ? S0[c * Rn1 + lane] : 0.f;
  }
  const int j = jbase + jl;
  // Z(j, r + r' R_n) = P(r', r): lane r' fills R_n entries of the warp's row
  // buffers as the last product forms them
  auto emit_z = [&](int r, float v) {
    const int q = lane * Rn + r;
    if (a.rec) a.dbg_z[(size_t)j * Q + q] = v;
    if (np == 1) {
      zrow[q] = __float2bfloat16_rn(v);
    } else {
      __nv_bfloat16 pc[3];
      bf16_pieces(v, 3, pc);
      zrow[q] = pc[0];
      zrow[Qp + q] = pc[1];
      zrow[2 * Qp + q] = pc[2];
    }
  };
  if (live)
    for (int q = Q + lane; q < Qp; q += 32)
      for (int p = 0; p < np; ++p) zrow[p * Qp + q] = __float2bfloat16_rn(0.f);
  if (L == 1 && live && lane < Rn1) {   // N = 2: P is the slice itself
#pragma unroll
    for (int r = 0; r < kGridRmax; ++r)
      if (r < Rn) emit_z(r, prow[r]);
  }
  for (int sf = 1; sf < L; ++sf) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // factor sf staged (and every warp done with the buffer the next copies go to)
    if (sf + 1 < L) stage(sf + 1, stg[(sf + 1) & 1]);
    if (live && lane < Rn1) {
      const int k = (n + 1 + sf) % N, Ra = a.R[k], Rb = a.R[(k + 1) % N];
      const float *S = stg[sf & 1] + jl * mat;
      if (sf + 1 < L) {   // the next row of P through this lane's own buffer
        chain_row(prow, S, Ra, Rb, [&](int r, float v) { pb[r] = v; });
#pragma unroll
        for (int c = 0; c < kGridRmax; ++c) prow[c] = c < Rb ? pb[c] : 0.f;
      } else {
        chain_row(prow, S, Ra, Rb, emit_z);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!live) return;
  __syncwarp();
  const int nvec = Qp / 8;   // 16-byte chunks of a row (Qp a multiple of 64)
  for (int p = 0; p < np; ++p) {
    const uint4 *src = reinterpret_cast<const uint4 *>(zrow + p * Qp);
    uint4 *dst = reinterpret_cast<uint4 *>(a.Z[p] + (size_t)j * a.ldz);
    for (int v = lane; v < nvec; v += 32) dst[v] = src[v];
  }
}

// ---- 3/4. tcgen05 GEMM fed by TMA --------------------------------------------
// D(m, n) = sum_k A(m, k) B(n, k) over the products of operand pieces
// (pa, pb) with pa + pb <= maxord.  A: M x K, B: N x K, both K-major BF16
// in global memory, described by 2-D tensor maps (boxes of 64 K-elements x
// 128 rows for A and x NT rows for B, 128-byte swizzle).  Tile 128 x NT, K in
// chunks of 64 through a ring of S shared-memory stages: one thread issues
// the TMA copies (completion on a "full" barrier per stage) and the MMAs
// (completion on an "empty" barrier per stage); the MMAs of chunk c are
// queued before the thread waits for chunk c - 1 to finish and refills that
// stage, so the tensor pipe always has work.  Accumulators in TMEM; every
// wait is bounded and a timeout latches TRSGD_ETIMEOUT.
struct __align__(64) GridGemmArgs {
  CUtensorMap tmA[3];
  CUtensorMap tmB[3];
  int npa, npb, maxord;
  int kchunks, kper;       // chunks of 64 along K in this launch / per split (blockIdx.z)
  int kbase;               // first chunk of K (sample range of the launch)
  int nbase;               // first output column (residual: first sample of the range)
  int NT, S;               // N tile (multiple of 16, <= 256), pipeline stages (2..4)
  int xpre;                // residual: gather the X tile at kernel start into its own region after the stages
  int mode;                // 0: FP32 partials C[z][m][n]; 1: residual epilogue
  float *C;
  long long ldc, cstride;
  int Mv, Nv;              // valid rows / columns of the output
  // residual epilogue: E(i, j) = D(i, j) - X(col_j, i), Ew = w E as pieces
  const void *xmode;
  long long ldx;
  int x_bf16;
  const long long *col;
  float w;
  __nv_bfloat16 *E[3];
  long long lde;
  int npe;
  float *dbg_e;            // [J][In] or null
  int *status;
  // Gram partials: only tiles that hold an entry (a, b) of the 32 x 32 block
  // lower triangle (block(a) >= block(b)), the entries the factorisation reads
  int lower_only;
};

__host__ __device__ inline size_t grid_gemm_stage_bytes(int npa, int npb, int NT) {
  return (size_t)npa * 128 * 128 + (size_t)npb * NT * 128;
}

namespace {

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand tile with 128-byte swizzle: rows of 128 bytes, 8-row atoms
// 1024 bytes apart (SBO); the K offset inside the row is added to the start
// address; layout type 2 (128-byte swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// 32 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

constexpr int kGemmThreads = 256;   // 2 warps per TMEM lane quarter in the epilogue

__global__ void __launch_bounds__(kGemmThreads) grid_gemm_kernel(const __grid_constant__ GridGemmArgs a) {
  // scalar arguments in registers: inside the lambdas below a reference to the
  // parameter struct would turn every field access into a generic load
  const int npa = a.npa, npb = a.npb, maxord = a.maxord, NT = a.NT, mode = a.mode, Mv = a.Mv, Nv = a.Nv;
  const int x_bf16 = a.x_bf16, npe = a.npe;
  const float w = a.w;
  float *const dbg_e = a.dbg_e;
  float *const Cout = a.C;
  const long long ldx = a.ldx, lde = a.lde, ldc = a.ldc, cstride = a.cstride;
  const unsigned char *const xmode = static_cast<const unsigned char *>(a.xmode);
  __nv_bfloat16 *const Eo[3] = {a.E[0], a.E[1], a.E[2]};
  const CUtensorMap *const tmA = a.tmA, *const tmB = a.tmB;
  int *const status = a.status;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[4], empty[4];
  __shared__ uint32_t tslot;
  __shared__ int last_s, bad_s;
  __shared__ long long col_s[256];   // residual epilogue: fiber columns of the tile's samples
  // the 128-byte swizzle repeats every 1024 bytes: align the stage ring to it
  unsigned char *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = a.nbase + blockIdx.y * NT;
  if (a.lower_only && (m0 + 127) / 32 < n0 / 32) return;   // a tile above the block diagonal: never read
  const int kbeg = a.kbase + blockIdx.z * a.kper, kend = min(kbeg + a.kper, a.kbase + a.kchunks);
  const int nck = max(0, kend - kbeg);
  const size_t stage = grid_gemm_stage_bytes(npa, npb, NT);
  const int S = a.S;
  const uint32_t tx_bytes = (uint32_t)stage;
  if (tid == 0) {
    for (int s = 0; s < 4; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    fence_mbar_init();
    last_s = -1;
    bad_s = 0;
  }
  if (warp == 0) tmem_alloc(&tslot, 256);
  if (mode == 1)
    for (int jl = tid; jl < NT; jl += kGemmThreads) col_s[jl] = (n0 + jl < Nv) ? a.col[n0 + jl] : 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  // residual epilogue: the CTA's X tile (NT fibers x 128 rows, xs[jl][row]) by
  // one burst of cp.async, either now into its own region (overlapping the
  // main loop) or after the main loop into the freed stage memory
  const int sx = x_bf16 ? 2 : 4;
  unsigned char *xs = smem + (a.xpre ? (size_t)S * stage : 0);
  auto gather_x = [&]() {
    const int cpc = 128 * sx / 16;   // 16-byte chunks per fiber segment
    for (int e = tid; e < NT * cpc; e += kGemmThreads) {
      const int jl = e / cpc, ch = e - jl * cpc, j = n0 + jl;
      const long long ms = m0 + (long long)ch * (16 / sx);
      if (j < Nv && ms < ldx)
        cp_async16(xs + (size_t)jl * 128 * sx + ch * 16, xmode + (col_s[jl] * ldx + ms) * sx);
    }
    cp_async_commit();
  };
  if (mode == 1 && a.xpre) gather_x();

  if (tid == 0 && nck > 0) {
    auto issue = [&](int c) {   // TMA copies of chunk c into stage c % S
      unsigned char *st = smem + (size_t)(c % S) * stage;
      const int k0 = (kbeg + c) * 64;
      mbar_arrive_expect_tx(&full[c % S], tx_bytes);
      for (int pa = 0; pa < npa; ++pa) tma_load_2d(st + pa * 16384, &tmA[pa], k0, m0, &full[c % S]);
      for (int pb = 0; pb < npb; ++pb)
        tma_load_2d(st + npa * 16384 + pb * NT * 128, &tmB[pb], k0, n0, &full[c % S]);
    };
    const uint32_t idesc = umma_idesc_bf16(128, NT, 0, 0);
    int issued = 0, last = -1;
    bool bad = false;
    for (; issued < min(S, nck); ++issued) issue(issued);
    for (int c = 0; c < nck && !bad; ++c) {
      if (!mbar_wait_bounded(&full[c % S], (uint32_t)((c / S) & 1), kGridWaitLimit)) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint32_t sb = smem_u32(smem + (size_t)(c % S) * stage);
      bool first = (c == 0);
      for (int ks = 0; ks < 4; ++ks)
        for (int pa = 0; pa < npa; ++pa)
          for (int pb = 0; pb < npb; ++pb) {
            if (pa + pb > maxord) continue;
            const uint64_t da = umma_desc_sw128(sb + pa * 16384 + ks * 32);
            const uint64_t db = umma_desc_sw128(sb + npa * 16384 + pb * NT * 128 + ks * 32);
            umma_bf16(tbase, da, db, idesc, !first);
            first = false;
          }
      umma_commit(&empty[c % S]);
      last = c;
      // refill the stage of chunk c - 1 once its MMAs are done
      if (c >= 1 && issued < nck) {
        if (!mbar_wait_bounded(&empty[(c - 1) % S], (uint32_t)(((c - 1) / S) & 1), kGridWaitLimit)) {
          bad = true;
          break;
        }
        issue(issued++);
      }
    }
    if (bad) {   // let the copies in flight land before the CTA exits
      latch_status(status, kStatusTimeout);
      for (int c = last + 1; c < issued; ++c) mbar_wait_bounded(&full[c % S], (uint32_t)((c / S) & 1), kGridWaitLimit);
    }
    last_s = last;
    bad_s = bad ? 1 : 0;
  }
  __syncthreads();
  const int last = last_s;
  bool ok = !bad_s && (nck == 0 || last == nck - 1);
  if (last >= 0 && !mbar_wait_bounded(&empty[last % S], (uint32_t)((last / S) & 1), kGridWaitLimit)) {
    latch_status(status, kStatusTimeout);
    ok = false;
  }
  tc_fence_after();
  if (mode == 1) {
    if (!a.xpre) gather_x();
    cp_async_wait_n<0>();
    __syncthreads();
  }

  // epilogue: thread = accumulator row (TMEM lane) of its lane quarter; the
  // two warps of a quarter take alternate 32-column blocks (32 columns per
  // TMEM load, then 8); results go to a row-major tile in shared memory (rows
  // padded by 16 bytes: conflict-free), which whole warps then copy out row by
  // row, so the global stores are coalesced.
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane, m = m0 + row;
  const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
  const size_t xbytes = (mode == 1 && !a.xpre) ? (size_t)NT * 128 * sx : 0;   // the X tile stays below
  unsigned char *otile = smem + (xbytes + 1023) / 1024 * 1024;
  const int ldo_b = mode == 0 ? (NT * 4 + 16) : (NT * 2 + 16);   // bytes per staged row
  auto emit8 = [&](int cl, const float *v) {   // tile columns cl .. cl + 7 of this row
    if (mode == 0) {
      float4 *dst = reinterpret_cast<float4 *>(otile + (size_t)row * ldo_b + cl * 4);
      dst[0] = make_float4(v[0], v[1], v[2], v[3]);
      dst[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
      float xv[8], ew[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {   // all loads first
        const int xo = (cl + u) * 128 + row;
        xv[u] = x_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(xs)[xo])
                       : reinterpret_cast<const float *>(xs)[xo];
      }
      const bool rv = m < Mv;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool valid = rv && (n0 + cl + u < Nv);
        const float e = v[u] - xv[u];
        ew[u] = valid ? e * w : 0.f;
        xv[u] = e;
      }
      if (dbg_e)
        for (int u = 0; u < 8; ++u)
          if (rv && n0 + cl + u < Nv) dbg_e[(long long)(n0 + cl + u) * Mv + m] = xv[u];
      __nv_bfloat16 pe[3][8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        __nv_bfloat16 p[3];
        bf16_pieces(ew[u], npe, p);
#pragma unroll
        for (int pc = 0; pc < 3; ++pc) pe[pc][u] = p[pc];
      }
      for (int pc = 0; pc < npe; ++pc)
        *reinterpret_cast<uint4 *>(otile + ((size_t)pc * 128 + row) * ldo_b + cl * 2) =
            *reinterpret_cast<const uint4 *>(pe[pc]);
    }
  };
  const int nfull = NT / 32;
  for (int b = half; b < nfull; b += 2) {
    const int cb = 32 * b;
    float v[32];
    if (ok && nck > 0) {
      tmem_ld32(trow + (uint32_t)cb, v);
    } else {
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = 0.f;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) emit8(cb + 8 * g, v + 8 * g);
  }
  for (int cb = 32 * nfull + 8 * half; cb < NT; cb += 16) {
    float v[8];
    if (ok && nck > 0) {
      tmem_ld8(trow + (uint32_t)cb, v);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0.f;
    }
    emit8(cb, v);
  }
  __syncthreads();
  if (mode == 0) {   // FP32 partials: valid rows, valid columns, one warp per row
    const int ncols = min(NT, Nv - n0);
    for (int r = warp; r < 128; r += kGemmThreads / 32) {
      if (m0 + r >= Mv) break;
      const float *src = reinterpret_cast<const float *>(otile + (size_t)r * ldo_b);
      float *dst = Cout + (long long)blockIdx.z * cstride + (long long)(m0 + r) * ldc + n0;
      for (int c = lane; c < ncols; c += 32) dst[c] = src[c];
    }
  } else {             // E pieces: whole tile rows (zeros outside the valid block), 16 bytes per lane
    const int chunks = NT / 8;
    for (int pc = 0; pc < npe; ++pc)
      for (int r = warp; r < 128; r += kGemmThreads / 32) {
        const unsigned char *src = otile + ((size_t)pc * 128 + r) * ldo_b;
        __nv_bfloat16 *dst = Eo[pc] + (long long)(m0 + r) * lde + n0;
        for (int c = lane; c < chunks; c += 32)
          reinterpret_cast<uint4 *>(dst)[c] = *reinterpret_cast<const uint4 *>(src + c * 16);
      }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
}

// ---- Z^T from Z (32 x 32 tiles through shared memory) ------------------------
__global__ void grid_transpose_kernel(const __nv_bfloat16 *__restrict__ Z, long long ldz, int row0, int rows,
                                      int cols, __nv_bfloat16 *__restrict__ ZT, long long ldzt) {
  __shared__ unsigned short tile[32][34];
  const int j0 = row0 + blockIdx.x * 32, q0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const unsigned short *z = reinterpret_cast<const unsigned short *>(Z);
  unsigned short *zt = reinterpret_cast<unsigned short *>(ZT);
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, q = q0 + tx;
    tile[r][tx] = (j < rows && q < cols) ? z[(size_t)j * ldz + q] : (unsigned short)0;
  }
  __syncthreads();
  // rows past the batch end up to the next 64-sample chunk are written as
  // zeros: a contraction over the batch reads whole chunks
  const int rows_pad = (rows + 63) / 64 * 64;
  for (int r = ty; r < 32; r += 8) {
    const int q = q0 + r, j = j0 + tx;
    if (q < cols && j < rows_pad) zt[(size_t)q * ldzt + j] = tile[tx][r];
  }
}

// ---- 5. sum of the partial gradients, step rule, update ---------------------
struct GridUpdateArgs {
  const float *gpart;
  long long cstride;
  int splits, In, Q, rule, rec;
  float alpha, eta, b;
  double eps;
  float *G, *acc;
  float *dbg_g, *dbg_p;
  int *status;
};

__global__ void grid_update_kernel(GridUpdateArgs a) {
  const long long total = (long long)a.In * a.Q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int z = 0; z < a.splits; ++z) g += __ldcg(a.gpart + z * a.cstride + e);   // fixed order
    const float p = -g;
    float d;
    if (a.rule == 0) {
      d = a.alpha * p;
    } else {
      const float s = __ldcg(a.acc + e) + p * p;
      a.acc[e] = s;
      const float base = a.b + s;
      d = !(base > 0.f) ? 0.f
                        : ((a.eps == 0.0) ? a.eta / sqrtf(base) : a.eta * powf(base, (float)(-(0.5 + a.eps)))) * p;
    }
    const float nv = __ldcg(a.G + e) + d;
    if (!isfinite(nv)) latch_status(a.status, kStatusNumeric);
    a.G[e] = nv;
    if (a.rec) {
      a.dbg_g[e] = g;
      a.dbg_p[e] = p;
    }
  }
}

// ---- host side --------------------------------------------------------------
static int grid_sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// stage ring plus 1 KB to align it to the 1024-byte swizzle period
size_t grid_gemm_smem(int npa, int npb, int NT, int S) { return grid_gemm_stage_bytes(npa, npb, NT) * S + 1024; }

// widest N tile with at least two pipeline stages: 256 for one piece, 128 for three
int grid_nt_max(int np) { return np == 1 ? 256 : 128; }

// stages (2..4) that fit beside `extra` bytes in the shared-memory budget, 0 if not even two
static int grid_stages_budget(int npa, int npb, int NT, size_t extra) {
  const size_t st = grid_gemm_stage_bytes(npa, npb, NT), budget = 220 * 1024 - 1024;
  if (extra + 2 * st > budget) return 0;
  return (int)std::min<size_t>(4, (budget - extra) / st);
}

// stages that fit in `budget` bytes (2..4), 0 if not even two
static int grid_stages(int npa, int npb, int NT) {
  const size_t st = grid_gemm_stage_bytes(npa, npb, NT), budget = 220 * 1024 - 1024;
  const int s = (int)std::min<size_t>(4, budget / st);
  return s >= 2 ? s : 0;
}

cudaError_t grid_prepare_gemm() {
  cudaError_t e = cudaFuncSetAttribute(grid_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(grid_samples_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grid_samples_smem(kGridRmax, kGridRmax * kGridRmax, 3, kMaxOrder));
  if (e == cudaSuccess) e = grid_fused_prepare();
  return e;
}

// Split-K unit of a contraction over nsamples samples with `tiles` output
// tiles: at most one wave of CTAs (the stages fill most of shared memory),
// at most max_splits partials, in chunks of 64 samples rounded to a multiple
// of 256 samples so that sample ranges on unit boundaries align with every
// N tile of the residual GEMM.
static long long split_unit(const GridPath &g, long long nsamples, int tiles) {
  const long long kch = (nsamples + 255) / 256 * 4;
  const long long splits = std::max<long long>(1, std::min<long long>(std::min<long long>(g.max_splits, kch),
                                                                      g.sms / std::max(tiles, 1)));
  long long kper = (kch + splits - 1) / splits;
  kper = (kper + 3) / 4 * 4;
  return kper * 64;
}

// N tiling over the Q columns of the gradient and the Gram: with the scaled
// variant both read Z^T through the same tensor maps, so both take the
// three-piece tile width
static int gemm_ntiles(const GridPath &g, int Q, int &NT) { return grid_ntiles(Q, g.scaled ? 3 : g.np, NT); }

long long grid_split_unit(const GridPath &g, const ProbDesc &D, int n, long long nsamples) {
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  int NT = 0;
  const int ntile = gemm_ntiles(g, Q, NT);
  return split_unit(g, nsamples, ((In + 127) / 128) * ntile);
}

static int nsplits(long long j0, long long j1, long long unit) { return (int)((j1 - j0 + unit - 1) / unit); }

// Split unit of the Gram partials: the unit of the same sample batch halved
// (at most twice) while it stays a multiple of 256 samples and the Gram's
// tiles times its splits stay within one wave of the SMs. A unit of the
// gradient then holds a whole number of Gram units, so a rank's range of
// gradient units is also a range of Gram units, and the fixed-order sum of
// the Gram partials does not depend on how the ranks split the batch.
long long grid_gram_unit(const GridPath &g, const ProbDesc &D, int n, long long nsamples) {
  const int N = D.N, Q = D.R[n] * D.R[(n + 1) % N];
  int NT = 0;
  const long long tiles = (long long)((Q + 127) / 128) * grid_ntiles(Q, 3, NT);
  long long unit = grid_split_unit(g, D, n, nsamples);
  for (int halvings = 0; halvings < 2; ++halvings) {
    const long long u2 = unit / 2;
    if (u2 < 256 || u2 % 256 != 0 || tiles * ((nsamples + u2 - 1) / u2) > g.sms) break;
    unit = u2;
  }
  return unit;
}

// Z (and Z^T) of the samples [j0, j1) on Philox stream `stream`; fiber
// columns only for the F batch
static cudaError_t launch_samples(const GridPath &g, const ProbDesc &D, int n, long long t, long long j0,
                                  long long j1, int stream, int rec, cudaStream_t s, bool transpose = true) {
  NvtxRange r("grid_samples_kernel (+ transposes)");
  const int N = D.N, Q = D.R[n] * D.R[(n + 1) % N];
  const int Qp = (Q + 63) / 64 * 64;
  GridSampleArgs sa = {};
  sa.N = N;
  sa.n = n;
  sa.J = D.J;
  sa.Q = Q;
  sa.Qp = Qp;
  sa.np = g.npz;
  sa.rec = rec;
  sa.j0 = (int)j0;
  sa.j1 = (int)j1;
  sa.stream = stream;
  for (int k = 0; k < N; ++k) {
    sa.I[k] = D.I[k];
    sa.R[k] = D.R[k];
    sa.cores[k] = static_cast<const float *>(D.cores[k]);
  }
  sa.seed = D.seed;
  sa.t = t;
  sa.col = stream == kStreamF ? g.col : nullptr;
  for (int p = 0; p < 3; ++p) sa.Z[p] = g.Zp[p];
  sa.ldz = g.ldz;
  sa.dbg_idx = D.dbg_idx;
  sa.dbg_pf = D.dbg_pf;
  sa.dbg_z = static_cast<float *>(D.dbg_z);
  sa.dbg_n = D.dbg_n;
  for (int k = 0; k < N; ++k) sa.bound[k] = D.dbg_bound[k] > 0 ? D.dbg_bound[k] : D.I[k];
  sa.status = D.status;
  int rmax = 1;
  for (int k = 0; k < N; ++k) rmax = std::max(rmax, D.R[k]);
  const int blocks = (int)((j1 - j0 + kSpc - 1) / kSpc);
  grid_samples_kernel<<<blocks, kSmpThreads, grid_samples_smem(rmax, Qp, g.npz, N), s>>>(sa);
  cudaError_t e = cudaGetLastError();
  if (!transpose) return e;
  // Z^T for the gradient's K-major B operand (and both Gram operands)
  for (int p = 0; p < g.npz && e == cudaSuccess; ++p) {
    dim3 grid((unsigned)(((j1 + 63) / 64 * 64 - j0 + 31) / 32), (Q + 31) / 32);
    grid_transpose_kernel<<<grid, 256, 0, s>>>(g.Zp[p], g.ldz, (int)j0, (int)j1, Q, g.ZTp[p], g.ldzt);
    e = cudaGetLastError();
  }
  return e;
}

// Z^T Z over the samples [j0, j1) held in Z^T, one FP32 partial per unit
static cudaError_t launch_gram(const GridPath &g, int Q, long long j0, long long j1, long long unit, int n,
                               float *hout, int *status, int rec, cudaStream_t s) {
  int NT = 0;
  const int ntile = grid_ntiles(Q, 3, NT);
  GridGemmArgs ga = {};
  for (int p = 0; p < 3; ++p) {
    ga.tmA[p] = g.tmZTa[p];
    ga.tmB[p] = g.tmZT[n][p];
  }
  ga.npa = ga.npb = 3;
  ga.maxord = 2;
  ga.kbase = (int)(j0 / 64);
  ga.kchunks = (int)((j1 - j0 + 63) / 64);
  ga.kper = (int)(unit / 64);
  ga.nbase = 0;
  ga.NT = NT;
  ga.S = grid_stages(3, 3, NT);
  if (ga.S < 2) return cudaErrorInvalidConfiguration;
  ga.mode = 0;
  ga.C = hout;
  ga.ldc = Q;
  ga.cstride = (long long)Q * Q;
  ga.Mv = Q;
  ga.Nv = Q;
  ga.status = status;
  ga.lower_only = rec ? 0 : 1;   // the record keeps the whole h
  dim3 grid((unsigned)((Q + 127) / 128), ntile, nsplits(j0, j1, unit));
  grid_gemm_kernel<<<grid, kGemmThreads, grid_gemm_smem(3, 3, NT, ga.S), s>>>(ga);
  return cudaGetLastError();
}

// the scaled variant's factorisation and direction for mode n, from the
// given partial gradients and Grams
static GridScaledArgs grid_scaled_args(const GridPath &g, const ProbDesc &D, int n, const float *gparts, int gsplits,
                                       const float *hparts, int hsplits, int rec) {
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  GridScaledArgs sa = {};
  sa.hpart = hparts;
  sa.hstride = (long long)Q * Q;
  sa.hsplits = hsplits;
  sa.gpart = gparts;
  sa.gstride = (long long)In * Q;
  sa.gsplits = gsplits;
  sa.In = In;
  sa.Q = Q;
  sa.sms = g.sms;
  sa.hscale = 1.0 / (double)(g.JH > 0 ? g.JH : D.J);
  sa.damping = D.damping;
  sa.Lfac = g.Lfac;
  sa.ok = g.fac_ok;
  sa.rule = D.rule;
  sa.alpha = (float)D.alpha;
  sa.eta = (float)D.eta;
  sa.b = (float)D.b;
  sa.eps = D.eps;
  sa.G = static_cast<float *>(D.cores[n]);
  sa.acc = static_cast<float *>(D.acc[n]);
  sa.dbg_g = rec ? static_cast<float *>(D.dbg_g) : nullptr;
  sa.dbg_p = rec ? static_cast<float *>(D.dbg_p) : nullptr;
  sa.dbg_h = rec ? D.dbg_h : nullptr;
  sa.status = D.status;
  return sa;
}

cudaError_t launch_grid_partial(const GridPath &g, const ProbDesc &D, int n, long long t, long long j0,
                                long long j1, long long h0, long long h1, int rec, float *gout, float *hout,
                                cudaStream_t s, const GridScaledArgs *fork_factor) {
  NvtxRange r("grid partial sums (G pieces, samples, tcgen05 GEMMs)");
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  const int Ip = (In + 127) / 128 * 128, Qp = (Q + 63) / 64 * 64;
  const int np = g.np;
  cudaError_t e;
  const long long unit = grid_split_unit(g, D, n, D.J);
  if (j0 < 0 || j1 > D.J || j0 > j1 || (j0 % unit) != 0 || ((j1 % unit) != 0 && j1 != D.J))
    return cudaErrorInvalidValue;
  const bool fpart = j1 > j0;   // a rank may hold no sample of F but some of H
  // 1. samples of F and Z (and Z^T)
  if (fpart && (e = launch_samples(g, D, n, t, j0, j1, kStreamF, rec, s)) != cudaSuccess) return e;
  // scaled variant with H = F: the partial Grams first; the factorisation may
  // then run on the second stream beside the residual and gradient GEMMs
  if (g.scaled && g.JH == 0 && fpart) {
    if ((e = launch_gram(g, Q, j0, j1, grid_gram_unit(g, D, n, D.J), n, hout, D.status, rec, s)) != cudaSuccess)
      return e;
    if (fork_factor) {
      if ((e = cudaEventRecord(g.ev_fork, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(g.s2, g.ev_fork, 0)) != cudaSuccess) return e;
      if ((e = launch_grid_factor(*fork_factor, g.s2)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(g.ev_join, g.s2)) != cudaSuccess) return e;
    }
  }
  // 2. operand pieces of G_n (after the fork: the factorisation does not wait for them)
  if (fpart) {
    const long long total = (long long)Ip * Qp;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    grid_prepare_kernel<<<blocks, 256, 0, s>>>(static_cast<const float *>(D.cores[n]), In, Q, Ip, Qp, g.ldg, np,
                                               g.Gp[0], g.Gp[1], g.Gp[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int maxord = np == 1 ? 0 : 2;
  // 3. residual: E = G_n Z^T - X_S (M = Ip, N = the samples of the range, K = Qp), weighted, as pieces
  if (fpart) {
    GridGemmArgs ga = {};
    for (int p = 0; p < 3; ++p) ga.E[p] = g.Ep[p];
    for (int p = 0; p < np; ++p) {
      ga.tmA[p] = g.tmG[p];
      ga.tmB[p] = g.tmZ[p];
    }
    ga.npa = ga.npb = np;
    ga.maxord = maxord;
    ga.kbase = 0;
    ga.kchunks = Qp / 64;
    ga.kper = ga.kchunks;
    ga.NT = g.nt_res;
    ga.nbase = (int)j0;
    {   // X tile in its own region when at least three stages still fit beside it
      const size_t xb = (size_t)ga.NT * 128 * (g.x_bf16 ? 2 : 4);
      const int sx3 = grid_stages_budget(np, np, ga.NT, xb);
      ga.xpre = sx3 >= 3 ? 1 : 0;
      ga.S = ga.xpre ? sx3 : grid_stages(np, np, ga.NT);
    }
    if (ga.S < 2) return cudaErrorInvalidConfiguration;
    ga.mode = 1;
    ga.Mv = In;
    ga.Nv = (int)j1;
    ga.xmode = D.xmode[n];
    ga.ldx = D.ldx[n];
    ga.x_bf16 = g.x_bf16;
    ga.col = g.col;
    ga.w = g.w;
    ga.lde = g.lde;
    ga.npe = np;
    ga.dbg_e = rec ? static_cast<float *>(D.dbg_e) : nullptr;
    ga.status = D.status;
    dim3 grid(Ip / 128, (unsigned)((j1 - j0 + ga.NT - 1) / ga.NT), 1);
    grid_gemm_kernel<<<grid, kGemmThreads, grid_gemm_smem(np, np, ga.NT, ga.S) + (ga.xpre ? (size_t)ga.NT * 128 * (g.x_bf16 ? 2 : 4) : 0), s>>>(ga);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 4. partial gradients: (E D) Z over the units of the range (M = Ip, N = Q, K = samples)
  if (fpart) {
    int NT = 0;
    const int ntile = gemm_ntiles(g, Q, NT);
    GridGemmArgs ga = {};
    for (int p = 0; p < np; ++p) {
      ga.tmA[p] = g.tmE[p];
      ga.tmB[p] = g.tmZT[n][p];
    }
    ga.npa = ga.npb = np;
    ga.maxord = maxord;
    ga.kbase = (int)(j0 / 64);
    ga.kchunks = (int)((j1 - j0 + 63) / 64);
    ga.kper = (int)(unit / 64);
    ga.nbase = 0;
    ga.NT = NT;
    ga.S = grid_stages(np, np, NT);
    if (ga.S < 2) return cudaErrorInvalidConfiguration;
    ga.mode = 0;
    ga.C = gout;
    ga.ldc = Q;
    ga.cstride = (long long)In * Q;
    ga.Mv = In;
    ga.Nv = Q;
    ga.status = D.status;
    dim3 grid(Ip / 128, ntile, nsplits(j0, j1, unit));
    grid_gemm_kernel<<<grid, kGemmThreads, grid_gemm_smem(np, np, NT, ga.S), s>>>(ga);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 5. scaled variant: partial Grams of the Hessian batch (H = F: the same samples)
  if (g.scaled) {
    if (g.JH > 0) {
      const long long uh = grid_gram_unit(g, D, n, g.JH);
      if (h0 < 0 || h1 > g.JH || h0 > h1 || (h0 % uh) != 0 || ((h1 % uh) != 0 && h1 != g.JH))
        return cudaErrorInvalidValue;
      if (h1 > h0) {
        if ((e = launch_samples(g, D, n, t, h0, h1, kStreamH, 0, s)) != cudaSuccess) return e;
        if ((e = launch_gram(g, Q, h0, h1, uh, n, hout, D.status, rec, s)) != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

cudaError_t launch_grid_apply(const GridPath &g, const ProbDesc &D, int n, const float *gparts, int gsplits,
                              const float *hparts, int hsplits, int rec, cudaStream_t s) {
  NvtxRange r("grid apply (sum of the partials, direction, step rule, update)");
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  if (g.scaled) return launch_grid_scaled(grid_scaled_args(g, D, n, gparts, gsplits, hparts, hsplits, rec), s);
  GridUpdateArgs ua = {};
  ua.gpart = gparts;
  ua.cstride = (long long)In * Q;
  ua.splits = gsplits;
  ua.In = In;
  ua.Q = Q;
  ua.rule = D.rule;
  ua.rec = rec;
  ua.alpha = (float)D.alpha;
  ua.eta = (float)D.eta;
  ua.b = (float)D.b;
  ua.eps = D.eps;
  ua.G = static_cast<float *>(D.cores[n]);
  ua.acc = static_cast<float *>(D.acc[n]);
  ua.dbg_g = static_cast<float *>(D.dbg_g);
  ua.dbg_p = static_cast<float *>(D.dbg_p);
  ua.status = D.status;
  const long long total = (long long)In * Q;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  grid_update_kernel<<<blocks, 256, 0, s>>>(ua);
  return cudaGetLastError();
}

// kernels one iteration of mode n launches (the handle's launch count)
int grid_step_kernels(const GridPath &g, const ProbDesc &D, int n) {
  if (g.fz_S[n] > 0) return 3;   // G_n's pieces, the samples, the fused kernel
  // prepare, samples, transposes, residual, gradient, update; scaled: (H samples
  // and transposes,) Gram, factor and direction instead of the update
  return 4 + g.npz + (g.scaled ? (g.JH > 0 ? 3 + g.npz : 2) : 1);
}

// one iteration t of the grid path on mode n: every sample on this GPU.  BF16
// operands, plain direction, Q <= 448: G_n's pieces, the samples and one fused
// kernel (residual, gradient, cluster sum, update); otherwise partial + apply.
cudaError_t launch_grid_step(const GridPath &g, const ProbDesc &D, int n, long long t, int rec, cudaStream_t s) {
  const int S = g.fz_S[n];
  if (S > 0) {
    const int In = D.I[n], Q = D.R[n] * D.R[(n + 1) % D.N];
    const int Ip = (In + 127) / 128 * 128, Qp = (Q + 63) / 64 * 64;
    const long long total = (long long)Ip * Qp;
    {
      NvtxRange r("grid_prepare_kernel");
      grid_prepare_kernel<<<(int)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(
          static_cast<const float *>(D.cores[n]), In, Q, Ip, Qp, g.ldg, 1, g.Gp[0], g.Gp[1], g.Gp[2]);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_samples(g, D, n, t, 0, D.J, kStreamF, rec, s, false);
    if (e == cudaSuccess) {
      NvtxRange r("grid_fused_kernel");
      e = launch_grid_fused(g.tmZc, g.tmG[0], g.gpart, D, n, g.col, g.w, S, rec, s);
    }
    return e;
  }
  const long long JH = g.JH > 0 ? g.JH : D.J;
  const int gs = nsplits(0, D.J, grid_split_unit(g, D, n, D.J));
  const int hs = g.scaled ? nsplits(0, JH, grid_gram_unit(g, D, n, JH)) : 0;
  if (g.scaled && g.JH == 0 && g.s2) {   // the factorisation beside the residual and gradient GEMMs
    const GridScaledArgs sa = grid_scaled_args(g, D, n, g.gpart, gs, g.hpart, hs, rec);
    cudaError_t e = launch_grid_partial(g, D, n, t, 0, D.J, 0, 0, rec, g.gpart, g.hpart, s, &sa);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.ev_join, 0);
    if (e == cudaSuccess) e = launch_grid_direction(sa, s);
    return e;
  }
  cudaError_t e = launch_grid_partial(g, D, n, t, 0, D.J, 0, g.JH, rec, g.gpart, g.hpart, s, nullptr);
  if (e == cudaSuccess) e = launch_grid_apply(g, D, n, g.gpart, gs, g.hpart, hs, rec, s);
  return e;
}

// N tiling of the gradient GEMM over the Q columns: the number of tiles and
// their common width NT (a multiple of 16, at most grid_nt_max)
int grid_ntiles(int Q, int np, int &NT) {
  const int ntmax = grid_nt_max(np);
  const int ntile = (Q + ntmax - 1) / ntmax;
  NT = (((Q + ntile - 1) / ntile) + 15) / 16 * 16;
  return ntile;
}

// buffer sizes of the grid path for problem c; fills the layout fields of g
void grid_layout(const int *I, const int *R, int N, int J, int np, int scaled, int JH, GridPath &g) {
  int Imax = 1, Qmax = 1;
  long long zcols = 1;   // columns of Z any tile reads: the K padding of the residual, the N tiles of the gradient
  for (int k = 0; k < N; ++k) {
    Imax = std::max(Imax, I[k]);
    const int Q = R[k] * R[(k + 1) % N];
    Qmax = std::max(Qmax, Q);
    int NT = 0;
    const int ntile = grid_ntiles(Q, np, NT);
    zcols = std::max<long long>(zcols, std::max<long long>((Q + 63) / 64 * 64, (long long)ntile * NT));
  }
  g.np = np;
  g.npz = scaled ? 3 : np;
  g.scaled = scaled;
  g.JH = scaled ? JH : 0;
  g.nt_res = grid_nt_max(np);
  g.Jp = (std::max(J, g.JH) + 255) / 256 * 256;
  g.Ip = (Imax + 127) / 128 * 128;
  g.Qp = (Qmax + 63) / 64 * 64;
  g.QTp = g.Qp;
  g.ldg = g.Qp;
  g.ldz = g.Qp;
  g.ldzt = g.Jp;
  g.lde = g.Jp;
  (void)zcols;
  g.max_splits = 16;
  g.sms = grid_sm_count();
  // a range of samples yields at most max_splits + 1 partials (unit rounding)
  // (and the fused BF16 kernel's 16 slots of rows padded to a multiple of 4 columns)
  g.gpart_elems = std::max((size_t)(g.max_splits + 1) * Imax * Qmax, (size_t)16 * Imax * ((Qmax + 3) & ~3));
  g.hpart_elems = scaled ? (size_t)(4 * g.max_splits + 1) * Qmax * Qmax : 0;   // Gram units: up to 4 per unit
}

}  // namespace trsgd

namespace trsgd {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_map(EncodeTiledFn fn, CUtensorMap *map, void *base, long long rows, long long cols,
                              int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t grid_tensor_maps(const int *R, int N, GridPath &g) {
  void *fp = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fp) return e != cudaSuccess ? e : cudaErrorNotSupported;
  const EncodeTiledFn fn = reinterpret_cast<EncodeTiledFn>(fp);
  for (int p = 0; p < g.np && e == cudaSuccess; ++p) {
    if ((e = encode_map(fn, &g.tmG[p], g.Gp[p], g.Ip, g.ldg, 128)) != cudaSuccess) break;
    if ((e = encode_map(fn, &g.tmZ[p], g.Zp[p], g.Jp, g.ldz, g.nt_res)) != cudaSuccess) break;
    if (p == 0 && (e = encode_map(fn, &g.tmZc, g.Zp[0], g.Jp, g.ldz, 64)) != cudaSuccess) break;
    if ((e = encode_map(fn, &g.tmE[p], g.Ep[p], g.Ip, g.lde, 128)) != cudaSuccess) break;
  }
  // Z^T: every kept piece, as the B operand of mode n's gradient (and Gram)
  // and as the A operand of the Gram
  for (int p = 0; p < g.npz && e == cudaSuccess; ++p) {
    for (int n = 0; n < N && e == cudaSuccess; ++n) {
      int NT = 0;
      grid_ntiles(R[n] * R[(n + 1) % N], g.scaled ? 3 : g.np, NT);
      e = encode_map(fn, &g.tmZT[n][p], g.ZTp[p], g.QTp, g.ldzt, NT);
    }
    if (e == cudaSuccess && g.scaled) e = encode_map(fn, &g.tmZTa[p], g.ZTp[p], g.QTp, g.ldzt, 128);
  }
  return e;
}

}  // namespace trsgd
