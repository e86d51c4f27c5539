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
//                           as BF16 pieces, row-major and transposed;
//   3. grid_gemm_kernel     E = G_n Z^T - X_S, weighted (residual epilogue
//                           reads the fibers straight from the mode-major
//                           copy of X);
//   4. grid_gemm_kernel     partial gradients (E D) Z over slices of the
//                           samples (split-K);
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
  int I[kMaxOrder], R[kMaxOrder];
  unsigned long long seed;
  long long t;
  const float *cores[kMaxOrder];
  long long *col;                       // [J] fiber column of X_[n]
  __nv_bfloat16 *Z[3];                  // [Jp][ldz] row-major pieces
  __nv_bfloat16 *ZT[3];                 // [QTp][ldzt] transposed pieces
  long long ldz, ldzt;
  int *dbg_idx;                         // [J][N] (-1 at n)
  double *dbg_pf;                       // [J]
  float *dbg_z;                         // [J][Q]
  int *dbg_n;
};

constexpr int kGridRmax = 32;
constexpr int kGridWarps = 2;

__global__ void __launch_bounds__(32 * kGridWarps) grid_samples_kernel(GridSampleArgs a) {
  __shared__ float Pbuf[kGridWarps][2][kGridRmax][kGridRmax + 1];
  __shared__ float Sbuf[kGridWarps][kGridRmax][kGridRmax + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = a.N, n = a.n, L = N - 1;
  int order[kMaxOrder];
#pragma unroll
  for (int s = 0; s < kMaxOrder; ++s) order[s] = (s < L) ? (n + 1 + s) % N : 0;
  if (a.rec && blockIdx.x == 0 && threadIdx.x == 0) *a.dbg_n = n;
  const int Rn = a.R[n], Rn1 = a.R[(n + 1) % N];
  for (int j = blockIdx.x * kGridWarps + warp; j < a.J; j += gridDim.x * kGridWarps) {
    // slice indices of the L cores in ring order, one lane per core
    int myi = 0;
    if (lane < L) {
      const int k = order[lane];
      const uint64_t u = draw_u64(a.seed, a.t, kStreamF, k, (uint32_t)j);
      myi = (int)mulhi64(u, (uint64_t)a.I[k]);
    }
    int idx[kMaxOrder];
#pragma unroll
    for (int s = 0; s < kMaxOrder; ++s) idx[s] = __shfl_sync(0xffffffffu, myi, s);
    if (lane == 0) {
      long long col = 0, st = 1;
      double pf = 1.0;
      for (int s = 0; s < L; ++s) {
        const int k = order[s];
        col += (long long)idx[s] * st;
        st *= a.I[k];
        pf = __dmul_rn(pf, __ddiv_rn(1.0, (double)a.I[k]));
      }
      a.col[j] = col;
      if (a.rec) {
        a.dbg_pf[j] = pf;
        for (int k = 0; k < N; ++k) a.dbg_idx[(size_t)j * N + k] = -1;
        for (int s = 0; s < L; ++s) a.dbg_idx[(size_t)j * N + order[s]] = idx[s];
      }
    }
    // P = G_{n+1}(i) ... G_{n-1}(i): R_{n+1} x R_n, one lane per column
    float(*P)[kGridRmax + 1] = Pbuf[warp][0];
    float(*Pn)[kGridRmax + 1] = Pbuf[warp][1];
    float(*S)[kGridRmax + 1] = Sbuf[warp];
    {
      const int k = order[0], Ra = a.R[k], Rb = a.R[(k + 1) % N];
      const float *g = a.cores[k] + (size_t)idx[0] * Ra * Rb;
      for (int e = lane; e < Ra * Rb; e += 32) P[e % Ra][e / Ra] = __ldcg(g + e);   // (a, b) at a + b Ra
    }
    for (int s = 1; s < L; ++s) {
      const int k = order[s], Ra = a.R[k], Rb = a.R[(k + 1) % N];
      const float *g = a.cores[k] + (size_t)idx[s] * Ra * Rb;
      __syncwarp();
      for (int e = lane; e < Ra * Rb; e += 32) S[e / Ra][e % Ra] = __ldcg(g + e);   // S[b][a] = G_k(a, b)
      __syncwarp();
      if (lane < Rb) {
        for (int r = 0; r < Rn1; ++r) {
          float acc = 0.f;
          for (int c = 0; c < Ra; ++c) acc = fmaf(P[r][c], S[lane][c], acc);
          Pn[r][lane] = acc;
        }
      }
      __syncwarp();
      float(*tmp)[kGridRmax + 1] = P;
      P = Pn;
      Pn = tmp;
    }
    __syncwarp();
    // Z(j, r + r' R_n) = P(r', r); zero the padding columns [Q, Qp)
    for (int q = lane; q < a.Qp; q += 32) {
      float v = 0.f;
      if (q < a.Q) {
        const int rp = q / Rn, r = q - rp * Rn;
        v = P[rp][r];
        if (a.rec) a.dbg_z[(size_t)j * a.Q + q] = v;
      }
      __nv_bfloat16 p[3];
      bf16_pieces(v, a.np, p);
      for (int pc = 0; pc < a.np; ++pc) {
        a.Z[pc][(size_t)j * a.ldz + q] = p[pc];
        if (q < a.Q) a.ZT[pc][(size_t)q * a.ldzt + j] = p[pc];
      }
    }
  }
}

// ---- 3/4. streaming tcgen05 GEMM -------------------------------------------
// D(m, n) = sum_k A(m, k) B(n, k) over the products of operand pieces
// (pa, pb) with pa + pb <= maxord.  A: M x K, B: N x K, both K-major BF16
// (row stride lda / ldb elements, buffers padded so that every tile read is
// in bounds).  Tile 128 x NT, K in chunks of 64 through a ring of S
// shared-memory stages filled by cp.async (the loads of chunk c + S - 2 are
// issued after the MMAs of chunk c - 2 completed, so the tensor pipe always
// has the next chunk queued); one thread issues the MMAs, accumulators in TMEM.
struct GridGemmArgs {
  const __nv_bfloat16 *A[3];
  const __nv_bfloat16 *B[3];
  long long lda, ldb;
  int npa, npb, maxord;
  int kchunks, kper;       // chunks of 64 along K in total / per split (blockIdx.z)
  int NT, S;               // N tile (multiple of 16, <= 256), pipeline stages (2..4)
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
};

__host__ __device__ inline size_t grid_gemm_stage_bytes(int npa, int npb, int NT) {
  return (size_t)npa * 128 * 128 + (size_t)npb * NT * 128;
}

__global__ void __launch_bounds__(128) grid_gemm_kernel(GridGemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bars[5];   // [0..3] MMA completion per stage, [4] spare
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * a.NT;
  const int kbeg = blockIdx.z * a.kper, kend = min(kbeg + a.kper, a.kchunks);
  const int nck = max(0, kend - kbeg);
  const size_t stage = grid_gemm_stage_bytes(a.npa, a.npb, a.NT);
  const int S = a.S, P = S - 2;   // prefetch distance
  if (tid == 0) {
    for (int s = 0; s < 4; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  auto load_chunk = [&](int c) {
    unsigned char *st = smem + (size_t)(c % S) * stage;
    const long long k0 = (long long)(kbeg + c) * 64;
    for (int pa = 0; pa < a.npa; ++pa) {
      const __nv_bfloat16 *src = a.A[pa] + (long long)m0 * a.lda + k0;
      unsigned char *dst = st + (size_t)pa * 16384;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + 128 * u, r = e >> 3, kc = e & 7;
        cp_async16(dst + kmaj_off(r, kc * 8, 8), src + (long long)r * a.lda + kc * 8);
      }
    }
    for (int pb = 0; pb < a.npb; ++pb) {
      const __nv_bfloat16 *src = a.B[pb] + (long long)n0 * a.ldb + k0;
      unsigned char *dst = st + (size_t)a.npa * 16384 + (size_t)pb * a.NT * 128;
      for (int e = tid; e < a.NT * 8; e += 128) {
        const int r = e >> 3, kc = e & 7;
        cp_async16(dst + kmaj_off(r, kc * 8, 8), src + (long long)r * a.ldb + kc * 8);
      }
    }
  };
  auto wait_mma = [&](int c) {   // MMAs of chunk c have completed
    if (!mbar_wait_bounded(&bars[c % S], (uint32_t)((c / S) & 1), kGridWaitLimit)) latch_status(a.status, kStatusTimeout);
  };
  const uint32_t idesc = umma_idesc_bf16(128, a.NT, 0, 0);

  for (int c = 0; c < P; ++c) {   // always P groups, so that group c holds chunk c
    if (c < nck) load_chunk(c);
    cp_async_commit();
  }
  for (int c = 0; c < nck; ++c) {
    const int cn = c + P;
    if (cn < nck) {
      if (cn >= S) wait_mma(cn - S);
      load_chunk(cn);
    }
    cp_async_commit();
    if (P == 2) cp_async_wait_n<2>();
    else if (P == 1) cp_async_wait_n<1>();
    else cp_async_wait_n<0>();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sb = smem_u32(smem + (size_t)(c % S) * stage);
      bool first = (c == 0);
      for (int ks = 0; ks < 4; ++ks) {
        for (int pa = 0; pa < a.npa; ++pa)
          for (int pb = 0; pb < a.npb; ++pb) {
            if (pa + pb > a.maxord) continue;
            const uint64_t da = umma_desc(sb + pa * 16384 + ks * 256, 128, 1024);
            const uint64_t db = umma_desc(sb + a.npa * 16384 + pb * a.NT * 128 + ks * 256, 128, 1024);
            umma_bf16(tbase, da, db, idesc, !first);
            first = false;
          }
      }
      umma_commit(&bars[c % S]);
    }
  }
  if (nck > 0) wait_mma(nck - 1);
  tc_fence_after();

  // epilogue: thread = accumulator row (TMEM lane), 8 columns per load
  const int row = warp * 32 + lane, m = m0 + row;
  for (int cb = 0; cb < a.NT / 8; ++cb) {
    float v[8];
    if (nck > 0) {
      tmem_ld8(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 8), v);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0.f;
    }
    const int nb = n0 + cb * 8;
    if (a.mode == 0) {
      if (m < a.Mv) {
        float *dst = a.C + (long long)blockIdx.z * a.cstride + (long long)m * a.ldc;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (nb + u < a.Nv) dst[nb + u] = v[u];
      }
    } else {
      __nv_bfloat16 pe[3][8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = nb + u;
        float ew = 0.f;
        if (m < a.Mv && j < a.Nv) {
          const long long xo = a.col[j] * a.ldx + m;
          const float x = a.x_bf16 ? __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(a.xmode) + xo))
                                   : __ldg(static_cast<const float *>(a.xmode) + xo);
          const float e = v[u] - x;
          if (a.dbg_e) a.dbg_e[(long long)j * a.Mv + m] = e;
          ew = e * a.w;
        }
        __nv_bfloat16 p[3];
        bf16_pieces(ew, a.npe, p);
#pragma unroll
        for (int pc = 0; pc < 3; ++pc) pe[pc][u] = p[pc];
      }
      for (int pc = 0; pc < a.npe; ++pc)
        *reinterpret_cast<uint4 *>(a.E[pc] + (long long)m * a.lde + nb) = *reinterpret_cast<const uint4 *>(pe[pc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
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

size_t grid_gemm_smem(int npa, int npb, int NT, int S) { return grid_gemm_stage_bytes(npa, npb, NT) * S; }

// widest N tile with at least two pipeline stages: 256 for one piece, 128 for three
int grid_nt_max(int np) { return np == 1 ? 256 : 128; }

// stages that fit in `budget` bytes (2..4), 0 if not even two
static int grid_stages(int npa, int npb, int NT) {
  const size_t st = grid_gemm_stage_bytes(npa, npb, NT), budget = 200 * 1024;
  const int s = (int)std::min<size_t>(4, budget / st);
  return s >= 2 ? s : 0;
}

cudaError_t grid_prepare_gemm() {
  return cudaFuncSetAttribute(grid_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// one iteration t of the grid path on mode n
cudaError_t launch_grid_step(const GridPath &g, const ProbDesc &D, int n, long long t, int rec, cudaStream_t s) {
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  const int Ip = (In + 127) / 128 * 128, Qp = (Q + 63) / 64 * 64;
  const int np = g.np;
  cudaError_t e;
  // 1. operand pieces of G_n
  {
    const long long total = (long long)Ip * Qp;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    grid_prepare_kernel<<<blocks, 256, 0, s>>>(static_cast<const float *>(D.cores[n]), In, Q, Ip, Qp, g.ldg, np,
                                               g.Gp[0], g.Gp[1], g.Gp[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 2. samples and Z
  {
    GridSampleArgs sa = {};
    sa.N = N;
    sa.n = n;
    sa.J = D.J;
    sa.Q = Q;
    sa.Qp = Qp;
    sa.np = np;
    sa.rec = rec;
    for (int k = 0; k < N; ++k) {
      sa.I[k] = D.I[k];
      sa.R[k] = D.R[k];
      sa.cores[k] = static_cast<const float *>(D.cores[k]);
    }
    sa.seed = D.seed;
    sa.t = t;
    sa.col = g.col;
    for (int p = 0; p < 3; ++p) {
      sa.Z[p] = g.Zp[p];
      sa.ZT[p] = g.ZTp[p];
    }
    sa.ldz = g.ldz;
    sa.ldzt = g.ldzt;
    sa.dbg_idx = D.dbg_idx;
    sa.dbg_pf = D.dbg_pf;
    sa.dbg_z = static_cast<float *>(D.dbg_z);
    sa.dbg_n = D.dbg_n;
    const int blocks = (int)std::min<long long>((D.J + kGridWarps - 1) / kGridWarps, 8 * grid_sm_count());
    grid_samples_kernel<<<blocks, 32 * kGridWarps, 0, s>>>(sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int maxord = np == 1 ? 0 : 2;
  // 3. residual: E = G_n Z^T - X_S (M = Ip, N = Jp, K = Qp), weighted, as pieces
  {
    GridGemmArgs ga = {};
    for (int p = 0; p < 3; ++p) {
      ga.A[p] = g.Gp[p];
      ga.B[p] = g.Zp[p];
      ga.E[p] = g.Ep[p];
    }
    ga.lda = g.ldg;
    ga.ldb = g.ldz;
    ga.npa = ga.npb = np;
    ga.maxord = maxord;
    ga.kchunks = Qp / 64;
    ga.kper = ga.kchunks;
    ga.NT = g.nt_res;
    ga.S = grid_stages(np, np, ga.NT);
    if (ga.S < 2) return cudaErrorInvalidConfiguration;
    ga.mode = 1;
    ga.Mv = In;
    ga.Nv = D.J;
    ga.xmode = D.xmode[n];
    ga.ldx = D.ldx[n];
    ga.x_bf16 = g.x_bf16;
    ga.col = g.col;
    ga.w = g.w;
    ga.lde = g.lde;
    ga.npe = np;
    ga.dbg_e = rec ? static_cast<float *>(D.dbg_e) : nullptr;
    ga.status = D.status;
    dim3 grid(Ip / 128, g.Jp / ga.NT, 1);
    grid_gemm_kernel<<<grid, 128, grid_gemm_smem(np, np, ga.NT, ga.S), s>>>(ga);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 4. partial gradients: (E D) Z over slices of the samples (M = Ip, N = Q, K = Jp)
  const int ntmax = grid_nt_max(np);
  const int ntile = (Q + ntmax - 1) / ntmax;
  const int NT = (((Q + ntile - 1) / ntile) + 15) / 16 * 16;
  int splits = 1;
  {
    const int tiles = (Ip / 128) * ntile, kch = g.Jp / 64;
    splits = std::max(1, std::min(std::min(g.max_splits, kch), (grid_sm_count() + tiles - 1) / tiles));
    const int kper = (kch + splits - 1) / splits;
    splits = (kch + kper - 1) / kper;
    GridGemmArgs ga = {};
    for (int p = 0; p < 3; ++p) {
      ga.A[p] = g.Ep[p];
      ga.B[p] = g.ZTp[p];
    }
    ga.lda = g.lde;
    ga.ldb = g.ldzt;
    ga.npa = ga.npb = np;
    ga.maxord = maxord;
    ga.kchunks = kch;
    ga.kper = kper;
    ga.NT = NT;
    ga.S = grid_stages(np, np, NT);
    if (ga.S < 2) return cudaErrorInvalidConfiguration;
    ga.mode = 0;
    ga.C = g.gpart;
    ga.ldc = Q;
    ga.cstride = (long long)In * Q;
    ga.Mv = In;
    ga.Nv = Q;
    ga.status = D.status;
    dim3 grid(Ip / 128, ntile, splits);
    grid_gemm_kernel<<<grid, 128, grid_gemm_smem(np, np, NT, ga.S), s>>>(ga);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 5. update
  {
    GridUpdateArgs ua = {};
    ua.gpart = g.gpart;
    ua.cstride = (long long)In * Q;
    ua.splits = splits;
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
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// buffer sizes of the grid path for problem c; fills the layout fields of g
void grid_layout(const int *I, const int *R, int N, int J, int np, GridPath &g) {
  int Imax = 1, Qmax = 1;
  for (int k = 0; k < N; ++k) {
    Imax = std::max(Imax, I[k]);
    Qmax = std::max(Qmax, R[k] * R[(k + 1) % N]);
  }
  g.np = np;
  g.nt_res = grid_nt_max(np);
  g.Jp = (J + 255) / 256 * 256;
  g.Ip = (Imax + 127) / 128 * 128;
  g.Qp = (Qmax + 63) / 64 * 64;
  g.QTp = (Qmax + 255) / 256 * 256;
  g.ldg = g.Qp;
  g.ldz = g.Qp;
  g.ldzt = g.Jp;
  g.lde = g.Jp;
  g.max_splits = 16;
  g.gpart_elems = (size_t)g.max_splits * Imax * Qmax;
}

}  // namespace trsgd
