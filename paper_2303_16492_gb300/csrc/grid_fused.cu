// One-kernel iteration body of the whole-GPU path for BF16 operands (the
// BF16-mixed mode, plain direction): the residual E = G_n Z^T - X_S, the
// gradient g = (E D) Z / (|F| J_n) of Eq. S_gradient, and the step rule and
// update of G_n, with no intermediate in global memory.
//
// Grid: one row tile of 128 rows of G_n per cluster, the samples split over
// the S CTAs of the cluster (S <= 16).  Each CTA
//   1. loads its 128 x Q tile of G_n in BF16 (written by the prepare kernel)
//      by TMA, in the 128-byte-swizzled K-major layout of a tcgen05 operand;
//   2. per chunk of 64 of its samples: loads the chunk's rows of Z (TMA, the
//      same swizzle), gathers the chunk's fibers of X from the mode-major
//      copy (cp.async), issues D_E = G_tile Z_chunk^T (M 128, N 64, K Q) into
//      tensor memory, turns D_E - X into the weighted residual in BF16 (the A
//      operand of the next product, written swizzled into shared memory),
//      and issues D_g += Ew Z_chunk, reading the same Z tile as an MN-major
//      operand (N = Q, K = the 64 samples), so Z is loaded once;
//   3. writes its D_g (128 x Q, FP32) into its slot of an L2-resident
//      scratch; after a cluster barrier CTA s sums rows [128 s / S,
//      128 (s+1) / S) over the S slots in increasing rank order (fixed,
//      deterministic) and applies fixed alpha or AdaGrad to those rows.
// One thread issues the TMA copies and the MMAs; every mbarrier wait is
// bounded (a timeout is latched and the operation drained by a second wait).
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

#include <cuda_bf16.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace trsgd {

namespace {

constexpr int kFzThreads = 288;          // warps 0-7: epilogue (two per TMEM lane quarter, one half of the
                                         // columns each); thread 0 issues; warp 8 gathers and sums
constexpr int kFzChunk = 64;             // samples per chunk
constexpr long long kFzWait = 1LL << 24;

__device__ __forceinline__ void fz_tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory descriptor, 128-byte swizzle: K-major (LBO unused, SBO = 8
// rows of 128 bytes) or MN-major (LBO = the byte stride between 64-element
// atoms along M/N, SBO = the stride between groups of 8 rows along K)
__device__ __forceinline__ uint64_t fz_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// byte offset of element (row r, k) in a swizzled K-major tile of 128-byte rows
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ r) & 7) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ bool fz_wait(uint64_t *bar, uint32_t parity, int *status) {
  if (mbar_wait_bounded(bar, parity, kFzWait)) return true;
  latch_status(status, kStatusTimeout);
  mbar_wait_bounded(bar, parity, kFzWait);
  return false;
}

__device__ __forceinline__ void tmem_ld32x(uint32_t taddr, float (&v)[32]) {
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

struct __align__(64) FusedArgs {
  CUtensorMap tmZ;                 // Z [Jp][ldz] BF16, boxes of 64 (q) x 64 (samples), 128-byte swizzle
  CUtensorMap tmG;                 // G_n as BF16 [Ip][ldg], boxes of 64 (q) x 128 (rows), 128-byte swizzle
  float *gpart;                    // [S][Ip][Q] per-CTA gradients of the cluster sum (L2-resident)
  const float *G;                  // G_n [In][Q], updated in place
  float *acc;                      // AdaGrad sums of core n (or null)
  const __nv_bfloat16 *xmode;      // mode-major copy of X for mode n (BF16)
  long long ldx;
  const long long *col;            // [J] fiber columns of the samples
  int In, Q, kq, J, S;             // kq = Qp / 64
  long long pstride;               // floats between two slots of gpart
  float w;                         // 1 / |F|
  int rule;
  float alpha, eta, b;
  double eps;
  float *dbg_e, *dbg_g, *dbg_p;    // records (or null)
  int *status;
};

size_t grid_fused_smem(int Q) {
  const int kq = (Q + 63) / 64;
  const size_t main = (size_t)kq * 16384 + (size_t)kq * 8192 + 16384 + 2 * (size_t)kFzChunk * 128 * 2;
  return main + 1024;
}

__global__ void __launch_bounds__(kFzThreads, 1) grid_fused_kernel(const __grid_constant__ FusedArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank(), S = a.S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * 128;
  const int In = a.In, Q = a.Q, kq = a.kq, J = a.J;
  extern __shared__ unsigned char fz_raw[];
  unsigned char *smem = fz_raw + ((1024 - (smem_u32(fz_raw) & 1023)) & 1023);
  unsigned char *As = smem;                                    // kq blocks of [128 rows][128 B]
  unsigned char *Zs = As + (size_t)kq * 16384;                 // kq blocks of [64 samples][128 B]
  unsigned char *Es = Zs + (size_t)kq * 8192;                  // [128 rows][64 samples] BF16, swizzled
  __nv_bfloat16 *Xs0 = reinterpret_cast<__nv_bfloat16 *>(Es + 16384);  // 2 x [64 fibers][128 rows]
  __shared__ uint64_t zfull, mdone, afull;
  __shared__ uint32_t tslot;
  const int nch = (J + kFzChunk - 1) / kFzChunk;
  const int c0 = nch * s / S, c1 = nch * (s + 1) / S;
  if (tid == 0) {
    mbar_init(&zfull, 1);
    mbar_init(&mdone, 1);
    mbar_init(&afull, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, 512);
  const unsigned char *xm = reinterpret_cast<const unsigned char *>(a.xmode);
  // the fibers of a chunk (cp.async, 16 x 16 B = 128 rows per fiber) into one of two buffers:
  // the next chunk's gather runs during this chunk's products
  auto gather = [&](int c, __nv_bfloat16 *dst) {
    const int j0 = c * kFzChunk;
    for (int e = tid; e < kFzChunk * 16; e += kFzThreads) {
      const int jl = e >> 4, ch = e & 15;
      const long long ms = m0 + (long long)ch * 8;
      if (j0 + jl < J && ms < a.ldx) cp_async16(dst + jl * 128 + ch * 8, xm + (__ldg(a.col + j0 + jl) * a.ldx + ms) * 2);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // the first chunk's Z rows and fibers are requested before the G tile is
  // converted, so that their latency overlaps the conversion
  if (c0 < c1) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&zfull, (uint32_t)kq * 8192);
      for (int kb = 0; kb < kq; ++kb) fz_tma_2d(Zs + (size_t)kb * 8192, &a.tmZ, kb * 64, c0 * kFzChunk, &zfull);
    }
    gather(c0, Xs0);
  }
  // 1. the BF16 G_n tile (written by the prepare kernel, zero outside In x Q):
  // kq TMA boxes of 64 columns x 128 rows, 128-byte swizzle
  if (tid == 0 && c0 < c1) {   // a CTA without samples never touches the tile
    mbar_arrive_expect_tx(&afull, (uint32_t)kq * 16384);
    for (int kb = 0; kb < kq; ++kb) fz_tma_2d(As + (size_t)kb * 16384, &a.tmG, kb * 64, m0, &afull);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tslot;                   // D_E: columns [0, 64); D_g: [64, 64 + Qp)
  const uint32_t idE = umma_idesc_bf16(128, kFzChunk, 0, 0);
  const int nA = kq * 64 > 256 ? 256 : kq * 64, nB = kq * 64 - nA;   // N of the two gradient products
  uint32_t pz = 0, pm = 0;
  bool any = false;
  for (int c = c0; c < c1; ++c) {
    const int j0 = c * kFzChunk;
    __nv_bfloat16 *Xs = Xs0 + ((c - c0) & 1) * (kFzChunk * 128);
    // Z rows of the chunk (TMA); the next chunk's fibers into the other buffer
    if (tid == 0 && c > c0) {
      mbar_arrive_expect_tx(&zfull, (uint32_t)kq * 8192);
      for (int kb = 0; kb < kq; ++kb) fz_tma_2d(Zs + (size_t)kb * 8192, &a.tmZ, kb * 64, j0, &zfull);
    }
    if (c + 1 < c1) gather(c + 1, Xs0 + ((c + 1 - c0) & 1) * (kFzChunk * 128));
    else asm volatile("cp.async.commit_group;" ::: "memory");   // an empty group keeps the count
    // residual product D_E = G_tile Z_chunk^T
    if (tid == 0) {
      if (c == c0) fz_wait(&afull, 0, a.status);
      fz_wait(&zfull, pz, a.status);
      tc_fence_after();
      for (int kb = 0; kb < kq; ++kb)
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t da = fz_desc(smem_u32(As + (size_t)kb * 16384) + ks * 32, 16, 1024);
          const uint64_t db = fz_desc(smem_u32(Zs + (size_t)kb * 8192) + ks * 32, 16, 1024);
          umma_bf16(tb, da, db, idE, kb > 0 || ks > 0);
        }
      umma_commit(&mdone);
    }
    pz ^= 1u;
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // this chunk's fibers (the next may be in flight)
    __syncthreads();
    fz_wait(&mdone, pm, a.status);
    pm ^= 1u;
    tc_fence_after();
    // weighted residual Ew = w (D_E - X) in BF16: row r of the tile per
    // thread, samples [32 half, 32 half + 32) of the chunk per warp
    if (warp < 8) {
      const int qw = warp & 3, half = warp >> 2;
      const int r = qw * 32 + lane, m = m0 + r;
      const uint32_t trow = tb + ((uint32_t)(qw * 32) << 16);
      float v[32];
      tmem_ld32x(trow + (uint32_t)(half * 32), v);
#pragma unroll
      for (int g8 = 0; g8 < 4; ++g8) {
        __nv_bfloat16 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int jl = half * 32 + g8 * 8 + u, j = j0 + jl;
          const bool valid = m < In && j < J;
          const float e = valid ? v[g8 * 8 + u] - __bfloat162float(Xs[jl * 128 + r]) : 0.f;
          if (valid && a.dbg_e) a.dbg_e[(size_t)j * In + m] = e;
          h[u] = __float2bfloat16_rn(e * a.w);
        }
        *reinterpret_cast<uint4 *>(Es + sw128_off(r, half * 32 + g8 * 8)) = *reinterpret_cast<const uint4 *>(h);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // gradient product D_g += Ew Z_chunk: A = Ew (K-major, K = 64 samples),
    // B = the Z tile read MN-major (N = q in 64-element atoms 8192 B apart,
    // K = samples in groups of 8 rows, 1024 B apart)
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idA = umma_idesc_bf16(128, nA, 0, 1), idB = umma_idesc_bf16(128, nB > 0 ? nB : 16, 0, 1);
      for (int ks = 0; ks < kFzChunk / 16; ++ks) {
        const uint64_t de = fz_desc(smem_u32(Es) + ks * 32, 16, 1024);
        umma_bf16(tb + 64, de, fz_desc(smem_u32(Zs) + ks * 2048, 8192, 1024), idA, any || ks > 0);
        if (nB > 0)
          umma_bf16(tb + 64 + nA, de, fz_desc(smem_u32(Zs + (size_t)(nA / 64) * 8192) + ks * 2048, 8192, 1024), idB,
                    any || ks > 0);
      }
      umma_commit(&mdone);
      fz_wait(&mdone, pm, a.status);   // the Z and Ew tiles are reused by the next chunk
    }
    pm ^= 1u;
    any = true;
    __syncthreads();
  }
  // 3. D_g straight from tensor memory into this CTA's slot of the L2-resident
  // scratch (rows padded to Q4 = a multiple of 4 columns: 16-byte stores; zero
  // when this CTA had no samples); after the cluster barrier, the fixed-order
  // sum over the S slots and the update of this CTA's rows
  // A tensor-memory load gives a thread one row; the 32 x 32 block a warp
  // loads goes through shared memory (the G tile is free now) and out as
  // whole 128-byte row segments, eight lanes per row. Two warps per lane
  // quarter take alternate blocks of 32 columns.
  const int Q4 = (Q + 3) & ~3;
  tc_fence_after();
  if (warp < 8) {
    const int qw = warp & 3, half = warp >> 2;
    const uint32_t trow = tb + 64 + ((uint32_t)(qw * 32) << 16);
    float *tp = reinterpret_cast<float *>(As) + warp * 32 * 33;   // [32 rows][33]
    float *slot = a.gpart + (size_t)s * a.pstride;
    const int rq = lane >> 3, c4 = (lane & 7) * 4;
    for (int cb = half; cb < kq * 2; cb += 2) {   // 32 columns per load
      float v[32];
      if (any) {
        tmem_ld32x(trow + (uint32_t)(cb * 32), v);
      } else {
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) tp[lane * 33 + u] = v[u];
      __syncwarp();
      const int c = cb * 32 + c4;
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int row = it * 4 + rq, m = m0 + qw * 32 + row;
        const float *t = tp + row * 33 + c4;
        if (m < In && c < Q4)
          __stcg(reinterpret_cast<float4 *>(slot + (size_t)m * Q4 + c), make_float4(t[0], t[1], t[2], t[3]));
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  cluster.sync();   // every CTA's slot written (release / acquire at cluster scope)
  const int r0 = 128 * s / S, rows = 128 * (s + 1) / S - r0;   // this CTA's rows of the tile
  float *Gn = const_cast<float *>(a.G);
  const bool g4 = (Q & 3) == 0 && (reinterpret_cast<uintptr_t>(Gn) & 15) == 0 &&
                  (a.rule == 0 || (reinterpret_cast<uintptr_t>(a.acc) & 15) == 0);
  const int nq4 = Q4 / 4, nvec = rows * nq4;
  constexpr int kUp = 2;   // groups of 4 columns per thread and round: 2 x S slot loads in flight
  for (int e0 = tid; e0 < nvec; e0 += kUp * kFzThreads) {
    float4 gsum[kUp];
    float gold[kUp][4], aold[kUp][4];
#pragma unroll
    for (int u = 0; u < kUp; ++u) {
      const int e = e0 + u * kFzThreads;
      const int rl = r0 + e / nq4, c = (e % nq4) * 4, m = m0 + rl;
      const bool live = e < nvec && m < In;
      float4 v[16];
#pragma unroll
      for (int cc = 0; cc < 16; ++cc)
        v[cc] = (cc < S && live) ? __ldcg(reinterpret_cast<const float4 *>(a.gpart + (size_t)cc * a.pstride +
                                                                           (size_t)m * Q4 + c))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      const size_t gi = (size_t)m * Q + c;
      if (live && g4) {
        const float4 x = __ldcg(reinterpret_cast<const float4 *>(Gn + gi));
        gold[u][0] = x.x; gold[u][1] = x.y; gold[u][2] = x.z; gold[u][3] = x.w;
        if (a.rule != 0) {
          const float4 y = __ldcg(reinterpret_cast<const float4 *>(a.acc + gi));
          aold[u][0] = y.x; aold[u][1] = y.y; aold[u][2] = y.z; aold[u][3] = y.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool ok = live && c + k < Q;
          gold[u][k] = ok ? __ldcg(Gn + gi + k) : 0.f;
          aold[u][k] = (ok && a.rule != 0) ? __ldcg(a.acc + gi + k) : 0.f;
        }
      }
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);   // increasing rank
#pragma unroll
      for (int cc = 0; cc < 16; ++cc)
        if (cc < S) {
          g.x += v[cc].x;
          g.y += v[cc].y;
          g.z += v[cc].z;
          g.w += v[cc].w;
        }
      gsum[u] = g;
    }
#pragma unroll
    for (int u = 0; u < kUp; ++u) {
      const int e = e0 + u * kFzThreads;
      const int rl = r0 + e / nq4, c = (e % nq4) * 4, m = m0 + rl;
      if (e >= nvec || m >= In) continue;
      const float gg[4] = {gsum[u].x, gsum[u].y, gsum[u].z, gsum[u].w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (c + k >= Q) continue;
        const size_t gi = (size_t)m * Q + c + k;
        const float g = gg[k], p = -g;
        float d;
        if (a.rule == 0) {
          d = a.alpha * p;
        } else {
          const float sa = aold[u][k] + p * p;
          a.acc[gi] = sa;
          const float base = a.b + sa;
          d = !(base > 0.f) ? 0.f
                            : ((a.eps == 0.0) ? a.eta / sqrtf(base) : a.eta * powf(base, (float)(-(0.5 + a.eps)))) * p;
        }
        const float nv = gold[u][k] + d;
        if (!isfinite(nv)) latch_status(a.status, kStatusNumeric);
        Gn[gi] = nv;
        if (a.dbg_g) {
          a.dbg_g[gi] = g;
          a.dbg_p[gi] = p;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tb, 512);
}

// ---- host side ----------------------------------------------------------------
// Cluster size for a mode: the largest S <= 16 (and <= the number of sample
// chunks) for which every row tile's cluster is resident at once (the
// occupancy API's count of co-resident clusters of that size), else the S
// with the most CTAs resident.  0: the kernel does not apply (Q > 448: D_g
// needs Q padded to 64 columns of tensor memory beside D_E's 64, and the
// G_n tile Q padded x 128 BF16 values of shared memory beside the Z tile).
int grid_fused_cluster(int In, int Q, int J) {
  if (Q > 448 || Q < 1) return 0;
  const int nch = (J + kFzChunk - 1) / kFzChunk, tiles = (In + 127) / 128;
  int best = 1, best_ctas = 0;
  for (int S = std::min(16, nch); S >= 1; --S) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)S, (unsigned)tiles, 1);
    cfg.blockDim = dim3(kFzThreads, 1, 1);
    cfg.dynamicSmemBytes = grid_fused_smem(Q);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, grid_fused_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n >= tiles) return S;
    if (n * S > best_ctas) {
      best_ctas = n * S;
      best = S;
    }
  }
  return best_ctas > 0 ? best : 0;
}

cudaError_t grid_fused_prepare() {
  cudaError_t e = cudaFuncSetAttribute(grid_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grid_fused_smem(448));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(grid_fused_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t launch_grid_fused(const CUtensorMap &tmZ, const CUtensorMap &tmG, float *gpart, const ProbDesc &D,
                              int n, const long long *col, float w, int S, int rec, cudaStream_t st) {
  const int N = D.N, In = D.I[n], Q = D.R[n] * D.R[(n + 1) % N];
  FusedArgs fa = {};
  fa.tmZ = tmZ;
  fa.tmG = tmG;
  fa.gpart = gpart;
  fa.pstride = (long long)In * ((Q + 3) & ~3);
  fa.G = static_cast<const float *>(D.cores[n]);
  fa.acc = static_cast<float *>(D.acc[n]);
  fa.xmode = static_cast<const __nv_bfloat16 *>(D.xmode[n]);
  fa.ldx = D.ldx[n];
  fa.col = col;
  fa.In = In;
  fa.Q = Q;
  fa.kq = (Q + 63) / 64;
  fa.J = D.J;
  fa.S = S;
  fa.w = w;
  fa.rule = D.rule;
  fa.alpha = (float)D.alpha;
  fa.eta = (float)D.eta;
  fa.b = (float)D.b;
  fa.eps = D.eps;
  fa.dbg_e = rec ? static_cast<float *>(D.dbg_e) : nullptr;
  fa.dbg_g = rec ? static_cast<float *>(D.dbg_g) : nullptr;
  fa.dbg_p = rec ? static_cast<float *>(D.dbg_p) : nullptr;
  fa.status = D.status;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)S, (unsigned)((In + 127) / 128), 1);
  cfg.blockDim = dim3(kFzThreads, 1, 1);
  cfg.dynamicSmemBytes = grid_fused_smem(Q);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grid_fused_kernel, fa);
}

}  // namespace trsgd
