// Scaled variant on the whole-GPU path (Sec. 3.3): the damped preconditioner
// h = Z_H^T D_H Z_H / (|H| J_n) + eta^t I for R_n R_{n+1} up to 512, its
// factorisation and the direction p = -g h^{-1} (Eq. scaledsg_direction),
// followed by the step rule and the update of G_n.
//
// The Gram matrix itself is a tcgen05 GEMM of the grid path (three BF16 pieces
// of Z, FP32 partial sums over slices of the samples); everything after it is
// double-float arithmetic (df64.cuh, about 44-48 significant bits on the FP32
// pipes, where native FP64 runs ~60x slower on this GPU):
//
//   grid_gram_factor_kernel   one cluster of 16 CTAs.  The fixed-order sum of
//       the partial Grams, scaled by 1/|H|, plus the damping, is cut into
//       32 x 32 blocks (the last block row padded with the identity), spread
//       over the CTAs' shared memory in column-major block order, and
//       factored h = L L^T by right-looking block elimination: per block
//       column k (1) the owner of the diagonal block eliminates it (LDL^T
//       with the row operations also applied to an identity, giving
//       L_kk^{-1} = D^{-1/2} U^{-1}); (2) every CTA holding a block of the
//       panel forms L_ik = A_ik L_kk^{-T}; (3) every trailing block takes
//       A_ij -= L_ik L_jk^T with the panel blocks copied in from their
//       owners through distributed shared memory.  A non-positive or
//       non-finite pivot restarts the whole factorisation with the damping
//       grown by 1e-12 tr(h)/Q * 10^m, m = 0..6 (then TRSGD_ENUMERIC).
//       Output: every block of L below the diagonal and the inverted
//       diagonal blocks, each stored as-is and transposed.
//   grid_scaled_apply_kernel  two warps per row of g (halves of the terms;
//       the rows spread over every SM, at most 8 per CTA), the blocks of L
//       streamed through a ring of shared-memory stages by bulk copies that
//       one producer warp issues: the fixed-order sum of the partial
//       gradients, then u L^T = -g
//       by blocked forward substitution and p L = u by blocked backward
//       substitution, each 32 x 32 diagonal step a product with the inverted
//       block; then fixed alpha or AdaGrad and the update, exactly as the
//       plain update kernel does with p = -g.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "nvtx.h"

namespace cg = cooperative_groups;

namespace trsgd {

namespace {

constexpr int kGfB = 32;                                   // block size
constexpr int kGfC = 16;                                   // CTAs of the cluster
constexpr int kGfT = 512;                                  // threads per CTA
constexpr int kGfMaxNb = kGridScaledMaxQ / kGfB;           // 16 block rows
constexpr int kGfSlots = (kGfMaxNb * (kGfMaxNb + 1) / 2 + kGfC - 1) / kGfC;   // blocks per CTA
constexpr int kGfPitchT = 33;                              // transposed staging pitch (conflict-free)
constexpr int kGfPlaneT = kGfB * kGfPitchT;                // floats per transposed plane
// output block: [orientation: X, X^T][hi, lo][32 rows][kLp], rows padded to
// kLp floats so that a lane reads four consecutive entries of its row as one
// 16-byte load without bank conflicts (8 lanes of a quarter warp: banks 4 c)
constexpr int kLp = 36;
constexpr int kLpl = kGfB * kLp;                           // floats per plane
constexpr int kBlkF = 4 * kLpl;                            // floats per output block

// shared memory of the factor kernel (floats): local blocks (hi plane, lo
// plane), the transposed panel staging, the row-major L_kk^{-1} / U^{-1}
// buffer, and its transposed copy
constexpr size_t kGfSlotF = 2 * kGfB * kGfB;
constexpr size_t kGfSmemFloats = kGfSlots * kGfSlotF + kGfMaxNb * 2 * kGfPlaneT + kGfSlotF + 2 * kGfPlaneT;

__device__ __forceinline__ df64 lds(const float *b, int e) { return df64{b[e], b[e + kGfB * kGfB]}; }
__device__ __forceinline__ void sts(float *b, int e, df64 v) {
  b[e] = v.hi;
  b[e + kGfB * kGfB] = v.lo;
}
__device__ __forceinline__ df64 ldt(const float *b, int e) { return df64{b[e], b[e + kGfPlaneT]}; }
__device__ __forceinline__ void stt(float *b, int e, df64 v) {
  b[e] = v.hi;
  b[e + kGfPlaneT] = v.lo;
}

// column-major packed position of block (i, j), i >= j, of an nb x nb block triangle
__device__ __forceinline__ int blk_cm(int i, int j, int nb) { return j * nb - j * (j - 1) / 2 + (i - j); }
// row-major packed position (output layout)
__host__ __device__ __forceinline__ int blk_rm(int i, int j) { return i * (i + 1) / 2 + j; }

}  // namespace

struct GramFactorArgs {
  const float *hpart;     // [splits][Q][Q] partial Grams (FP32, row-major)
  long long pstride;      // elements between consecutive partials
  int splits, Q, nb;
  double scale;           // 1 / |H|
  double damping;         // eta^t
  float *Lout;            // [nb (nb + 1) / 2][kBlkF] blocks of the factor (row-major packed)
  double *dbg_h;          // [Q][Q] the damped h actually factored (FP64), or null
  int *ok;                // 1: factored; 0: every rung of the ladder failed
  int *status;
};

// s + lo -= (ah + al)(bh + bl), the sum kept unnormalised: the leading
// product is split exactly (Dekker's two-product through an FMA) and
// subtracted from s exactly (Knuth's two-sum); the two-sum's error, the
// product's error and the two cross terms are summed in float and added to
// lo.  11 float operations, one of them on each accumulator's dependency
// chain; the pair is renormalised once, after the last term.
__device__ __forceinline__ void dacc_fnms(float ah, float al, float bh, float bl, float &s, float &lo) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  const float t = s - p;
  const float bb = t - s;
  const float err = (s - (t - bb)) + (-p - bb);
  lo += fmaf(-al, bh, fmaf(-ah, bl, err - e));
  s = t;
}

// the four accumulators of dacc_fnms renormalised and added in a fixed order
__device__ __forceinline__ df64 dacc_total(const float (&s)[4], const float (&lo)[4]) {
  df64 r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = df_two_sum(s[k], lo[k]);
  return df_add(df_add(r[0], r[1]), df_add(r[2], r[3]));
}

// ready flags of the factor's blocks, read and written at cluster scope
__device__ __forceinline__ int gf_ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void gf_st_release(int *p, int v) {
  asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
constexpr long long kGfSpin = 1LL << 22;   // polls of a ready flag before a wait gives up
// outcome of a wait or of an attempt, shared by the CTA's threads
enum : int { kGfOk = 0, kGfAbandoned = 1, kGfTimedOut = 2 };

__global__ void __launch_bounds__(kGfT, 1) grid_gram_factor_kernel(const __grid_constant__ GramFactorArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cta = (int)cluster.block_rank();
  extern __shared__ __align__(16) float gfs[];
  float *slots = gfs;                                     // [kGfSlots][2][32 * 32]
  float *panelT = slots + kGfSlots * kGfSlotF;            // [kGfMaxNb][2][32 * 33], block (i, k) transposed
  float *W = panelT + (size_t)kGfMaxNb * 2 * kGfPlaneT;   // [2][32 * 32] U^{-1} of the diagonal elimination
  float *linvT = W + kGfSlotF;                            // [2][32 * 33] L_kk^{-1} transposed
  __shared__ int blk_i[kGfSlots], blk_j[kGfSlots], nslots_s;
  __shared__ unsigned char own_tab[kGfMaxNb * (kGfMaxNb + 1) / 2], slot_tab[kGfMaxNb * (kGfMaxNb + 1) / 2];
  __shared__ int ready[kGfSlots];   // epoch in which the slot's block became final (L_ik, or L_kk^{-1})
  __shared__ int fail_flag;         // 4 epoch + outcome of an attempt this CTA abandoned
  __shared__ int wait_s;            // outcome of the last wait, for every thread of the CTA
  __shared__ double diag_s[kGridScaledMaxQ];
  const int tid = threadIdx.x, cc = tid & 31, r0 = tid >> 5;
  const int nb = a.nb, Q = a.Q;
  // Block ownership, the same table in every CTA: column-major order dealt
  // round robin over the CTAs, so that the blocks of one column (the panel
  // of a step) are formed by different CTAs in parallel.
  if (tid == 0) {
    for (int idx = 0; idx < nb * (nb + 1) / 2; ++idx) {
      own_tab[idx] = (unsigned char)(idx % kGfC);
      slot_tab[idx] = (unsigned char)(idx / kGfC);
    }
    int n = 0;
    for (int j = 0; j < nb; ++j)
      for (int i = j; i < nb; ++i) {
        const int idx = blk_cm(i, j, nb);
        if (own_tab[idx] != cta) continue;
        const int sl = slot_tab[idx];
        blk_i[sl] = i;
        blk_j[sl] = j;
        ready[sl] = 0;
        ++n;
      }
    nslots_s = n;
    fail_flag = 0;
  }
  __syncthreads();
  const int nslots = nslots_s;
  const df64 scale = df_from_double(a.scale);
  auto owner = [&](int i, int j) { return (int)own_tab[blk_cm(i, j, nb)]; };
  auto slot_of = [&](int i, int j) { return (int)slot_tab[blk_cm(i, j, nb)]; };

  // h(ga, gb) as double-float: the partials summed in increasing order
  auto gram_entry = [&](int ga, int gb) {
    df64 v = df64{0.f, 0.f};
    for (int z = 0; z < a.splits; ++z) v = df_add(v, df64{__ldcg(a.hpart + z * a.pstride + (long long)ga * Q + gb), 0.f});
    return df_mul(v, scale);
  };
  auto publish = [&](int slot, int epoch) {   // after every thread's writes to the block
    __syncthreads();
    if (tid == 0) gf_st_release(&ready[slot], epoch);
  };
  // thread 0 waits until the blocks (i, k), i in `rows`, are final in this
  // epoch, or until the owner of one of them abandoned the attempt; every
  // thread returns the outcome
  auto wait_rows = [&](int k, unsigned rows, int epoch) -> int {
    if (tid == 0) {
      int res = kGfOk;
      for (int i = k; i < nb && res == kGfOk; ++i) {
        if (!((rows >> i) & 1u)) continue;
        const int o = owner(i, k);
        const int *rf = cluster.map_shared_rank(&ready[slot_of(i, k)], o);
        const int *ff = cluster.map_shared_rank(&fail_flag, o);
        res = kGfTimedOut;
        for (long long it = 0; it < kGfSpin; ++it) {
          if (gf_ld_acquire(rf) == epoch) {
            res = kGfOk;
            break;
          }
          if ((gf_ld_acquire(ff) >> 2) == epoch) {
            res = kGfAbandoned;
            break;
          }
        }
      }
      wait_s = res;
    }
    __syncthreads();
    const int res = wait_s;
    __syncthreads();
    return res;
  };
  // the panel blocks (i, k), i in `rows`, into panelT[i] (transposed) from
  // their owners' shared memory
  auto fetch = [&](int k, unsigned rows, int epoch) -> int {
    if (!rows) return kGfOk;
    const int res = wait_rows(k, rows, epoch);
    if (res != kGfOk) return res;
    for (int i = k + 1; i < nb; ++i) {
      if (!((rows >> i) & 1u)) continue;
      const float *src = cluster.map_shared_rank(slots + slot_of(i, k) * kGfSlotF, owner(i, k));
      float *dst = panelT + (size_t)i * 2 * kGfPlaneT;
      for (int e = tid; e < kGfB * kGfB; e += kGfT) stt(dst, (e & 31) * kGfPitchT + (e >> 5), lds(src, e));
    }
    __syncthreads();
    return kGfOk;
  };
  // diagonal block (k, k), held here: LDL^T with the row operations applied
  // to an identity, then L_kk^{-1} = D^{-1/2} U^{-1} into the block's slot
  // (and the output); false on a non-positive or non-finite pivot
  auto diag = [&](int k) -> bool {
    float *A = slots + slot_of(k, k) * kGfSlotF;
    for (int e = tid; e < kGfB * kGfB; e += kGfT) sts(W, e, df64{(e >> 5) == (e & 31) ? 1.f : 0.f, 0.f});
    __syncthreads();
    for (int j = 0; j < kGfB; ++j) {
      const df64 d = lds(A, j * kGfB + j);
      if (!(d.hi > 0.f) || !isfinite(d.hi)) return false;   // the same value in every thread
      const df64 invd = df_rcp(d);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + 16 * h;
        if (r > j) {   // the same in the whole warp
          // columns right of the pivot in A, the others in W: one select, no divergence
          float *B = cc > j ? A : W;
          const df64 l = df_mul(lds(A, r * kGfB + j), invd);
          sts(B, r * kGfB + cc, df_fnms_fast(l, lds(B, j * kGfB + cc), lds(B, r * kGfB + cc)));
        }
      }
      __syncthreads();
    }
    df64 v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + 16 * h;
      const df64 qr = df_rcp(df_sqrt(lds(A, r * kGfB + r)));
      v[h] = cc <= r ? df_mul(lds(W, r * kGfB + cc), qr) : df64{0.f, 0.f};
    }
    __syncthreads();   // every thread has read the pivots
#pragma unroll
    for (int h = 0; h < 2; ++h) sts(A, (r0 + 16 * h) * kGfB + cc, v[h]);
    return true;
  };
  // a final block (slot s, position (i, j)) into the output, in both
  // orientations; after its ready flag, off the critical path
  auto write_out = [&](int s, int i, int j) {
    const float *A = slots + s * kGfSlotF;
    float *o = a.Lout + (size_t)blk_rm(i, j) * kBlkF;
    for (int e = tid; e < kGfB * kGfB; e += kGfT) {
      const int r = e >> 5, c = e & 31;
      const df64 v = lds(A, e);
      o[r * kLp + c] = v.hi;
      o[kLpl + r * kLp + c] = v.lo;
    }
    for (int e = tid; e < kGfB * kGfB; e += kGfT) {   // consecutive threads: consecutive entries of a transposed row
      const int c = e >> 5, r = e & 31;
      const df64 v = lds(A, r * kGfB + c);
      o[2 * kLpl + c * kLp + r] = v.hi;
      o[3 * kLpl + c * kLp + r] = v.lo;
    }
  };
  // L_kk^{-1} (final in its owner) into linvT, transposed
  auto stage_linv = [&](int k) {
    const float *Lk = cluster.map_shared_rank(slots + slot_of(k, k) * kGfSlotF, owner(k, k));
    for (int e = tid; e < kGfB * kGfB; e += kGfT) stt(linvT, (e & 31) * kGfPitchT + (e >> 5), lds(Lk, e));
    __syncthreads();
  };
  // panel block in slot s, (i, k): L_ik = A_ik L_kk^{-T} (linvT staged), then
  // its ready flag and its output
  auto panel_block = [&](int s, int k, int epoch) {
    float *A = slots + s * kGfSlotF;
    df64 out[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + 16 * h;
      // four unnormalised partial sums (t mod 4); L_kk^{-1} holds exact zeros
      // above its diagonal, so the terms t > cc add nothing
      float sa[4] = {0.f, 0.f, 0.f, 0.f}, la[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
      for (int t = 0; t < kGfB; ++t) {
        const df64 x = lds(A, r * kGfB + t), y = ldt(linvT, t * kGfPitchT + cc);
        dacc_fnms(-x.hi, -x.lo, y.hi, y.lo, sa[t & 3], la[t & 3]);
      }
      out[h] = dacc_total(sa, la);
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) sts(A, (r0 + 16 * h) * kGfB + cc, out[h]);
    publish(s, epoch);
    write_out(s, blk_i[s], k);
  };
  // the panel blocks (i, k), i > k, held here and not in `done` (a slot
  // mask), once L_kk^{-1} is final (`staged`: already in linvT)
  auto panel_col = [&](int k, int epoch, unsigned done, bool staged) -> int {
    bool have = false;
    for (int s = 0; s < nslots; ++s) have |= (blk_j[s] == k && blk_i[s] > k && !((done >> s) & 1u));
    if (!have) return kGfOk;
    if (!staged) {
      const int res = wait_rows(k, 1u << k, epoch);
      if (res != kGfOk) return res;
      stage_linv(k);
    }
    for (int s = 0; s < nslots; ++s)
      if (blk_j[s] == k && blk_i[s] > k && !((done >> s) & 1u)) panel_block(s, k, epoch);
    return kGfOk;
  };
  // trailing update A_ij -= L_ik L_jk^T of the block in slot s (panels staged)
  auto trail = [&](int s) {
    float *A = slots + s * kGfSlotF;
    const float *Pi = panelT + (size_t)blk_i[s] * 2 * kGfPlaneT;
    const float *Pj = panelT + (size_t)blk_j[s] * 2 * kGfPlaneT;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + 16 * h;
      const df64 a0 = lds(A, r * kGfB + cc);
      float sa[4] = {a0.hi, 0.f, 0.f, 0.f}, la[4] = {a0.lo, 0.f, 0.f, 0.f};
#pragma unroll 8
      for (int t = 0; t < kGfB; ++t) {
        const df64 x = ldt(Pi, t * kGfPitchT + r), y = ldt(Pj, t * kGfPitchT + cc);
        dacc_fnms(x.hi, x.lo, y.hi, y.lo, sa[t & 3], la[t & 3]);
      }
      sts(A, r * kGfB + cc, dacc_total(sa, la));
    }
  };

  bool ok = false, timed_out = false;
  double extra = 0.0, tr = -1.0;
  for (int m = -1; m < 7 && !ok && !timed_out; ++m) {
    const int epoch = m + 2;
    if (m >= 0) {
      if (tr < 0.0) {   // trace of the undamped h, same fixed order in every CTA
        for (int q = tid; q < Q; q += kGfT) diag_s[q] = df_to_double(gram_entry(q, q));
        __syncthreads();
        if (tid == 0) {
          double sum = 0.0;
          for (int q = 0; q < Q; ++q) sum += diag_s[q];
          diag_s[0] = sum;
        }
        __syncthreads();
        tr = diag_s[0];
        __syncthreads();
      }
      extra = 1e-12 * tr / Q * pow(10.0, (double)m);
    }
    const df64 damp = df_from_double(a.damping + extra);
    // load: this CTA's blocks of the damped h (identity on the padding)
    for (int s = 0; s < nslots; ++s) {
      float *A = slots + s * kGfSlotF;
      // the two entries of this thread: every partial loaded before the sums
      float part[2][16];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = tid + h * kGfT;
        const int ga = blk_i[s] * kGfB + (e >> 5), gb = blk_j[s] * kGfB + (e & 31);
#pragma unroll
        for (int z = 0; z < 16; ++z)
          part[h][z] = (z < a.splits && ga < Q && gb < Q) ? __ldcg(a.hpart + z * a.pstride + (long long)ga * Q + gb) : 0.f;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = tid + h * kGfT;
        const int ga = blk_i[s] * kGfB + (e >> 5), gb = blk_j[s] * kGfB + (e & 31);
        df64 v;
        if (ga < Q && gb < Q) {
          v = df64{0.f, 0.f};
#pragma unroll
          for (int z = 0; z < 16; ++z)
            if (z < a.splits) v = df_add(v, df64{part[h][z], 0.f});
          for (int z = 16; z < a.splits; ++z)
            v = df_add(v, df64{__ldcg(a.hpart + z * a.pstride + (long long)ga * Q + gb), 0.f});
          v = df_mul(v, scale);
          if (ga == gb) v = df_add(v, damp);
        } else {
          v = df64{ga == gb ? 1.f : 0.f, 0.f};
        }
        sts(A, e, v);
      }
    }
    __syncthreads();
    cluster.sync();   // every block loaded; the previous attempt's remote reads are over
    // Right-looking block elimination with look-ahead: in step k a CTA first
    // updates its blocks of column k + 1, so that the diagonal block k + 1 is
    // factored and the panel of column k + 1 formed while the rest of the
    // trailing update of step k is still running elsewhere; the blocks a
    // step needs are waited for through their owners' ready flags.
    int res = kGfOk;
    if (owner(0, 0) == cta) {
      if (diag(0)) publish(slot_of(0, 0), epoch);
      else res = kGfAbandoned;
    }
    if (res == kGfOk) res = panel_col(0, epoch, 0u, false);
    if (res == kGfOk && owner(0, 0) == cta) write_out(slot_of(0, 0), 0, 0);
    for (int k = 0; k + 1 < nb && res == kGfOk; ++k) {
      const int kd = k + 1;
      unsigned fetched = 0u, trailed = 0u, paneled = 0u;   // rows of column k; slots done in this step
      bool staged = false;                                 // L_{kd kd}^{-1} in linvT
      if (owner(kd, kd) == cta) {
        // the critical chain first: the diagonal block of column kd, factored
        // as soon as it is updated, then the block below it (held here too)
        const int sd = slot_of(kd, kd);
        if ((res = fetch(k, 1u << kd, epoch)) != kGfOk) break;
        fetched |= 1u << kd;
        trail(sd);
        trailed |= 1u << sd;
        __syncthreads();
        if (!diag(kd)) {
          res = kGfAbandoned;
          break;
        }
        publish(sd, epoch);
        if (kd + 1 < nb && owner(kd + 1, kd) == cta) {
          const int sb = slot_of(kd + 1, kd);
          if ((res = fetch(k, 1u << (kd + 1), epoch)) != kGfOk) break;
          fetched |= 1u << (kd + 1);
          trail(sb);
          trailed |= 1u << sb;
          __syncthreads();
          stage_linv(kd);
          staged = true;
          panel_block(sb, kd, epoch);
          paneled |= 1u << sb;
        }
      }
      unsigned need1 = 0u, need2 = 0u;   // rows of column k the rest of the update reads
      for (int s = 0; s < nslots; ++s) {
        if ((trailed >> s) & 1u) continue;
        if (blk_j[s] == kd) need1 |= (1u << blk_i[s]) | (1u << kd);
        else if (blk_j[s] > kd) need2 |= (1u << blk_i[s]) | (1u << blk_j[s]);
      }
      need1 &= ~fetched;
      if ((res = fetch(k, need1, epoch)) != kGfOk) break;
      fetched |= need1;
      for (int s = 0; s < nslots; ++s)
        if (blk_j[s] == kd && !((trailed >> s) & 1u)) trail(s);
      __syncthreads();
      if ((res = panel_col(kd, epoch, paneled, staged)) != kGfOk) break;
      if (owner(kd, kd) == cta) write_out(slot_of(kd, kd), kd, kd);
      need2 &= ~fetched;
      if ((res = fetch(k, need2, epoch)) != kGfOk) break;
      for (int s = 0; s < nslots; ++s)
        if (blk_j[s] > kd) trail(s);
      __syncthreads();   // panelT is rewritten by the next step's fetch
    }
    if (res != kGfOk && tid == 0) gf_st_release(&fail_flag, 4 * epoch + res);
    cluster.sync();   // the attempt is over in every CTA
    bool any = false;
    for (int c = 0; c < kGfC; ++c) {
      const int f = *cluster.map_shared_rank(&fail_flag, c);
      if ((f >> 2) == epoch) {
        any = true;
        timed_out |= (f & 3) == kGfTimedOut;
      }
    }
    ok = !any;
    cluster.sync();   // every CTA has read the flags before the next attempt can set them
  }
  if (cta == 0 && tid == 0) {
    *a.ok = ok ? 1 : 0;
    if (!ok) latch_status(a.status, timed_out ? kStatusTimeout : kStatusNumeric);
  }
  if (ok && a.dbg_h) {   // the damped h that was factored, for the record
    const double dtot = a.damping + extra;
    for (long long e = (long long)cta * kGfT + tid; e < (long long)Q * Q; e += (long long)kGfC * kGfT) {
      const int ga = (int)(e / Q), gb = (int)(e % Q);
      a.dbg_h[e] = df_to_double(gram_entry(ga, gb)) + (ga == gb ? dtot : 0.0);
    }
  }
}

// ---- direction, step rule and update ---------------------------------------
struct ScaledApplyArgs {
  const float *gpart;     // [splits][In][Q] partial gradients
  long long cstride;
  int splits, In, Q, nb;
  int rows;               // rows of g per CTA (one consumer warp each)
  const float *Lblk;      // blocks written by grid_gram_factor_kernel
  const int *ok;
  int rule;
  float alpha, eta, b;
  double eps;
  float *G, *acc;
  float *dbg_g, *dbg_p;
  int *status;
};

constexpr int kApMaxRows = 8;                  // rows of g per CTA at most (two consumer warps each)
constexpr int kApDepth = 8;                    // staged blocks in flight
constexpr int kApStage = 2 * kLpl;             // floats per stage: one orientation, hi and lo planes
constexpr long long kApWait = 1LL << 24;

__device__ __forceinline__ void ap_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Four accumulators (one per t mod 4) of a 32-term row product, renormalised
// and added in a fixed order.
struct DAcc4 {
  float s[4], lo[4];
  __device__ __forceinline__ void reset(df64 first) {
    s[0] = first.hi;
    lo[0] = first.lo;
    s[1] = s[2] = s[3] = lo[1] = lo[2] = lo[3] = 0.f;
  }
  // this lane's row of a staged plane pair (X[c][t]: hi at xh, lo at xl)
  // against the vector v[0..31]; sign -1: subtract, +1: add
  template <int SIGN>
  __device__ __forceinline__ void row(const float *xh, const float *xl, const df64 *v) {
    const float4 *h4 = reinterpret_cast<const float4 *>(xh);
    const float4 *l4 = reinterpret_cast<const float4 *>(xl);
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
#pragma unroll
    for (int t4 = 0; t4 < kGfB / 4; ++t4) {
      const float4 h = h4[t4], l = l4[t4], u01 = v4[2 * t4], u23 = v4[2 * t4 + 1];
      const float sg = SIGN < 0 ? 1.f : -1.f;
      dacc_fnms(sg * h.x, sg * l.x, u01.x, u01.y, s[0], lo[0]);
      dacc_fnms(sg * h.y, sg * l.y, u01.z, u01.w, s[1], lo[1]);
      dacc_fnms(sg * h.z, sg * l.z, u23.x, u23.y, s[2], lo[2]);
      dacc_fnms(sg * h.w, sg * l.w, u23.z, u23.w, s[3], lo[3]);
    }
  }
  // the same for the terms t of one half, [16 half, 16 half + 16)
  template <int SIGN>
  __device__ __forceinline__ void half_row(const float *xh, const float *xl, const df64 *v, int half) {
    const float4 *h4 = reinterpret_cast<const float4 *>(xh) + 4 * half;
    const float4 *l4 = reinterpret_cast<const float4 *>(xl) + 4 * half;
    const float4 *v4 = reinterpret_cast<const float4 *>(v) + 8 * half;
#pragma unroll
    for (int t4 = 0; t4 < kGfB / 8; ++t4) {
      const float4 h = h4[t4], l = l4[t4], u01 = v4[2 * t4], u23 = v4[2 * t4 + 1];
      const float sg = SIGN < 0 ? 1.f : -1.f;
      dacc_fnms(sg * h.x, sg * l.x, u01.x, u01.y, s[0], lo[0]);
      dacc_fnms(sg * h.y, sg * l.y, u01.z, u01.w, s[1], lo[1]);
      dacc_fnms(sg * h.z, sg * l.z, u23.x, u23.y, s[2], lo[2]);
      dacc_fnms(sg * h.w, sg * l.w, u23.z, u23.w, s[3], lo[3]);
    }
  }
  __device__ __forceinline__ df64 total() const { return dacc_total(s, lo); }
};

// Two warps per row of g (each takes half of the 32 terms of every block
// product; the halves meet in shared memory at the end of each block row),
// rows() rows per CTA, plus one producer warp whose lane 0 streams the blocks
// of L through a ring of kApDepth shared stages by bulk copies (TMA engine),
// each completing on its stage's "full" mbarrier; a consumer warp that is
// done with a stage arrives on its "empty" mbarrier, which the producer waits
// on before refilling it.  The sequence of stages: forward (block row b:
// (b, m), m < b, then the inverted diagonal block), as stored; backward
// (block column b = nb-1 .. 0: (m, b), m > b, then the inverted diagonal
// block), transposed.  Every wait is bounded: a timeout latches
// TRSGD_ETIMEOUT and the stage is waited for once more, so that no copy is
// left in flight when the CTA exits.
__global__ void __launch_bounds__(32 * (2 * kApMaxRows + 1), 1) grid_scaled_apply_kernel(const __grid_constant__ ScaledApplyArgs a) {
  if (!*a.ok) return;   // no factor: the status is latched, G_n stays as it is
  extern __shared__ __align__(128) float aps[];
  __shared__ __align__(8) uint64_t full[kApDepth], empty[kApDepth];
  const int RW = a.rows, nb = a.nb, Q = a.Q, Qp = nb * kGfB;
  float *ring = aps;
  df64 *vecb = reinterpret_cast<df64 *>(aps + kApDepth * kApStage);
  df64 *cmbb = vecb + (size_t)RW * Qp;   // [RW][32]: the second half's partial sums
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nfw = nb * (nb + 1) / 2, S = 2 * nfw;
  if (tid == 0) {
    for (int k = 0; k < kApDepth; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], (uint32_t)(2 * RW));
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == 2 * RW) {   // producer
    if (lane == 0) {
      int b = 0, m = 0;   // block of stage s: forward row b, column m (m == b: diagonal)
      for (int s = 0; s < S; ++s) {
        const int slot = s % kApDepth;
        if (s >= kApDepth && !mbar_wait_bounded(&empty[slot], (uint32_t)((s / kApDepth - 1) & 1), kApWait))
          latch_status(a.status, kStatusTimeout);
        int bi, bj, tr;
        if (s < nfw) {
          bi = b;
          bj = m;
          tr = 0;
          if (++m > b) {
            ++b;
            m = 0;
          }
          if (s + 1 == nfw) {   // first backward stage: column nb-1, its diagonal block
            b = nb - 1;
            m = nb - 1;
          }
        } else {
          bi = m;
          bj = b;
          tr = 1;
          if (--m < b) {   // after the diagonal block of column b: column b-1 from row nb-1
            --b;
            m = nb - 1;
          }
        }
        mbar_arrive_expect_tx(&full[slot], (uint32_t)(kApStage * sizeof(float)));
        tma_load_1d(ring + (size_t)slot * kApStage, a.Lblk + (size_t)blk_rm(bi, bj) * kBlkF + tr * kApStage,
                    (uint32_t)(kApStage * sizeof(float)), &full[slot]);
      }
    }
    return;
  }
  const int pr = warp >> 1, half = warp & 1;   // row of the CTA, half of the terms
  df64 *v = vecb + (size_t)pr * Qp;
  df64 *cmb = cmbb + (size_t)pr * kGfB;
  const int row = blockIdx.x * RW + pr;
  const bool live = row < a.In;
  // the two warps of a row meet at a named barrier of their own (id 1 + pr)
  auto pair_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + pr) : "memory"); };
  // -g of this row (the plain update's fixed-order sum of the partials)
  for (int q = lane + 32 * half; q < Qp; q += 64) {
    float g = 0.f;
    if (live && q < Q)
      for (int z = 0; z < a.splits; ++z) g += __ldcg(a.gpart + z * a.cstride + (long long)row * Q + q);
    v[q] = df64{-g, 0.f};
    if (live && q < Q && a.dbg_g) a.dbg_g[(long long)row * Q + q] = g;
  }
  pair_sync();
  int s = 0;
  auto acquire = [&]() -> const float * {
    const int slot = s % kApDepth;
    const uint32_t par = (uint32_t)((s / kApDepth) & 1);
    if (!mbar_wait_bounded(&full[slot], par, kApWait)) {
      latch_status(a.status, kStatusTimeout);
      mbar_wait_bounded(&full[slot], par, kApWait);
    }
    return ring + (size_t)slot * kApStage + lane * kLp;   // this lane's row of the hi plane
  };
  auto release = [&]() {
    __syncwarp();
    if (lane == 0) ap_arrive(&empty[s % kApDepth]);
    ++s;
  };
  // the row's two halves of an entry summed into v[i] (the first half's warp
  // adds the second's, read after the pair barrier), visible to both after
  // the second barrier
  auto combine_into = [&](int i, df64 part) {
    if (half) cmb[lane] = part;
    pair_sync();
    if (!half) v[i] = df_add(part, cmb[lane]);
    pair_sync();
  };
  DAcc4 acc;
  // forward: u L^T = -g; block row b: r = -g_b - sum_{m<b} C_bm u_m, u_b = L_bb^{-1} r
  for (int b = 0; b < nb; ++b) {
    acc.reset(half == 0 ? v[b * kGfB + lane] : df64{0.f, 0.f});
    for (int m = 0; m < b; ++m) {
      const float *X = acquire();
      acc.half_row<-1>(X, X + kLpl, v + m * kGfB, half);
      release();
    }
    combine_into(b * kGfB + lane, acc.total());
    const float *X = acquire();
    acc.reset(df64{0.f, 0.f});
    acc.half_row<1>(X, X + kLpl, v + b * kGfB, half);   // the inverse is lower triangular: zeros above the diagonal
    const df64 u = acc.total();
    release();
    combine_into(b * kGfB + lane, u);
  }
  // backward: p L = u; block column b: s = u_b - sum_{m>b} C_mb^T p_m, p_b = L_bb^{-T} s
  for (int b = nb - 1; b >= 0; --b) {
    acc.reset(half == 0 ? v[b * kGfB + lane] : df64{0.f, 0.f});
    for (int m = nb - 1; m > b; --m) {
      const float *X = acquire();
      acc.half_row<-1>(X, X + kLpl, v + m * kGfB, half);
      release();
    }
    combine_into(b * kGfB + lane, acc.total());
    const float *X = acquire();
    acc.reset(df64{0.f, 0.f});
    acc.half_row<1>(X, X + kLpl, v + b * kGfB, half);
    const df64 p = acc.total();
    release();
    combine_into(b * kGfB + lane, p);
  }
  if (!live) return;
  // step rule and update (as the plain update kernel, with this p)
  for (int q = lane + 32 * half; q < Q; q += 64) {
    const df64 pd = v[q];
    const float p = pd.hi + pd.lo;
    const long long e = (long long)row * Q + q;
    float d;
    if (a.rule == 0) {
      d = a.alpha * p;
    } else {
      const float sacc = __ldcg(a.acc + e) + p * p;
      a.acc[e] = sacc;
      const float base = a.b + sacc;
      d = !(base > 0.f) ? 0.f
                        : ((a.eps == 0.0) ? a.eta / sqrtf(base) : a.eta * powf(base, (float)(-(0.5 + a.eps)))) * p;
    }
    const float nv = __ldcg(a.G + e) + d;
    if (!isfinite(nv)) latch_status(a.status, kStatusNumeric);
    a.G[e] = nv;
    if (a.dbg_p) a.dbg_p[e] = p;
  }
}

// ---- host side ----------------------------------------------------------------
size_t grid_scaled_factor_floats(int Q) {
  const int nb = (Q + kGfB - 1) / kGfB;
  return (size_t)(nb * (nb + 1) / 2) * kBlkF;
}

cudaError_t grid_scaled_prepare() {
  const int smem = (int)(kGfSmemFloats * sizeof(float));
  cudaError_t e = cudaFuncSetAttribute(grid_gram_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(grid_gram_factor_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(grid_scaled_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kApDepth * kApStage * sizeof(float) +
                                   (size_t)kApMaxRows * (kGridScaledMaxQ + kGfB) * sizeof(df64)));
  return e;
}

cudaError_t launch_grid_factor(const GridScaledArgs &s, cudaStream_t st) {
  const int nb = (s.Q + kGfB - 1) / kGfB;
  if (s.Q < 1 || s.Q > kGridScaledMaxQ) return cudaErrorInvalidValue;
  {
    NvtxRange r("grid_gram_factor_kernel");
    GramFactorArgs fa = {};
    fa.hpart = s.hpart;
    fa.pstride = s.hstride;
    fa.splits = s.hsplits;
    fa.Q = s.Q;
    fa.nb = nb;
    fa.scale = s.hscale;
    fa.damping = s.damping;
    fa.Lout = s.Lfac;
    fa.dbg_h = s.dbg_h;
    fa.ok = s.ok;
    fa.status = s.status;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kGfC, 1, 1);
    cfg.blockDim = dim3(kGfT, 1, 1);
    cfg.dynamicSmemBytes = kGfSmemFloats * sizeof(float);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kGfC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grid_gram_factor_kernel, fa);
  }
}

cudaError_t launch_grid_direction(const GridScaledArgs &s, cudaStream_t st) {
  const int nb = (s.Q + kGfB - 1) / kGfB;
  if (s.Q < 1 || s.Q > kGridScaledMaxQ) return cudaErrorInvalidValue;
  NvtxRange r("grid_scaled_apply_kernel");
  ScaledApplyArgs aa = {};
  aa.gpart = s.gpart;
  aa.cstride = s.gstride;
  aa.splits = s.gsplits;
  aa.In = s.In;
  aa.Q = s.Q;
  aa.nb = nb;
  aa.Lblk = s.Lfac;
  aa.ok = s.ok;
  aa.rule = s.rule;
  aa.alpha = s.alpha;
  aa.eta = s.eta;
  aa.b = s.b;
  aa.eps = s.eps;
  aa.G = s.G;
  aa.acc = s.acc;
  aa.dbg_g = s.dbg_g;
  aa.dbg_p = s.dbg_p;
  aa.status = s.status;
  // rows per CTA: the rows spread over every SM (one CTA each) where they allow
  const int sms = s.sms > 0 ? s.sms : 1;
  aa.rows = std::min(kApMaxRows, std::max(1, (s.In + sms - 1) / sms));
  const size_t smem =
      (size_t)kApDepth * kApStage * sizeof(float) + (size_t)aa.rows * (nb * kGfB + kGfB) * sizeof(df64);
  grid_scaled_apply_kernel<<<(s.In + aa.rows - 1) / aa.rows, 32 * (2 * aa.rows + 1), smem, st>>>(aa);
  return cudaGetLastError();
}

cudaError_t launch_grid_scaled(const GridScaledArgs &s, cudaStream_t st) {
  cudaError_t e = launch_grid_factor(s, st);
  return e == cudaSuccess ? launch_grid_direction(s, st) : e;
}

}  // namespace trsgd
