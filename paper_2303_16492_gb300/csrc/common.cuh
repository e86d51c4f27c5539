// Shared device helpers of the TR-BRSGD library (sm_103a).
//
// Philox4x32-10 is written from its published definition (Salmon, Moraes,
// Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).  The
// counter layout of the sampler:
//   word0 = sample j, word1 = (stream << 24) | slot, word2/3 = t low/high,
//   key   = (seed low, seed high);
// a draw is u = (x1 << 32) | x0; a uniform index in [0, m) is
// floor(u * m / 2^64), and a draw from integer weights with inclusive prefix
// sums C (total W) is the smallest i with floor(u * W / 2^64) < C[i].
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>

namespace trsgd {

enum : int { kStreamMode = 0, kStreamF = 1, kStreamH = 2, kStreamOpt = 3 };
enum : int { kMaxOrder = 8 };
enum : int { kStatusOk = 0, kStatusNumeric = 4, kStatusTimeout = 5, kStatusBadIndex = 7 };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

struct Philox4 { uint32_t x0, x1, x2, x3; };

// Ten Philox4x32 rounds with the key bumped by the Weyl constants in between.
__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                         uint32_t c3, uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = mulhi32(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = mulhi32(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

__host__ __device__ __forceinline__ uint64_t draw_u64(uint64_t seed, int64_t t, int stream, int slot,
                                                     uint32_t j) {
  const uint64_t tu = (uint64_t)t;
  const Philox4 o = philox4x32_10(j, ((uint32_t)stream << 24) | (uint32_t)slot, (uint32_t)tu,
                                  (uint32_t)(tu >> 32), (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)o.x1 << 32) | (uint64_t)o.x0;
}

// Mode of iteration t: uniform over {0..N-1} (Algorithm 3).
__host__ __device__ __forceinline__ int draw_mode(uint64_t seed, int64_t t, int N) {
  return (int)mulhi64(draw_u64(seed, t, kStreamMode, 0, 0u), (uint64_t)N);
}

// Smallest i in [0, n) with target < cdf[i]; cdf is nondecreasing, cdf[n-1] > target.
__device__ __forceinline__ int cdf_search(const unsigned long long *__restrict__ cdf, int n,
                                          uint64_t target) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((uint64_t)__ldcg(cdf + mid) > target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// ---- typed loads / stores (cores are read through L2 only: they are
// rewritten by other CTAs of the cluster between steps) --------------------
template <typename T> __device__ __forceinline__ T ld_l2(const T *p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T to_compute(T v) { return v; }
__device__ __forceinline__ float to_compute(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> struct CoreOf { using type = T; };

// ---- shared-memory address helpers ---------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's generic-proxy writes to global memory before later
// async-proxy (bulk copy) reads of the same bytes, by any thread that
// synchronises with it afterwards.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait on an mbarrier phase: returns false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t addr = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared (TMA engine), completion on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Per-thread asynchronous 16-byte copy global -> shared (L2 only: the source
// may have been rewritten by another CTA of the cluster since the last step).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in TMEM) ----------
// Shared-memory matrix descriptor, no swizzle: start address, leading-byte
// offset (LBO) and stride-byte offset (SBO) in 16-byte units, descriptor
// version 1 in bits 46-47.  Operands are tiled in core matrices of 8 rows x
// 16 bytes (128 contiguous bytes).  K-major operand: LBO = stride between
// core matrices adjacent along K, SBO = stride along M/N.  MN-major operand:
// LBO = stride along K, SBO = stride along M/N.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with BF16 A/B and FP32 accumulation.
__host__ __device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A * B^T, M = 128, N from the instruction descriptor, K = 16.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
               "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc)
               : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 8 consecutive 32-bit TMEM columns of this thread's lane (warp w reads lanes
// 32*(w%4) .. 32*(w%4)+31).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit TMEM columns of this thread's lane, one wait.
// Pointer p into this CTA's dynamic shared memory, re-derived from an extern
// __shared__ symbol plus an offset so that loads and stores through it in a
// non-inlined function use the shared-memory instructions: a pointer
// parameter alone is generic, and generic accesses take the longer L1TEX path.
// p must point into dynamic shared memory.
extern __shared__ __align__(16) unsigned char trsgd_dyn_smem[];
template <typename P>
__device__ __forceinline__ P *smem_ptr(P *p) {
  const uint32_t off = (uint32_t)(__cvta_generic_to_shared((const void *)p) - __cvta_generic_to_shared(trsgd_dyn_smem));
  return reinterpret_cast<P *>(trsgd_dyn_smem + off);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (r, k) in a no-swizzle K-major tile whose rows hold
// kc core matrices (kc = K / 8 for 16-bit elements).
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kc) {
  return (uint32_t)(((r >> 3) * kc + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void latch_status(int *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Index checks of the debug build (-DTRSGD_DEBUG): an index outside
// [0, bound) latches TRSGD_EBADINDEX and is replaced by 0, so that nothing is
// read outside its buffer; the product build compiles the checks out.
#ifdef TRSGD_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
template <typename I>
__device__ __forceinline__ I debug_checked(I i, long long bound, int *status) {
  if (kDebugChecks && (i < 0 || (long long)i >= bound)) {
    latch_status(status, kStatusBadIndex);
    return I(0);
  }
  return i;
}

}  // namespace trsgd
