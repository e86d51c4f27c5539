// Host side of the C-ABI declared in include/trsgd.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "trsgd.h"
#include "common.cuh"
#include "internal.h"
#include "nvtx.h"
#include "tables.cuh"

using namespace trsgd;

namespace {

constexpr int kMaxRank = 16;       // register bound of the slice chain
constexpr int kMaxQPlain = 256;
constexpr int kMaxQScaled = 128;

size_t dtype_size(int d) { return d == TRSGD_DTYPE_F64 ? 8 : d == TRSGD_DTYPE_F32 ? 4 : 2; }
size_t rup(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Buffers {
  std::vector<void *> ptrs;
  ~Buffers() {
    for (void *p : ptrs) cudaFree(p);
  }
  cudaError_t alloc(void **out, size_t bytes) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    ptrs.push_back(p);
    *out = p;
    return cudaSuccess;
  }
};

trsgd_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TRSGD_OK;
  if (e == cudaErrorMemoryAllocation) return TRSGD_ENOMEM;
  return TRSGD_ECUDA;
}

}  // namespace

struct trsgd_handle {
  int nprob = 0;
  std::vector<trsgd_config> cfg;
  cudaStream_t stream = nullptr;
  int core_dtype = 1, xc_dtype = 1, rmax = 4;
  int fp32_pieces = 1;   // FP32 contractions on the tensor cores as three BF16 pieces when they fit
  std::vector<ProbDesc> hdesc;
  ProbDesc *ddesc = nullptr;   // in launch order: cluster b steps problem perm[b]
  std::vector<int> perm;       // launch order of the problems
  std::vector<ProbDesc> ldesc; // host copy in launch order (the source of the last upload)
  Buffers buf;
  StepLayout lay = {};
  int threads = 512;
  int *d_status = nullptr;
  double *d_sums = nullptr;
  double *d_rse_part = nullptr;   // per-CTA sums of the relative error, problem with the most tiles
  long long rse_part_n = 0;
  long long *d_t = nullptr;   // device-resident iteration counter (trsgd_step_counter)
  std::vector<const void *> X;
  int64_t t_next = 0;
  int64_t launches = 0;
  bool dbg = false;
  bool optimal = false;   // problem 0 samples from the optimal distribution
  bool grid = false;      // whole-GPU path (grid.cu) instead of the fused cluster kernel
  GridPath gp = {};
  GdBuffers gdb;          // full-gradient iterations (trsgd_gd_step), allocated at first use
  bool gd_ready = false;
  OptBuffers opt = {};
  size_t dbg_bytes[8] = {};
  void *dbg_ptr[8] = {};
};

// Limits of the fused cluster kernel (ranks held in registers, one problem
// per cluster in shared memory).
static bool cluster_fits(const trsgd_config *cfg, int32_t np) {
  for (int p = 0; p < np; ++p) {
    const trsgd_config &c = cfg[p];
    if (c.dist == TRSGD_DIST_OPTIMAL && np > 1) return false;
    for (int k = 0; k < c.N; ++k) {
      if (c.R[k] > kMaxRank) return false;
      const int64_t Q = c.R[k] * c.R[(k + 1) % c.N];
      if (Q > kMaxQPlain) return false;
      if (c.variant == TRSGD_SCALED && Q > kMaxQScaled) return false;
    }
  }
  return true;
}

// Limits of the whole-GPU path (grid.cu).
static bool grid_fits(const trsgd_config *cfg, int32_t np) {
  if (np != 1) return false;
  const trsgd_config &c = cfg[0];
  if (c.dist != TRSGD_DIST_UNIFORM || c.prec == TRSGD_FP64) return false;
  if (c.prec == TRSGD_FP32 && c.fp32_units == TRSGD_FP32_FMA) return false;   // pieces only
  if (c.J > (1LL << 24) || c.J_H > (1LL << 24)) return false;
  for (int k = 0; k < c.N; ++k) {
    if (c.R[k] > 32 || c.R[k] * c.R[(k + 1) % c.N] > 512) return false;
    if (c.variant == TRSGD_SCALED && c.R[k] * c.R[(k + 1) % c.N] > kGridScaledMaxQ) return false;
    if (c.I[k] > (1LL << 24)) return false;
  }
  return true;
}

static trsgd_status validate(const trsgd_config *cfg, int32_t np) {
  if (!cfg || np < 1) return TRSGD_EINVAL;
  for (int p = 0; p < np; ++p) {
    const trsgd_config &c = cfg[p];
    if (c.N < 2 || c.N > TRSGD_MAX_ORDER) return TRSGD_EINVAL;
    for (int k = 0; k < c.N; ++k) {
      if (c.I[k] < 1 || c.I[k] > (1LL << 30)) return TRSGD_EINVAL;
      if (c.R[k] < 1 || c.R[k] > 4096) return TRSGD_EINVAL;
    }
    if (c.J < 1 || c.J > (1LL << 30) || c.J_H < 0) return TRSGD_EINVAL;
    if (c.dist < 0 || c.dist > 3 || c.variant < 0 || c.variant > 1 || c.rule < 0 || c.rule > 1)
      return TRSGD_EINVAL;
    if (c.prec < 0 || c.prec > 2 || c.x_dtype < 0 || c.x_dtype > 2) return TRSGD_EINVAL;
    if (!std::isfinite(c.alpha) || !std::isfinite(c.eta) || !std::isfinite(c.b) ||
        !std::isfinite(c.eps) || !std::isfinite(c.damping))
      return TRSGD_EINVAL;
    if (c.damping < 0 || c.b < 0 || c.eps < 0 || c.eta < 0) return TRSGD_EINVAL;
    double numel = 1;
    for (int k = 0; k < c.N; ++k) numel *= (double)c.I[k];
    if (numel > 9.0e15) return TRSGD_EINVAL;
    if (c.prec != cfg[0].prec || c.x_dtype != cfg[0].x_dtype) return TRSGD_EINVAL;
    if (c.prec == TRSGD_FP64 && c.x_dtype != TRSGD_DTYPE_F64) return TRSGD_EINVAL;
    if (c.prec == TRSGD_FP32 && c.x_dtype != TRSGD_DTYPE_F32) return TRSGD_EINVAL;
    if (c.prec == TRSGD_BF16_MIXED && c.x_dtype == TRSGD_DTYPE_F64) return TRSGD_EINVAL;
    if (c.path < TRSGD_PATH_AUTO || c.path > TRSGD_PATH_GRID || c.path != cfg[0].path)
      return TRSGD_EINVAL;
    if ((c.fp32_units != TRSGD_FP32_PIECES && c.fp32_units != TRSGD_FP32_FMA) || c.fp32_units != cfg[0].fp32_units)
      return TRSGD_EINVAL;
  }
  // this build
  const bool cf = cluster_fits(cfg, np), gf = grid_fits(cfg, np);
  if (cfg[0].path == TRSGD_PATH_CLUSTER && !cf) return TRSGD_EUNSUPPORTED;
  if (cfg[0].path == TRSGD_PATH_GRID && !gf) return TRSGD_EUNSUPPORTED;
  if (!cf && !gf) return TRSGD_EUNSUPPORTED;
  return TRSGD_OK;
}

// Shared-memory layout for cluster size C (returns false if it does not fit).
// Fixed part: barrier, scalars, per-sample indices/columns/weights, fibers,
// Z and Z^T.  Tail region [off_reg, total): G_n chunk / partial gradient
// (reg), the FP64 Gram (scaled), the owned rows; the staged slices of the
// chain and the CDF scratch alias the same tail.
static bool make_layout_p(const trsgd_handle &h, int C, int tcp, bool tab, StepLayout &L) {
  const size_t st = h.core_dtype == 0 ? 8 : 4;
  const size_t sx = dtype_size(h.xc_dtype);
  int Imax = 1, Qmax = 1, Jmax = 1, QH = 0;
  size_t sbq = 0;   // max over problems and modes of sum_{k != n} padded Q_k
  int pst = 1;      // max over problems and modes of R_{n+1} * max_k R_k
  bool scaled = false;
  for (const auto &c : h.cfg) {
    Jmax = std::max(Jmax, (int)c.J);
    size_t qsum = 0;
    for (int k = 0; k < c.N; ++k) qsum += rup((size_t)(c.R[k] * c.R[(k + 1) % c.N]), 16 / st);
    for (int k = 0; k < c.N; ++k) {
      Imax = std::max(Imax, (int)c.I[k]);
      const int Q = (int)(c.R[k] * c.R[(k + 1) % c.N]);
      Qmax = std::max(Qmax, Q);
      if (c.variant == TRSGD_SCALED) QH = std::max(QH, Q);
      sbq = std::max(sbq, qsum - rup((size_t)Q, 16 / st));
    }
    int rmx = 1;
    for (int k = 0; k < c.N; ++k) rmx = std::max<int>(rmx, (int)c.R[k]);
    for (int k = 0; k < c.N; ++k) pst = std::max<int>(pst, (int)c.R[(k + 1) % c.N] * rmx);
    scaled |= c.variant == TRSGD_SCALED;
  }
  L = {};
  L.C = C;
  L.cw0 = (scaled && C > 1) ? 1 : 0;
  L.JB = (Jmax + (C - L.cw0) - 1) / (C - L.cw0);
  const bool tc = tcp > 0;   // tensor-core path with tcp BF16 pieces per operand
  L.tcp = tcp;
  const size_t JB4 = rup((size_t)L.JB, 4);
  L.ldxs = (int)rup((size_t)Imax, tc ? 8 : 4);
  {
    int q = (int)rup((size_t)Qmax, 4);
    if (st == 4) { while (q % 32 != 4) ++q; }
    else { while (q % 16 != 2) ++q; }
    L.ldq = q;
  }
  L.ldg = (int)rup((size_t)Qmax, 4);
  L.QH = scaled ? QH : 0;
  L.qp = (int)rup((size_t)Qmax, 16);
  L.jbp = (int)rup((size_t)L.JB, 16);
  if (tc && (L.qp > 256 || L.jbp > 256)) return false;
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = rup(off, align);
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.off_bar = take(32, 16);   // fibers, MMA completion, G_n pieces
  L.off_misc = take(64, 16);
  L.off_const = take(32 * 8, 16);
  L.off_ord = take(3 * kMaxOrder * 4, 16);   // chain order, staged-slice offsets and pitches
  // leverage / Euclidean: the CDF (u64) and p (f64) of the sampled cores of a step
  L.tab_ok = 0;
  if (tab) {
    size_t tb = 0;
    for (const auto &c : h.cfg) {
      if (c.dist != TRSGD_DIST_LEVERAGE && c.dist != TRSGD_DIST_EUCLIDEAN) continue;
      for (int n = 0; n < c.N; ++n) {
        size_t b = 0;
        for (int k = 0; k < c.N; ++k)
          if (k != n) b += (size_t)c.I[k] * 16;
        tb = std::max(tb, b);
      }
    }
    if (tb > 0) {
      L.off_tab = take(tb, 16);
      L.tab_ok = 1;
    }
  }
  L.off_desc = take(rup(sizeof(ProbDesc), 16), 16);
  L.off_idx = take((size_t)L.JB * kMaxOrder * 4, 16);
  L.off_col = take((size_t)L.JB * 8, 16);
  L.off_wt = take(JB4 * st, 16);
  L.off_x = take(JB4 * L.ldxs * (tc ? sx : std::max(sx, st)), 128);
  L.off_z = take(JB4 * L.ldq * st, 128);
  {
    int JHmax = 0;
    for (const auto &c : h.cfg)
      if (c.variant == TRSGD_SCALED) JHmax = std::max(JHmax, (int)c.J_H);
    L.JBH = (JHmax + C - 1) / C;
    if (L.JBH > 0) {
      const size_t JBH4 = rup((size_t)L.JBH, 4);
      L.off_hz = take(JBH4 * L.ldq * st, 128);
      L.off_hidx = take((size_t)L.JBH * kMaxOrder * 4, 16);
      L.off_hw = take(JBH4 * st, 16);
    }
  }
  for (int k = 0; k < tcp; ++k) L.off_zp[k] = take((size_t)L.jbp * L.qp * 2, 128);
  const size_t limit = (size_t)step_max_smem() - 1024;
  const size_t tail0 = rup(off, 128);
  if (tail0 >= limit) return false;
  const size_t avail = limit - tail0;
  const size_t h64b = scaled ? (size_t)QH * (QH | 1) * 8 : 0;   // Gram, then the factor at an odd pitch
  const size_t hdb = scaled ? (size_t)QH * 8 : 0;
  // rows of g a CTA owns: per chunk of TI rows ceil(TI / C); the scaled
  // variant keeps them for every chunk until the solve
  auto own_rows_for = [&](int TI) {
    return scaled ? (Imax + C - 1) / C + (Imax + TI - 1) / TI : (TI + C - 1) / C + 1;
  };
  auto reg_bytes = [&](int ti) {
    size_t reg = std::max((size_t)ti * L.ldg, (size_t)ti * L.ldq);
    if (scaled) reg = std::max(reg, (size_t)QH * L.ldq);
    size_t b = reg * st;
    if (scaled)   // the direction's blocked solves: inverted diagonal blocks and one warp's buffer at least
      b = std::max(b, (size_t)gram_solve_scratch(QH, 1) * 8);
    if (tcp == 2)   // split-BF16 G chunk (hi, lo) | partial gradient FP32 + Ew tile
      b = std::max(std::max(b, (size_t)2 * 128 * L.qp * 2),
                   rup((size_t)128 * L.ldq * st, 128) + (size_t)128 * L.jbp * 2);
    if (tcp == 3)   // G pieces, then the Ew pieces, then the FP32 partial, in turn (each dead
                    // once the tensor cores have read it)
      b = std::max(b, std::max((size_t)3 * 128 * L.qp * 2, (size_t)3 * 128 * L.jbp * 2));
    return b;
  };
  auto tail_bytes = [&](int ti) {
    return rup(reg_bytes(ti), 128) + rup(h64b, 16) + rup(hdb, 16) + (size_t)own_rows_for(ti) * L.ldq * st + 64;
  };
  int TI = tc ? 128 : (int)rup((size_t)Imax, 4);
  while (!tc && TI > 4 && tail_bytes(TI) > avail) TI = std::max(4, (TI * 7 / 8) & ~3);
  if (tail_bytes(TI) > avail) return false;
  L.TI = TI;
  L.rows_own = own_rows_for(TI);
  L.nsolve = 0;
  if (scaled) {   // as many solving warps (up to 16) as the reg region has buffers for
    const size_t spare = reg_bytes(TI) - (size_t)gram_solve_scratch(QH, 0) * 8;
    L.nsolve = (int)std::min<size_t>(std::min<size_t>(16, (size_t)L.rows_own), spare / ((size_t)(QH + kGsB) * 8));
  }
  off = tail0;
  L.off_reg = take(reg_bytes(TI), 128);
  L.off_ew = tcp == 3 ? L.off_reg : L.off_reg + rup((size_t)128 * L.ldq * st, 128);
  L.off_sb = L.off_reg;
  if (scaled) {
    L.off_h64 = take(h64b, 16);
    L.off_hdiag = take(hdb, 16);
  }
  L.off_gown = take((size_t)L.rows_own * L.ldq * st, 16);
  size_t end = std::max(off, tail0 + (size_t)Imax * 16);
  // staged slices followed by the two chain buffers, all aliasing the tail
  L.pstride = pst;
  // for all JB samples if they fit, else for the largest group of 32k (or
  // fewer) samples that does; the chain then runs group by group
  auto sb_need = [&](int s) {
    return rup((size_t)s * sbq * st, 128) + 2 * rup((size_t)s * pst * st, 128);
  };
  int sbj = L.JB;
  while (sbj > 0 && tail0 + sb_need(sbj) > limit) sbj = sbj > 32 ? (sbj - 1) / 32 * 32 : sbj - 1;
  const size_t sb_bytes = rup((size_t)sbj * sbq * st, 128);
  const size_t pb_bytes = rup((size_t)sbj * pst * st, 128);
  L.sbj = std::max(sbj, 1);
  L.off_p0 = tail0 + sb_bytes;
  L.off_p1 = L.off_p0 + pb_bytes;
  L.sb_ok = sbj > 0 ? 1 : 0;
  if (L.sb_ok) end = std::max(end, tail0 + sb_need(sbj));
  // the leverage table of the updated core is rebuilt in the tail by CTA 0
  for (const auto &c : h.cfg) {
    if (c.dist != TRSGD_DIST_LEVERAGE) continue;
    for (int k = 0; k < c.N; ++k)
      end = std::max(end, tail0 + leverage_scratch_bytes((int)c.I[k], (int)(c.R[k] * c.R[(k + 1) % c.N]), st));
  }
  // the tensor-core path allocates all 512 TMEM columns: keep one CTA per SM
  if (tc) end = std::max(end, (size_t)120 * 1024);
  L.total = rup(end, 128);
  return L.total <= limit;
}

// BF16-mixed: two pieces; FP32: three pieces when they fit, else the FMA
// units; FP64: the FMA units.
static bool make_layout(const trsgd_handle &h, int C, StepLayout &L) {
  // with the staged sampling tables if they fit, else without
  for (int tab = 1; tab >= 0; --tab) {
    if (h.xc_dtype == TRSGD_DTYPE_BF16) {
      if (make_layout_p(h, C, 2, tab, L)) return true;
      continue;
    }
    if (h.core_dtype == 1 && h.fp32_pieces && make_layout_p(h, C, 3, tab, L)) return true;
    if (make_layout_p(h, C, 0, tab, L)) return true;
  }
  return false;
}

static int default_cluster(const trsgd_handle &h) {
  int Jmax = 1;
  for (const auto &c : h.cfg) Jmax = std::max(Jmax, (int)c.J);
  int C = 1;
  while (C < 16 && (Jmax + C - 1) / C > 64) C *= 2;
  if (h.nprob > 1) C = std::min(C, std::max(1, 128 / h.nprob));
  return C;
}

// The preferred cluster size first, then smaller ones, then larger ones (a
// larger cluster splits the samples finer, so its per-CTA buffers shrink).
static trsgd_status choose_layout(trsgd_handle &h, int C) {
  int order[10], n = 0;
  for (int c = C; c >= 1; c /= 2) order[n++] = c;
  for (int c = C * 2; c <= 16; c *= 2) order[n++] = c;
  for (int i = 0; i < n; ++i) {
    StepLayout L;
    if (make_layout(h, order[i], L)) {
      h.lay = L;
      return from_cuda(step_kernel_prepare(h.core_dtype, h.xc_dtype, h.rmax, h.lay));
    }
  }
  return TRSGD_EUNSUPPORTED;
}

extern "C" {

const char *trsgd_status_string(trsgd_status s) {
  switch (s) {
    case TRSGD_OK: return "ok";
    case TRSGD_EINVAL: return "invalid argument";
    case TRSGD_ENOMEM: return "out of memory";
    case TRSGD_ECUDA: return "CUDA error";
    case TRSGD_ENUMERIC: return "numerical failure (non-finite step or non-SPD preconditioner)";
    case TRSGD_ETIMEOUT: return "bounded device wait timed out";
    case TRSGD_EUNSUPPORTED: return "unsupported configuration";
    case TRSGD_EBADINDEX: return "index out of range (debug build checks)";
  }
  return "unknown status";
}

// the whole-GPU path's second stream and its events
static void release_grid_streams(trsgd_handle *h) {
  if (h->gp.s2) {
    cudaStreamSynchronize(h->gp.s2);
    cudaStreamDestroy(h->gp.s2);
    h->gp.s2 = nullptr;
  }
  if (h->gp.ev_fork) cudaEventDestroy(h->gp.ev_fork);
  if (h->gp.ev_join) cudaEventDestroy(h->gp.ev_join);
  h->gp.ev_fork = h->gp.ev_join = nullptr;
}

// The descriptors in launch order: batched problems are stepped by one
// cluster each, in order of decreasing work (sum over the modes of
// I_n R_n R_{n+1} |F|), so that when the clusters run in waves the largest
// problems share the first wave and the last wave holds the smallest.
static void launch_order(trsgd_handle *h) {
  const int P = h->nprob;
  std::vector<double> cost(P, 0.0);
  for (int p = 0; p < P; ++p) {
    const trsgd_config &c = h->cfg[p];
    for (int k = 0; k < c.N; ++k) cost[p] += (double)c.I[k] * (double)(c.R[k] * c.R[(k + 1) % c.N]) * (double)c.J;
  }
  h->perm.resize(P);
  for (int p = 0; p < P; ++p) h->perm[p] = p;
  std::stable_sort(h->perm.begin(), h->perm.end(), [&](int a, int b) { return cost[a] > cost[b]; });
}

static cudaError_t upload_descs(trsgd_handle *h) {
  h->ldesc.resize(h->nprob);
  for (int b = 0; b < h->nprob; ++b) h->ldesc[b] = h->hdesc[h->perm[b]];
  cudaError_t e = cudaMemcpyAsync(h->ddesc, h->ldesc.data(), sizeof(ProbDesc) * h->nprob, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

trsgd_status trsgd_init(const trsgd_config *cfg, int32_t nproblems, const void *const *X_dev,
                        void *const *cores_dev, void *stream, trsgd_handle **out) {
  if (!out) return TRSGD_EINVAL;
  *out = nullptr;
  trsgd_status st = validate(cfg, nproblems);
  if (st != TRSGD_OK) return st;
  if (!X_dev || !cores_dev) return TRSGD_EINVAL;
  int ncore = 0;
  for (int p = 0; p < nproblems; ++p) {
    if (!X_dev[p]) return TRSGD_EINVAL;
    for (int k = 0; k < cfg[p].N; ++k)
      if (!cores_dev[ncore + k]) return TRSGD_EINVAL;
    ncore += cfg[p].N;
  }
  trsgd_handle *h = new (std::nothrow) trsgd_handle();
  if (!h) return TRSGD_ENOMEM;
  h->nprob = nproblems;
  h->cfg.assign(cfg, cfg + nproblems);
  h->stream = static_cast<cudaStream_t>(stream);
  h->core_dtype = cfg[0].prec == TRSGD_FP64 ? 0 : 1;
  h->xc_dtype = cfg[0].prec == TRSGD_BF16_MIXED ? TRSGD_DTYPE_BF16 : cfg[0].x_dtype;
  h->fp32_pieces = cfg[0].fp32_units == TRSGD_FP32_PIECES ? 1 : 0;
  int rmax = 1;
  for (int p = 0; p < nproblems; ++p)
    for (int k = 0; k < cfg[p].N; ++k) rmax = std::max<int>(rmax, (int)cfg[p].R[k]);
  h->rmax = rmax;
  auto fail = [&](trsgd_status s) {
    release_grid_streams(h);
    delete h;
    return s;
  };
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return fail(TRSGD_ECUDA);
  if (prop.major < 10) return fail(TRSGD_EUNSUPPORTED);

  cudaError_t e;
  if ((e = h->buf.alloc((void **)&h->d_status, 16)) != cudaSuccess) return fail(from_cuda(e));
  if ((e = h->buf.alloc((void **)&h->d_sums, 16)) != cudaSuccess) return fail(from_cuda(e));
  if ((e = h->buf.alloc((void **)&h->d_t, 16)) != cudaSuccess) return fail(from_cuda(e));
  cudaMemsetAsync(h->d_status, 0, 16, h->stream);
  cudaMemsetAsync(h->d_t, 0, 16, h->stream);
  const size_t sxc = dtype_size(h->xc_dtype);
  const size_t score = h->core_dtype == 0 ? 8 : 4;
  h->hdesc.resize(nproblems);
  ncore = 0;
  for (int p = 0; p < nproblems; ++p) {
    const trsgd_config &c = cfg[p];
    ProbDesc &D = h->hdesc[p];
    std::memset(&D, 0, sizeof(D));
    D.N = c.N;
    D.J = (int)c.J;
    D.JH = c.variant == TRSGD_SCALED ? (int)c.J_H : 0;
    D.dist = c.dist;
    D.variant = c.variant;
    D.rule = c.rule;
    D.prec = c.prec;
    for (int k = 0; k < c.N; ++k) {
      D.I[k] = (int)c.I[k];
      D.R[k] = (int)c.R[k];
    }
    if (c.variant == TRSGD_SCALED) {   // factor of h and reciprocal pivots, written by CTA 0 each step
      size_t qm = 1;
      for (int k = 0; k < c.N; ++k) qm = std::max<size_t>(qm, (size_t)(c.R[k] * c.R[(k + 1) % c.N]));
      if ((e = h->buf.alloc(&D.lfac, (qm * qm + qm) * 8)) != cudaSuccess) return fail(from_cuda(e));
    }
    D.alpha = c.alpha;
    D.eta = c.eta;
    D.b = c.b;
    D.eps = c.eps;
    D.damping = c.damping;
    D.seed = c.seed;
    D.status = h->d_status;
    for (int k = 0; k < c.N; ++k) {
      const size_t qb = (size_t)c.R[k] * c.R[(k + 1) % c.N] * score;
      if (qb % 16 == 0 && ((uintptr_t)cores_dev[ncore + k] % 16) == 0) D.slice_tma |= 1 << k;
    }
    h->X.push_back(X_dev[p]);
    for (int k = 0; k < c.N; ++k) {
      D.cores[k] = cores_dev[ncore + k];
      // mode-major copy of X for mode k
      long long A = 1, B = 1;
      for (int m = 0; m < k; ++m) A *= c.I[m];
      for (int m = k + 1; m < c.N; ++m) B *= c.I[m];
      const long long ld = (long long)rup((size_t)c.I[k], 16 / sxc);
      void *copy = nullptr;
      if ((e = h->buf.alloc(&copy, (size_t)ld * A * B * sxc)) != cudaSuccess) return fail(from_cuda(e));
      if (ld != c.I[k]) cudaMemsetAsync(copy, 0, (size_t)ld * A * B * sxc, h->stream);
      if ((e = launch_mode_copy(c.x_dtype, h->xc_dtype, X_dev[p], copy, A, c.I[k], B, ld, h->stream)) !=
          cudaSuccess)
        return fail(from_cuda(e));
      D.xmode[k] = copy;
      D.ldx[k] = ld;
      const int64_t Q = c.R[k] * c.R[(k + 1) % c.N];
      if (c.rule == TRSGD_STEP_ADAGRAD) {
        if ((e = h->buf.alloc(&D.acc[k], (size_t)c.I[k] * Q * score)) != cudaSuccess) return fail(from_cuda(e));
        cudaMemsetAsync(D.acc[k], 0, (size_t)c.I[k] * Q * score, h->stream);
      }
      if (c.dist != TRSGD_DIST_UNIFORM) {
        if ((e = h->buf.alloc((void **)&D.prob[k], (size_t)c.I[k] * 8)) != cudaSuccess ||
            (e = h->buf.alloc((void **)&D.cdf[k], (size_t)c.I[k] * 8)) != cudaSuccess ||
            (e = h->buf.alloc((void **)&D.snorm[k], (size_t)c.I[k] * 8)) != cudaSuccess)
          return fail(from_cuda(e));
        if (c.dist == TRSGD_DIST_LEVERAGE &&
            (e = launch_leverage_table(h->core_dtype, D.cores[k], (int)c.I[k], (int)Q, D.prob[k], D.cdf[k],
                                       h->d_status, h->stream)) != cudaSuccess)
          return fail(from_cuda(e));
        if (c.dist == TRSGD_DIST_EUCLIDEAN &&
            (e = launch_euclid_table(h->core_dtype, D.cores[k], (int)c.I[k], (int)Q, D.snorm[k], D.prob[k],
                                     D.cdf[k], h->stream)) != cudaSuccess)
          return fail(from_cuda(e));
      }
    }
    ncore += c.N;
  }
  if (cfg[0].dist == TRSGD_DIST_OPTIMAL) {
    const trsgd_config &c = cfg[0];
    long long jnmax = 1;
    for (int n = 0; n < c.N; ++n) {
      long long jn = 1;
      for (int k = 0; k < c.N; ++k)
        if (k != n) jn *= c.I[k];
      jnmax = std::max(jnmax, jn);
    }
    const long long nb = (jnmax + 1023) / 1024;
    OptBuffers &b = h->opt;
    if ((e = h->buf.alloc((void **)&b.a, jnmax * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.q, jnmax * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.cdf, jnmax * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.bsum, nb * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.btot, nb * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.total, 16)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.idx, (size_t)c.J * c.N * 4)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.pf, (size_t)c.J * 8)) != cudaSuccess ||
        (e = h->buf.alloc((void **)&b.dims, kMaxOrder * 4)) != cudaSuccess)
      return fail(from_cuda(e));
    int dims[kMaxOrder] = {};
    for (int k = 0; k < c.N; ++k) dims[k] = (int)c.I[k];
    cudaMemcpyAsync(b.dims, dims, sizeof(dims), cudaMemcpyHostToDevice, h->stream);
    h->hdesc[0].ext_idx = b.idx;
    h->hdesc[0].ext_pf = b.pf;
    h->optimal = true;
  }
  // recording buffers sized for problem 0
  {
    const trsgd_config &c = cfg[0];
    size_t Imax = 1, Qmax = 1;
    for (int k = 0; k < c.N; ++k) {
      Imax = std::max<size_t>(Imax, c.I[k]);
      Qmax = std::max<size_t>(Qmax, c.R[k] * c.R[(k + 1) % c.N]);
    }
    const size_t J = c.J;
    h->dbg_bytes[TRSGD_DBG_MODE] = 4;
    h->dbg_bytes[TRSGD_DBG_IDX] = J * c.N * 4;
    h->dbg_bytes[TRSGD_DBG_PF] = J * 8;
    h->dbg_bytes[TRSGD_DBG_Z] = J * Qmax * score;
    h->dbg_bytes[TRSGD_DBG_E] = J * Imax * score;
    h->dbg_bytes[TRSGD_DBG_G] = Imax * Qmax * score;
    h->dbg_bytes[TRSGD_DBG_P] = Imax * Qmax * score;
    h->dbg_bytes[TRSGD_DBG_H] = Qmax * Qmax * 8;
  }
  if ((e = cudaMalloc((void **)&h->ddesc, sizeof(ProbDesc) * nproblems)) != cudaSuccess) return fail(from_cuda(e));
  h->buf.ptrs.push_back(h->ddesc);
  h->grid = cfg[0].path == TRSGD_PATH_GRID || !cluster_fits(cfg, nproblems);
  if (!h->grid) {
    st = choose_layout(*h, default_cluster(*h));
    if (st == TRSGD_EUNSUPPORTED && cfg[0].path == TRSGD_PATH_AUTO && grid_fits(cfg, nproblems)) h->grid = true;
    else if (st != TRSGD_OK) return fail(st);
  }
  // FP32 cores of plain problems: room for the BF16 pieces of every core in the
  // tensor-core operand tile layout (used by the launches that take the
  // tensor-core step; the layout's qp does not change with the cluster size)
  if (!h->grid && h->core_dtype == 1 && h->lay.qp <= 256) {
    for (int p = 0; p < nproblems; ++p) {
      ProbDesc &D = h->hdesc[p];
      if (cfg[p].variant == TRSGD_SCALED) continue;
      for (int k = 0; k < cfg[p].N; ++k) {
        const size_t b = (size_t)((cfg[p].I[k] + 127) / 128) * 3 * 128 * h->lay.qp * 2;
        if ((e = h->buf.alloc(&D.gpc[k], b)) != cudaSuccess) return fail(from_cuda(e));
        cudaMemsetAsync(D.gpc[k], 0, b, h->stream);
      }
    }
  }
  if (h->grid) {
    const trsgd_config &c = cfg[0];
    GridPath &g = h->gp;
    int Ii[kMaxOrder] = {}, Ri[kMaxOrder] = {};
    for (int k = 0; k < c.N; ++k) {
      Ii[k] = (int)c.I[k];
      Ri[k] = (int)c.R[k];
    }
    const int np = c.prec == TRSGD_BF16_MIXED ? 1 : 3;
    const int scaled = c.variant == TRSGD_SCALED ? 1 : 0;
    grid_layout(Ii, Ri, c.N, (int)c.J, np, scaled, (int)c.J_H, g);
    g.x_bf16 = h->xc_dtype == TRSGD_DTYPE_BF16 ? 1 : 0;
    g.w = (float)(1.0 / (double)c.J);
    const size_t bf = 2;
    for (int p = 0; p < 3; ++p) g.Gp[p] = g.Zp[p] = g.ZTp[p] = g.Ep[p] = nullptr;
    for (int p = 0; p < g.npz && e == cudaSuccess; ++p) {
      if ((e = h->buf.alloc((void **)&g.Zp[p], (size_t)g.Jp * g.ldz * bf)) != cudaSuccess ||
          (e = h->buf.alloc((void **)&g.ZTp[p], (size_t)g.QTp * g.ldzt * bf)) != cudaSuccess)
        break;
      cudaMemsetAsync(g.Zp[p], 0, (size_t)g.Jp * g.ldz * bf, h->stream);
      cudaMemsetAsync(g.ZTp[p], 0, (size_t)g.QTp * g.ldzt * bf, h->stream);
      if (p < np && ((e = h->buf.alloc((void **)&g.Gp[p], (size_t)g.Ip * g.ldg * bf)) != cudaSuccess ||
                     (e = h->buf.alloc((void **)&g.Ep[p], (size_t)g.Ip * g.lde * bf)) != cudaSuccess))
        break;
    }
    if (e == cudaSuccess) e = h->buf.alloc((void **)&g.gpart, g.gpart_elems * 4);
    if (e == cudaSuccess) e = h->buf.alloc((void **)&g.col, (size_t)c.J * 8);
    if (e == cudaSuccess && scaled) {
      int qmax = 1;
      for (int k = 0; k < c.N; ++k) qmax = std::max(qmax, Ri[k] * Ri[(k + 1) % c.N]);
      if ((e = h->buf.alloc((void **)&g.hpart, g.hpart_elems * 4)) == cudaSuccess &&
          (e = h->buf.alloc((void **)&g.Lfac, grid_scaled_factor_floats(qmax) * 4)) == cudaSuccess &&
          (e = h->buf.alloc((void **)&g.fac_ok, 16)) == cudaSuccess)
        e = grid_scaled_prepare();
      // the factorisation's own stream (beside the GEMMs of the same iteration)
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.s2, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev_fork, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev_join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = grid_prepare_gemm();
    if (e == cudaSuccess) e = grid_tensor_maps(Ri, c.N, g);
    // the fused BF16 kernel for the modes it takes, its cluster size per mode
    for (int k = 0; k < c.N; ++k)
      g.fz_S[k] = (np == 1 && !scaled && g.x_bf16) ? grid_fused_cluster(Ii[k], Ri[k] * Ri[(k + 1) % c.N], (int)c.J) : 0;
    if (e != cudaSuccess) return fail(from_cuda(e));
  }
  h->threads = 512;
  launch_order(h);
  if ((e = upload_descs(h)) != cudaSuccess) return fail(from_cuda(e));
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(from_cuda(e));
  *out = h;
  return TRSGD_OK;
}

static trsgd_status read_status(trsgd_handle *h) {
  int s = 0;
  cudaError_t e = cudaMemcpyAsync(&s, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  if (s == 0) return TRSGD_OK;
  cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
  if (s == kStatusTimeout) return TRSGD_ETIMEOUT;
  if (s == kStatusNumeric) return TRSGD_ENUMERIC;
  if (s == kStatusBadIndex) return TRSGD_EBADINDEX;
  return TRSGD_ECUDA;
}

static trsgd_status launch_steps(trsgd_handle *h, int64_t t0, int64_t nsteps) {
  if (h->grid) {   // the mode is drawn on the host; five kernels per iteration
    const ProbDesc &D = h->hdesc[0];
    for (int64_t t = t0; t < t0 + nsteps; ++t) {
      NvtxRange r("trsgd iteration (whole GPU)");
      const int n = draw_mode(D.seed, t, D.N);
      cudaError_t e = launch_grid_step(h->gp, D, n, t, h->dbg ? 1 : 0, h->stream);
      if (e != cudaSuccess) return from_cuda(e);
      h->launches += grid_step_kernels(h->gp, D, n);
    }
    return TRSGD_OK;
  }
  if (h->optimal) {   // per step: the optimal distribution of this step's mode, its draws, then the step
    const ProbDesc &D = h->hdesc[0];
    for (int64_t t = t0; t < t0 + nsteps; ++t) {
      NvtxRange r("trsgd iteration (optimal distribution)");
      const int n = draw_mode(D.seed, t, D.N);
      cudaError_t e = launch_optimal_sampling(h->core_dtype, h->xc_dtype, D.N, n, D.I, D.R,
                                              (const void *const *)D.cores, D.xmode[n], D.ldx[n], D.seed, t, D.J,
                                              h->opt, h->stream);
      if (e == cudaSuccess)
        e = launch_step(h->core_dtype, h->xc_dtype, h->rmax, h->ddesc, h->nprob, h->lay, h->threads, t, 1, nullptr,
                        h->stream);
      if (e != cudaSuccess) return from_cuda(e);
      ++h->launches;
    }
    return TRSGD_OK;
  }
  while (nsteps > 0) {
    NvtxRange r("trsgd step_cluster_kernel launch (K iterations)");
    const int n = (int)std::min<int64_t>(nsteps, 1 << 20);
    cudaError_t e = launch_step(h->core_dtype, h->xc_dtype, h->rmax, h->ddesc, h->nprob, h->lay, h->threads, t0,
                                n, nullptr, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    ++h->launches;
    t0 += n;
    nsteps -= n;
  }
  return TRSGD_OK;
}

trsgd_status trsgd_step(trsgd_handle *h, int64_t t) {
  if (!h || t < 0) return TRSGD_EINVAL;
  trsgd_status s = launch_steps(h, t, 1);
  if (s == TRSGD_OK) h->t_next = t + 1;
  return s;
}

trsgd_status trsgd_step_counter(trsgd_handle *h, int64_t T) {
  if (!h || T < 0 || T > (1 << 20)) return TRSGD_EINVAL;
  // the optimal distribution and the whole-GPU path draw the mode on the host
  if (h->optimal || h->grid) return TRSGD_EUNSUPPORTED;
  if (T == 0) return TRSGD_OK;
  cudaError_t e = launch_step(h->core_dtype, h->xc_dtype, h->rmax, h->ddesc, h->nprob, h->lay, h->threads, 0,
                              (int)T, h->d_t, h->stream);
  if (e == cudaSuccess) e = launch_advance_counter(h->d_t, T, 0, h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  ++h->launches;
  return TRSGD_OK;
}

trsgd_status trsgd_set_counter(trsgd_handle *h, int64_t t) {
  if (!h || t < 0) return TRSGD_EINVAL;
  cudaError_t e = launch_advance_counter(h->d_t, t, 1, h->stream);
  return e == cudaSuccess ? TRSGD_OK : from_cuda(e);
}

trsgd_status trsgd_rel_error(trsgd_handle *h, int32_t problem, const void *Xref_dev, double *out) {
  if (!h || !out || problem < 0 || problem >= h->nprob) return TRSGD_EINVAL;
  NvtxRange r("trsgd_rel_error");
  const trsgd_config &c = h->cfg[problem];
  const ProbDesc &D = h->hdesc[problem];
  // the reference is read in the cores' dtype: the caller's own X only when it has that dtype
  if (!Xref_dev && c.x_dtype != (h->core_dtype == 0 ? TRSGD_DTYPE_F64 : TRSGD_DTYPE_F32)) return TRSGD_EUNSUPPORTED;
  const void *ref = Xref_dev ? Xref_dev : h->X[problem];
  const long long np = reconstruct_partials(h->core_dtype, c.N, D.I, D.R);
  cudaError_t e = cudaSuccess;
  if (np > h->rse_part_n) {   // grown once to the largest problem evaluated
    if ((e = h->buf.alloc((void **)&h->d_rse_part, (size_t)np * sizeof(double))) != cudaSuccess)
      return from_cuda(e);
    h->rse_part_n = np;
  }
  e = launch_reconstruct(h->core_dtype, c.N, D.I, D.R, (const void *const *)D.cores, nullptr, ref, h->d_sums,
                         h->d_rse_part, h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  double sums[2];
  e = cudaMemcpyAsync(sums, h->d_sums, 16, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  *out = sums[1] > 0 ? std::sqrt(sums[0] / sums[1]) : std::sqrt(sums[0]);
  return read_status(h);
}

trsgd_status trsgd_run(trsgd_handle *h, int64_t t0, int64_t T, int64_t chunk, double tol,
                       double max_seconds, const void *Xref_dev, int64_t *steps_done, double *rse_out) {
  if (!h || T < 0 || t0 < 0) return TRSGD_EINVAL;
  if (steps_done) *steps_done = 0;
  if (rse_out) *rse_out = -1.0;
  const bool checks = tol > 0 || max_seconds > 0;
  if (chunk <= 0) chunk = checks ? std::max<int64_t>(1, std::min<int64_t>(T, 100)) : std::max<int64_t>(T, 1);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (checks) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, h->stream);
  }
  double device_s = 0.0;
  int64_t done = 0;
  trsgd_status st = TRSGD_OK;
  while (done < T) {
    const int64_t n = std::min(chunk, T - done);
    st = launch_steps(h, t0 + done, n);
    if (st != TRSGD_OK) break;
    done += n;
    h->t_next = t0 + done;
    if (checks) {
      cudaEventRecord(ev1, h->stream);
      cudaEventSynchronize(ev1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      device_s += ms * 1e-3;
      double r = -1.0;
      st = trsgd_rel_error(h, 0, Xref_dev, &r);
      if (st != TRSGD_OK) break;
      if (rse_out) *rse_out = r;
      cudaEventRecord(ev0, h->stream);   // evaluation time is not counted
      if ((tol > 0 && r <= tol) || (max_seconds > 0 && device_s >= max_seconds)) break;
    }
  }
  if (steps_done) *steps_done = done;
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (st != TRSGD_OK) return st;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  return read_status(h);
}

trsgd_status trsgd_reconstruct(int32_t N, const int64_t *I, const int64_t *R, int32_t dtype,
                               const void *const *cores_dev, void *X_dev, void *stream) {
  if (N < 2 || N > TRSGD_MAX_ORDER || !I || !R || !cores_dev || !X_dev) return TRSGD_EINVAL;
  if (dtype != TRSGD_DTYPE_F64 && dtype != TRSGD_DTYPE_F32) return TRSGD_EUNSUPPORTED;
  int Ii[TRSGD_MAX_ORDER], Ri[TRSGD_MAX_ORDER];
  for (int k = 0; k < N; ++k) {
    if (I[k] < 1 || R[k] < 1 || I[k] > (1LL << 30)) return TRSGD_EINVAL;
    if (R[k] > 32) return TRSGD_EUNSUPPORTED;
    if (!cores_dev[k]) return TRSGD_EINVAL;
    Ii[k] = (int)I[k];
    Ri[k] = (int)R[k];
  }
  return from_cuda(launch_reconstruct(dtype == TRSGD_DTYPE_F64 ? 0 : 1, N, Ii, Ri, cores_dev, X_dev, nullptr,
                                      nullptr, nullptr, static_cast<cudaStream_t>(stream)));
}

trsgd_status trsgd_sampled_loss_grad(int32_t N, const int64_t *I, const int64_t *R, int32_t n, int64_t J,
                                     const int32_t *idx_dev, const float *XS_dev, const float *w_dev,
                                     const float *const *cores_dev, float *const *grads_dev, float *loss_dev,
                                     void *stream) {
  if (N < 2 || N > TRSGD_MAX_ORDER || !I || !R || n < 0 || n >= N || J < 0 || J > (1LL << 30)) return TRSGD_EINVAL;
  if (!idx_dev || !XS_dev || !w_dev || !cores_dev || !loss_dev) return TRSGD_EINVAL;
  int Ii[TRSGD_MAX_ORDER], Ri[TRSGD_MAX_ORDER];
  for (int k = 0; k < N; ++k) {
    if (I[k] < 1 || R[k] < 1 || !cores_dev[k]) return TRSGD_EINVAL;
    if (grads_dev && !grads_dev[k]) return TRSGD_EINVAL;
    if (R[k] > 16) return TRSGD_EUNSUPPORTED;
    Ii[k] = (int)I[k];
    Ri[k] = (int)R[k];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
  for (int k = 0; k < N && grads_dev && e == cudaSuccess; ++k)
    e = cudaMemsetAsync(grads_dev[k], 0, (size_t)Ii[k] * Ri[k] * Ri[(k + 1) % N] * sizeof(float), s);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(launch_sampled_loss_grad(N, Ii, Ri, n, (int)J, idx_dev, XS_dev, w_dev, cores_dev,
                                            grads_dev, loss_dev, s));
}

trsgd_status trsgd_set_debug(trsgd_handle *h, int32_t on) {
  if (!h) return TRSGD_EINVAL;
  ProbDesc &D = h->hdesc[0];
  if (on && !h->dbg_ptr[0]) {
    for (int i = 0; i < 8; ++i) {
      cudaError_t e = h->buf.alloc(&h->dbg_ptr[i], h->dbg_bytes[i]);
      if (e != cudaSuccess) return from_cuda(e);
      cudaMemsetAsync(h->dbg_ptr[i], 0, h->dbg_bytes[i], h->stream);
    }
    D.dbg_n = (int *)h->dbg_ptr[TRSGD_DBG_MODE];
    D.dbg_idx = (int *)h->dbg_ptr[TRSGD_DBG_IDX];
    D.dbg_pf = (double *)h->dbg_ptr[TRSGD_DBG_PF];
    D.dbg_z = h->dbg_ptr[TRSGD_DBG_Z];
    D.dbg_e = h->dbg_ptr[TRSGD_DBG_E];
    D.dbg_g = h->dbg_ptr[TRSGD_DBG_G];
    D.dbg_p = h->dbg_ptr[TRSGD_DBG_P];
    D.dbg_h = (double *)h->dbg_ptr[TRSGD_DBG_H];
  }
  D.dbg = on ? 1 : 0;
  h->dbg = on != 0;
  return from_cuda(upload_descs(h));
}

trsgd_status trsgd_set_wait_limit(trsgd_handle *h, int64_t polls) {
  if (!h) return TRSGD_EINVAL;
  for (auto &D : h->hdesc) D.wait_limit = polls;
  return from_cuda(upload_descs(h));
}

trsgd_status trsgd_debug_index_bound(trsgd_handle *h, int32_t k, int64_t bound) {
  if (!h || h->nprob < 1) return TRSGD_EINVAL;
  for (const auto &c : h->cfg)
    if (k < 0 || k >= c.N || bound < 0 || bound > c.I[k]) return TRSGD_EINVAL;
  if (kDebugChecks) {
    for (auto &D : h->hdesc) D.dbg_bound[k] = (int)bound;
    return from_cuda(upload_descs(h));
  }
  return TRSGD_EUNSUPPORTED;   // the product build has no checks compiled in
}

trsgd_status trsgd_get_debug(trsgd_handle *h, int32_t item, void *out_host, size_t bytes, size_t *written) {
  if (!h || item < 0 || item > 7 || !out_host) return TRSGD_EINVAL;
  if (!h->dbg_ptr[item]) return TRSGD_EINVAL;
  const size_t n = std::min(bytes, h->dbg_bytes[item]);
  cudaError_t e = cudaMemcpyAsync(out_host, h->dbg_ptr[item], n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  if (written) *written = n;
  return read_status(h);
}

trsgd_status trsgd_adagrad_state(trsgd_handle *h, int32_t problem, int32_t core, void *host, size_t bytes,
                                 int32_t dir) {
  if (!h || !host || problem < 0 || problem >= h->nprob) return TRSGD_EINVAL;
  const trsgd_config &c = h->cfg[problem];
  if (core < 0 || core >= c.N || (dir != 0 && dir != 1)) return TRSGD_EINVAL;
  void *acc = h->hdesc[problem].acc[core];
  if (!acc) return TRSGD_EINVAL;
  const size_t need = (size_t)c.I[core] * c.R[core] * c.R[(core + 1) % c.N] * (h->core_dtype == 0 ? 8 : 4);
  if (bytes != need) return TRSGD_EINVAL;
  cudaError_t e = dir == 0 ? cudaMemcpyAsync(host, acc, need, cudaMemcpyDeviceToHost, h->stream)
                           : cudaMemcpyAsync(acc, host, need, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return from_cuda(e);
}

// The scaled variant's factorisation holds the 4 x 4 blocks of the Gram
// matrix's lower triangle in registers, at most two blocks per thread.
static bool threads_fit(const trsgd_handle &h, int T) {
  if (h.lay.QH <= 0) return true;
  const int Qb = (h.lay.QH + 3) / 4;
  return Qb * (Qb + 1) / 2 <= 2 * T;
}

trsgd_status trsgd_launch_shape(trsgd_handle *h, int32_t set, int32_t *cluster, int32_t *threads) {
  if (!h || !cluster || !threads) return TRSGD_EINVAL;
  if (h->grid) {   // whole-GPU path: no cluster; 256-thread GEMM CTAs
    if (set != 0) return TRSGD_EUNSUPPORTED;
    *cluster = 0;
    *threads = 256;
    return TRSGD_OK;
  }
  if (set == 0) {
    *cluster = h->lay.C;
    *threads = h->threads;
    return TRSGD_OK;
  }
  if (set != 1) return TRSGD_EINVAL;
  const int C = *cluster ? *cluster : h->lay.C;
  const int T = *threads ? *threads : h->threads;
  if (C < 1 || C > 16 || (C & (C - 1)) || (T != 128 && T != 256 && T != 512)) return TRSGD_EINVAL;
  if (!threads_fit(*h, T)) return TRSGD_EUNSUPPORTED;
  StepLayout L;
  if (!make_layout(*h, C, L)) return TRSGD_EUNSUPPORTED;
  cudaError_t e = step_kernel_prepare(h->core_dtype, h->xc_dtype, h->rmax, L);
  if (e != cudaSuccess) return from_cuda(e);
  h->lay = L;
  h->threads = T;
  return TRSGD_OK;
}

trsgd_status trsgd_autotune(trsgd_handle *h, int32_t steps_per_trial) {
  if (!h || steps_per_trial < 1) return TRSGD_EINVAL;
  if (h->grid) return TRSGD_OK;   // tile shapes follow from the problem sizes
  // scratch copies of every core so that the trial steps leave the cores unchanged
  std::vector<std::vector<void *>> saved(h->nprob);
  std::vector<std::vector<size_t>> sizes(h->nprob);
  Buffers scratch;
  const size_t score = h->core_dtype == 0 ? 8 : 4;
  for (int p = 0; p < h->nprob; ++p) {
    const trsgd_config &c = h->cfg[p];
    for (int k = 0; k < c.N; ++k) {
      const size_t b = (size_t)c.I[k] * c.R[k] * c.R[(k + 1) % c.N] * score;
      void *cp = nullptr;
      cudaError_t e = scratch.alloc(&cp, b);
      if (e != cudaSuccess) return from_cuda(e);
      cudaMemcpyAsync(cp, h->hdesc[p].cores[k], b, cudaMemcpyDeviceToDevice, h->stream);
      saved[p].push_back(cp);
      sizes[p].push_back(b);
      if (h->hdesc[p].acc[k]) {
        void *ap = nullptr;
        if ((e = scratch.alloc(&ap, b)) != cudaSuccess) return from_cuda(e);
        cudaMemcpyAsync(ap, h->hdesc[p].acc[k], b, cudaMemcpyDeviceToDevice, h->stream);
        saved[p].push_back(ap);
        sizes[p].push_back(b);
      }
    }
  }
  const StepLayout keep_lay = h->lay;
  const int keep_threads = h->threads;
  float best = 1e30f;
  StepLayout best_lay = keep_lay;
  int best_threads = keep_threads;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int C = 1; C <= 16; C *= 2) {
    StepLayout L;
    if (!make_layout(*h, C, L)) continue;
    if (step_kernel_prepare(h->core_dtype, h->xc_dtype, h->rmax, L) != cudaSuccess) continue;
    for (int T : {256, 512}) {
      if (!threads_fit(*h, T)) continue;
      h->lay = L;
      h->threads = T;
      if (launch_steps(h, 0, 1) != TRSGD_OK) { cudaGetLastError(); continue; }  // warm-up
      cudaEventRecord(a, h->stream);
      if (launch_steps(h, 1, steps_per_trial) != TRSGD_OK) { cudaGetLastError(); continue; }
      cudaEventRecord(b, h->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) { cudaGetLastError(); continue; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) {
        best = ms;
        best_lay = L;
        best_threads = T;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  // restore the cores, the AdaGrad sums and the sampling tables
  for (int p = 0; p < h->nprob; ++p) {
    const trsgd_config &c = h->cfg[p];
    size_t s = 0;
    for (int k = 0; k < c.N; ++k) {
      cudaMemcpyAsync(h->hdesc[p].cores[k], saved[p][s], sizes[p][s], cudaMemcpyDeviceToDevice, h->stream);
      ++s;
      if (h->hdesc[p].acc[k]) {
        cudaMemcpyAsync(h->hdesc[p].acc[k], saved[p][s], sizes[p][s], cudaMemcpyDeviceToDevice, h->stream);
        ++s;
      }
      if (c.dist == TRSGD_DIST_EUCLIDEAN)
        launch_euclid_table(h->core_dtype, h->hdesc[p].cores[k], (int)c.I[k], (int)(c.R[k] * c.R[(k + 1) % c.N]),
                            h->hdesc[p].snorm[k], h->hdesc[p].prob[k], h->hdesc[p].cdf[k], h->stream);
      if (c.dist == TRSGD_DIST_LEVERAGE)
        launch_leverage_table(h->core_dtype, h->hdesc[p].cores[k], (int)c.I[k], (int)(c.R[k] * c.R[(k + 1) % c.N]),
                              h->hdesc[p].prob[k], h->hdesc[p].cdf[k], h->d_status, h->stream);
    }
  }
  h->lay = best_lay;
  h->threads = best_threads;
  cudaError_t e = step_kernel_prepare(h->core_dtype, h->xc_dtype, h->rmax, h->lay);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  return read_status(h);
}

int64_t trsgd_launch_count(const trsgd_handle *h) { return h ? h->launches : -1; }

trsgd_status trsgd_shard_plan(trsgd_handle *h, int64_t t, int32_t rank, int32_t world, trsgd_shard *out) {
  if (!h || !out || t < 0 || world < 1 || rank < 0 || rank >= world) return TRSGD_EINVAL;
  if (!h->grid) return TRSGD_EUNSUPPORTED;
  const ProbDesc &D = h->hdesc[0];
  const GridPath &g = h->gp;
  const int n = draw_mode(D.seed, t, D.N);
  const long long Q = (long long)D.R[n] * D.R[(n + 1) % D.N];
  trsgd_shard sh = {};
  sh.mode = n;
  auto deal = [&](long long total, long long unit, int64_t &a, int64_t &b, int64_t &cnt, int64_t &mx) {
    const long long U = (total + unit - 1) / unit;
    const long long u0 = U * rank / world, u1 = U * (rank + 1) / world;
    a = std::min<long long>(u0 * unit, total);
    b = std::min<long long>(u1 * unit, total);
    cnt = u1 - u0;
    mx = (U + world - 1) / world;
  };
  sh.gunit = grid_split_unit(g, D, n, D.J);
  deal(D.J, sh.gunit, sh.j0, sh.j1, sh.gsplits, sh.gsplits_max);
  sh.gelems = (long long)D.I[n] * Q;
  if (g.scaled) {
    const long long JH = g.JH > 0 ? g.JH : D.J;
    sh.hunit = grid_gram_unit(g, D, n, JH);
    if (g.JH > 0) {
      deal(JH, sh.hunit, sh.h0, sh.h1, sh.hsplits, sh.hsplits_max);
    } else {   // H = F: the Gram over this rank's F samples, in Gram units (whole ones: hunit divides gunit)
      sh.h0 = sh.j0;
      sh.h1 = sh.j1;
      sh.hsplits = (sh.j1 - sh.j0 + sh.hunit - 1) / sh.hunit;
      sh.hsplits_max = sh.gsplits_max * (sh.gunit / sh.hunit);
    }
    sh.helems = Q * Q;
  }
  *out = sh;
  return TRSGD_OK;
}

trsgd_status trsgd_step_partial(trsgd_handle *h, int64_t t, const trsgd_shard *plan, float *gpart_dev,
                                float *hpart_dev) {
  if (!h || !plan || t < 0 || !gpart_dev) return TRSGD_EINVAL;
  if (!h->grid) return TRSGD_EUNSUPPORTED;
  const ProbDesc &D = h->hdesc[0];
  const GridPath &g = h->gp;
  const int n = draw_mode(D.seed, t, D.N);
  if (plan->mode != n || (g.scaled && !hpart_dev)) return TRSGD_EINVAL;
  if (plan->gsplits > plan->gsplits_max || plan->hsplits > plan->hsplits_max) return TRSGD_EINVAL;
  cudaError_t e = launch_grid_partial(g, D, n, t, plan->j0, plan->j1, g.JH > 0 ? plan->h0 : 0,
                                      g.JH > 0 ? plan->h1 : 0, h->dbg ? 1 : 0, gpart_dev, hpart_dev, h->stream,
                                      nullptr);
  if (e == cudaErrorInvalidValue) return TRSGD_EINVAL;
  // zero partials up to the common count, so that a gather of every rank's
  // buffer sums to the same values
  if (e == cudaSuccess && plan->gsplits_max > plan->gsplits)
    e = cudaMemsetAsync(gpart_dev + plan->gsplits * plan->gelems, 0,
                        (size_t)(plan->gsplits_max - plan->gsplits) * plan->gelems * sizeof(float), h->stream);
  if (e == cudaSuccess && g.scaled && plan->hsplits_max > plan->hsplits)
    e = cudaMemsetAsync(hpart_dev + plan->hsplits * plan->helems, 0,
                        (size_t)(plan->hsplits_max - plan->hsplits) * plan->helems * sizeof(float), h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  // prepare, samples, transposes, residual, gradient (+ H samples and transposes), Gram
  h->launches += 4 + g.npz + (g.scaled ? (g.JH > 0 ? 2 + g.npz : 1) : 0);
  return TRSGD_OK;
}

trsgd_status trsgd_step_apply(trsgd_handle *h, int64_t t, const float *gparts_dev, int64_t gsplits,
                              const float *hparts_dev, int64_t hsplits) {
  if (!h || t < 0 || !gparts_dev || gsplits < 1 || gsplits > (1 << 20)) return TRSGD_EINVAL;
  if (!h->grid) return TRSGD_EUNSUPPORTED;
  const GridPath &g = h->gp;
  if (g.scaled && (!hparts_dev || hsplits < 1 || hsplits > (1 << 20))) return TRSGD_EINVAL;
  const ProbDesc &D = h->hdesc[0];
  const int n = draw_mode(D.seed, t, D.N);
  cudaError_t e = launch_grid_apply(g, D, n, gparts_dev, (int)gsplits, hparts_dev, (int)hsplits, h->dbg ? 1 : 0,
                                    h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  h->launches += g.scaled ? 2 : 1;
  h->t_next = t + 1;
  return TRSGD_OK;
}

trsgd_status trsgd_gd_step(trsgd_handle *h, int32_t scaled, double alpha, double damping) {
  if (!h || (scaled != 0 && scaled != 1) || !std::isfinite(alpha) || !std::isfinite(damping) || damping < 0)
    return TRSGD_EINVAL;
  const trsgd_config &c = h->cfg[0];
  if (h->xc_dtype == TRSGD_DTYPE_BF16 || c.dist != TRSGD_DIST_UNIFORM) return TRSGD_EUNSUPPORTED;
  for (int k = 0; k < c.N; ++k) {
    const int64_t Q = c.R[k] * c.R[(k + 1) % c.N];
    if (c.R[k] > 16 || (scaled && Q > 128)) return TRSGD_EUNSUPPORTED;
  }
  const ProbDesc &D = h->hdesc[0];
  GdArgs a = {};
  a.N = c.N;
  for (int k = 0; k < c.N; ++k) {
    a.I[k] = (int)c.I[k];
    a.R[k] = (int)c.R[k];
    a.cores[k] = D.cores[k];
    a.xmode[k] = D.xmode[k];
    a.ldx[k] = D.ldx[k];
  }
  for (int n = 0; n < c.N; ++n) {
    long long Jn = 1;
    for (int k = 0; k < c.N; ++k)
      if (k != n) Jn *= c.I[k];
    a.J[n] = Jn;
  }
  if (!h->gd_ready) {
    const size_t st = h->core_dtype == 0 ? 8 : 4;
    size_t zmax = 0, pmax = 0;
    int qmax = 1;
    for (int n = 0; n < c.N; ++n) {
      const size_t Q = (size_t)(c.R[n] * c.R[(n + 1) % c.N]);
      zmax = std::max(zmax, (size_t)a.J[n] * Q);
      pmax = std::max(pmax, std::max((size_t)c.I[n], Q) * Q);
      qmax = std::max(qmax, (int)Q);
    }
    cudaError_t e = h->buf.alloc(&h->gdb.Z, zmax * st);
    if (e == cudaSuccess) e = h->buf.alloc(&h->gdb.part, (size_t)h->gdb.max_chunks * pmax * st);
    for (int n = 0; n < c.N && e == cudaSuccess; ++n) {
      const size_t Q = (size_t)(c.R[n] * c.R[(n + 1) % c.N]);
      e = h->buf.alloc(&h->gdb.M[n], (size_t)c.I[n] * Q * st);
      void *g = nullptr;
      if (e == cudaSuccess) e = h->buf.alloc(&g, Q * Q * sizeof(double));
      h->gdb.Gam[n] = static_cast<double *>(g);
    }
    void *f = nullptr;
    if (e == cudaSuccess) e = h->buf.alloc(&f, (size_t)qmax * qmax * sizeof(double));
    h->gdb.fac = static_cast<double *>(f);
    if (e == cudaSuccess) e = gd_prepare();
    if (e != cudaSuccess) return from_cuda(e);
    h->gd_ready = true;
  }
  cudaError_t e = launch_gd_iteration(h->core_dtype, a, scaled, alpha, damping, h->gdb, h->d_status, h->stream);
  if (e != cudaSuccess) return from_cuda(e);
  h->launches += (6 + (scaled ? 1 : 0)) * c.N;   // per mode: Z, 2 x (A^T Z, reduce), factor, update
  return TRSGD_OK;
}

int32_t trsgd_tensor_pieces(const trsgd_handle *h) {
  if (!h) return -1;
  return h->grid ? h->gp.np : h->lay.tcp;
}

void trsgd_destroy(trsgd_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  release_grid_streams(h);
  delete h;
}

}  // extern "C"
