// Internal descriptors shared by the host library and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

namespace trsgd {

// One TR problem as the step kernel sees it.
struct ProbDesc {
  int N, J, dist, variant, rule, prec;
  int JH;                         // |H| of the scaled variant (0: H = F)
  int I[8], R[8];
  double alpha, eta, b, eps, damping;
  unsigned long long seed;
  void *cores[8];                 // G_{k(2)}, core dtype
  const void *xmode[8];           // mode-major copies: fiber col of X_[k] at xmode[k] + col*ldx[k]
  long long ldx[8];               // row stride of xmode[k] in elements (16-byte multiple)
  void *acc[8];                   // AdaGrad sums (core dtype), or null
  // FP32 cores on the tensor-core path, plain variant: core k as BF16 pieces in
  // the operand tile layout (per chunk of 128 rows, per piece, a no-swizzle
  // K-major 128 x qp tile; 3 pieces of room), rebuilt by every launch and kept
  // current by the update; null: G_n is converted per chunk instead
  void *gpc[8];
  double *prob[8];                // p_k (non-uniform distributions)
  unsigned long long *cdf[8];     // inclusive prefix sums of round(p_k * 2^52)
  double *snorm[8];               // Euclidean slice norms ||G_k(i)||_F^2
  int slice_tma;                  // bit k set: core k's slices can be bulk-copied (16-byte rows)
  void *lfac;                     // scaled variant: Cholesky factor of h (column-major, Q x Q) then
                                  // the Q reciprocal pivots, in the Gram-solve scalar (8 bytes each)
  const int *ext_idx;             // optimal distribution: this step's indices [J][N] and p_F [J]
  const double *ext_pf;
  // polls of a bounded mbarrier wait before it latches TRSGD_ETIMEOUT (0: the
  // default 2^22; negative: none, every first try times out); the timed-out
  // operation is then drained by a second wait of the default length
  long long wait_limit;
  // upper bounds of the debug build's checks of the drawn indices of core k
  // (0: I_k); see trsgd_debug_index_bound
  int dbg_bound[8];
  // recording of intermediates (problem 0 only)
  int dbg;
  int *dbg_n, *dbg_idx;
  double *dbg_pf, *dbg_h;
  void *dbg_z, *dbg_e, *dbg_g, *dbg_p;
  int *status;
};

// Shared-memory layout of the step kernel (byte offsets), identical for all
// CTAs of a launch.
struct StepLayout {
  int C;          // CTAs per cluster (per problem)
  int JB;         // max samples per CTA
  int ldxs;       // fiber rows in smem (elements of the fiber dtype; multiple of 4)
  int ldq;        // Z rows (elements; = 4 mod 32 for conflict-free n-major reads)
  int ldg;        // G_n chunk rows (elements; multiple of 4)
  int TI;         // rows of G_n per chunk (multiple of 4)
  int QH;         // max Q of the scaled variant (0: none)
  int rows_own;   // max rows of g owned by one CTA
  int sb_ok;      // sampled slices staged in shared memory (else read through L2)
  int sbj;        // samples whose slices are staged at a time (the chain runs per group)
  int tab_ok;     // leverage / Euclidean tables of the sampled cores staged in shared memory
  int pstride;    // per-sample stride of the chain intermediates
  int qp, jbp;    // tensor-core path: Q and samples padded to 16 (tile extents)
  int tcp;        // BF16 pieces per tensor-core operand: 2 (BF16-mixed), 3 (FP32), 0 (FMA units)
  int nsolve;     // scaled variant: warps that solve rows of the direction (one buffer each in the reg region)
  // off_sb aliases the region [off_reg, total): the staged slices are dead
  // before the Gram / chunk buffers and the CDF scratch are written
  size_t off_desc, off_idx, off_col, off_wt, off_bar, off_x, off_z, off_reg, off_h64,
      off_hdiag, off_gown, off_misc, off_const, off_sb, off_p0, off_p1, off_zp[3], off_ew, off_ord, off_tab,
      off_hz, off_hidx, off_hw, total;
  int JBH;        // max Hessian-batch samples per CTA
  int cw0;        // first CTA that takes samples: 1 for the scaled variant with C > 1 (CTA 0
                  // factorises the Gram matrix meanwhile), else 0
};

// Block size of the scaled variant's blocked triangular solves (gramsolve.cuh):
// the diagonal blocks of the Gram factor L are kGsB x kGsB (the last one
// Q - kGsB (nb - 1) wide), nb = ceil(Q / kGsB).
constexpr int kGsB = 32;

// Entries (8 bytes each) of shared memory the blocked solves use: the
// inverted diagonal blocks of L (block b at b kGsB (kGsB + 1), column j of it
// at + j (kGsB + 1); the last block only as wide as it is), then one buffer of
// Q + kGsB per solving warp.
__host__ __device__ constexpr int gram_solve_scratch(int Q, int warps) {
  return ((Q - 1) / kGsB) * kGsB * (kGsB + 1) + (Q - (Q - 1) / kGsB * kGsB) * (kGsB + 1) + warps * (Q + kGsB);
}

// Device buffers of the optimal distribution (sized for the largest J_n).
struct OptBuffers {
  double *a, *bsum, *total, *q, *pf;
  unsigned long long *cdf, *btot;
  int *idx, *dims;
};

// Buffers and layout of the whole-GPU path (grid.cu) for one problem.
// Operand pieces are BF16, K-major, zero-padded: G_n [Ip][ldg], Z [Jp][ldz],
// Z^T [QTp][ldzt], weighted residual E [Ip][lde]; gpart holds the FP32
// partial gradients of the split samples.  Each piece buffer has a TMA tensor
// map (boxes of 64 K-elements, 128-byte swizzle); Z^T's box height depends on
// the mode, so it has one map per mode.
struct GridPath {
  // scaled variant, H = F: a second stream on which the Gram factorisation
  // (one cluster of 16 SMs) runs beside the residual and gradient GEMMs
  cudaStream_t s2;
  cudaEvent_t ev_fork, ev_join;
  int np;                  // BF16 pieces per operand of the residual and gradient GEMMs (1 or 3)
  int npz;                 // pieces of Z kept (3 for the scaled variant: its Gram is formed from three)
  int scaled;              // scaled variant (Sec. 3.3)
  int JH;                  // |H| of an independent Hessian batch (0: H = F)
  int nt_res;              // N tile of the residual GEMM
  int Jp, Ip, Qp, QTp;     // padded J (256; the larger of |F| and |H|), I (128), Q (64)
  long long ldg, ldz, ldzt, lde;
  int max_splits;
  int sms;                 // SMs of the device (split-K sizing)
  size_t gpart_elems, hpart_elems;
  int x_bf16;              // mode-major copies of X in BF16 (else FP32)
  float w;                 // uniform sampling: every weight 1/|F|
  __nv_bfloat16 *Gp[3], *Zp[3], *ZTp[3], *Ep[3];
  float *gpart;            // [splits][I_n][Q] partial gradients
  float *hpart;            // [splits][Q][Q] partial Grams (scaled)
  float *Lfac;             // blocks of the Gram factor (scaled)
  int *fac_ok;             // 1 when the last factorisation succeeded
  long long *col;
  CUtensorMap tmG[3], tmZ[3], tmE[3];
  CUtensorMap tmZT[8][3];  // Z^T as the B operand (box height of mode n's N tile)
  CUtensorMap tmZTa[3];    // Z^T as the A operand of the Gram (box height 128)
  CUtensorMap tmZc;        // Z (first piece) in boxes of 64 samples (fused BF16 kernel)
  int fz_S[8];             // cluster size of the fused BF16 kernel per mode (0: not used)
};

// Fused BF16 iteration body (grid_fused.cu): cluster size for a mode (0: not
// applicable), set-up and launch.
int grid_fused_cluster(int In, int Q, int J);
int grid_step_kernels(const GridPath &g, const ProbDesc &D, int n);
cudaError_t grid_fused_prepare();
cudaError_t launch_grid_fused(const CUtensorMap &tmZ, const CUtensorMap &tmG, float *gpart, const ProbDesc &D,
                              int n, const long long *col, float w, int S, int rec, cudaStream_t st);

// Largest R_n R_{n+1} of the scaled variant on the whole-GPU path.
constexpr int kGridScaledMaxQ = 512;

// Arguments of the scaled variant's factorisation and direction (grid_scaled.cu).
struct GridScaledArgs {
  const float *hpart;      // partial Grams [hsplits][Q][Q]
  long long hstride;
  int hsplits;
  const float *gpart;      // partial gradients [gsplits][In][Q]
  long long gstride;
  int gsplits;
  int In, Q;
  int sms;                 // SMs of the device (rows of the direction spread over them)
  double hscale;           // 1 / |H|
  double damping;
  float *Lfac;
  int *ok;
  int rule;
  float alpha, eta, b;
  double eps;
  float *G, *acc;
  float *dbg_g, *dbg_p;
  double *dbg_h;
  int *status;
};
size_t grid_scaled_factor_floats(int Q);
cudaError_t grid_scaled_prepare();
cudaError_t launch_grid_scaled(const GridScaledArgs &s, cudaStream_t st);
cudaError_t launch_grid_factor(const GridScaledArgs &s, cudaStream_t st);
cudaError_t launch_grid_direction(const GridScaledArgs &s, cudaStream_t st);

// kernel launchers (defined in the .cu files)
void grid_layout(const int *I, const int *R, int N, int J, int np, int scaled, int JH, GridPath &g);
cudaError_t grid_tensor_maps(const int *R, int N, GridPath &g);
int grid_nt_max(int np);
int grid_ntiles(int Q, int np, int &NT);
cudaError_t grid_prepare_gemm();
cudaError_t launch_grid_step(const GridPath &g, const ProbDesc &D, int n, long long t, int rec, cudaStream_t s);
// Split-K unit of mode n (samples per partial, a multiple of 256) and the
// number of partials a sample range [j0, j1) produces.
long long grid_split_unit(const GridPath &g, const ProbDesc &D, int n, long long nsamples);
long long grid_gram_unit(const GridPath &g, const ProbDesc &D, int n, long long nsamples);
// The two halves of an iteration: the partial gradient (and partial Gram)
// over the sample ranges [j0, j1) of F and [h0, h1) of H, written as one
// FP32 partial per split unit; then the fixed-order sum of gsplits (hsplits)
// partials, the direction, the step rule and the update of G_n.
cudaError_t launch_grid_partial(const GridPath &g, const ProbDesc &D, int n, long long t, long long j0,
                                long long j1, long long h0, long long h1, int rec, float *gout, float *hout,
                                cudaStream_t s, const GridScaledArgs *fork_factor);
cudaError_t launch_grid_apply(const GridPath &g, const ProbDesc &D, int n, const float *gparts, int gsplits,
                              const float *hparts, int hsplits, int rec, cudaStream_t s);
cudaError_t launch_optimal_sampling(int core_dtype, int x_dtype, int N, int n, const int *I, const int *R,
                                    const void *const *cores, const void *xmode, long long ldx,
                                    unsigned long long seed, long long t, int J, OptBuffers &b, cudaStream_t s);
cudaError_t launch_step(int core_dtype, int x_dtype, int rmax, const ProbDesc *descs, int nprob,
                        const StepLayout &lay, int threads, long long t0, int nsteps,
                        const long long *t_dev, cudaStream_t s);
cudaError_t launch_advance_counter(long long *t, long long T, int set, cudaStream_t s);
cudaError_t step_kernel_prepare(int core_dtype, int x_dtype, int rmax, const StepLayout &lay);
int step_max_smem();
// instantiated per (core type, fiber type, BF16 pieces) in step_<variant>.cu, with
// the scaled variant compiled in (SC, step_<variant>_scaled.cu) or out
template <typename T, typename XT, int RMAX, int NPC, bool SC>
cudaError_t step_prepare_t(const StepLayout &lay);
template <typename T, typename XT, int RMAX, int NPC, bool SC>
cudaError_t step_launch_t(const ProbDesc *descs, int nprob, const StepLayout &lay, int threads, long long t0,
                          int nsteps, const long long *t_dev, cudaStream_t s);

// Full-gradient iterations (gd.cu): one problem's shape, cores and mode-major copies.
struct GdArgs {
  int N;
  int I[8], R[8];
  long long J[8];          // J_n = prod_{k != n} I_k
  void *cores[8];          // G_{k(2)}, core dtype
  const void *xmode[8];    // mode-major copies of X (core dtype)
  long long ldx[8];
};
struct GdBuffers {
  void *Z = nullptr;               // J_n x Q subchain matrix (largest mode)
  void *part = nullptr;            // max_chunks x max(I_n, Q) x Q column-chunk partials
  void *M[8] = {};         // M_n = X_[n] Z, I_n x Q
  double *Gam[8] = {};     // Gamma_n = Z^T Z, Q x Q
  double *fac = nullptr;           // FP64 Cholesky factor of Gamma_n + damping I
  int max_chunks = 608;
};
cudaError_t gd_prepare();
cudaError_t launch_gd_iteration(int core_dtype, const GdArgs &a, int scaled, double alpha, double damping,
                                GdBuffers &b, int *status, cudaStream_t s);

cudaError_t launch_mode_copy(int src_dtype, int dst_dtype, const void *X, void *out, long long A,
                             long long In, long long B, long long ld, cudaStream_t s);
cudaError_t launch_euclid_table(int core_dtype, const void *G, int I, int Q, double *snorm,
                                double *prob, unsigned long long *cdf, cudaStream_t s);
cudaError_t launch_leverage_table(int core_dtype, const void *G, int I, int Q, double *prob,
                                  unsigned long long *cdf, int *status, cudaStream_t s);
// sums (nullable) receives sum (x - x_ref)^2 and sum x_ref^2, reduced in a
// fixed order through `partials` (reconstruct_partials(...) doubles).
cudaError_t launch_reconstruct(int dtype, int N, const int *I, const int *R,
                               const void *const *cores, void *X, const void *Xref,
                               double *sums, double *partials, cudaStream_t s);
long long reconstruct_partials(int dtype, int N, const int *I, const int *R);
cudaError_t launch_sampled_loss_grad(int N, const int *I, const int *R, int n, int J,
                                     const int *idx, const float *XS, const float *w,
                                     const float *const *cores, float *const *grads,
                                     float *loss, cudaStream_t s);

}  // namespace trsgd
