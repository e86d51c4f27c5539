/*
 * trsgd.h - C-ABI of the GB300 (sm_103a) block-randomized stochastic tensor
 * ring solver: TR-BRSGD and TR-ScaledBRSGD of Yu, Li and Zhou, "Block-
 * Randomized Stochastic Methods for Tensor Ring Decomposition"
 * (arXiv 2303.16492).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Indices are 0-based (the paper is 1-based).
 * - A tensor X of order N and dims I[0..N-1] is a dense device buffer with
 *   i_1 fastest (Definition of the multi-index, Sec. 2): X(i_1..i_N) sits at
 *   offset i_1 + i_2 I_1 + i_3 I_1 I_2 + ...
 * - Core n (ranks R_n x I_n x R_{n+1}, R_{N+1} = R_1) is stored as its
 *   classical mode-2 unfolding G_{n(2)} (Sec. 2): a row-major I_n x
 *   (R_n R_{n+1}) matrix whose row i is the lateral slice G_n(i) stored
 *   column-major, so G_n(r, i, r') sits at i*R_n*R_{n+1} + r + r'*R_n.  A torch
 *   tensor of shape (I_n, R_{n+1}, R_n) views it directly.
 * - Every pointer named *_dev is device memory owned by the caller unless
 *   stated otherwise; host pointers are named *_host.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Compute entry points only enqueue work on it and return; the
 *   ones documented as synchronising wait for it.
 * - The status code is the only error channel.  Argument checks happen
 *   before any CUDA call, so an invalid argument returns TRSGD_EINVAL without
 *   touching the device.  Errors found on the device (a bounded wait that ran
 *   out, a non-finite step, a failed factorisation) are latched in a device
 *   status word and returned by the next synchronising call on the handle.
 * - A handle is not thread-safe; independent handles on different streams
 *   are.
 */
#ifndef TRSGD_H
#define TRSGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRSGD_MAX_ORDER 8

typedef enum {
  TRSGD_OK = 0,
  TRSGD_EINVAL = 1,       /* invalid argument or configuration            */
  TRSGD_ENOMEM = 2,       /* device or host allocation failed             */
  TRSGD_ECUDA = 3,        /* a CUDA runtime call failed                   */
  TRSGD_ENUMERIC = 4,     /* non-finite step or non-SPD preconditioner    */
  TRSGD_ETIMEOUT = 5,     /* a bounded device wait ran out                */
  TRSGD_EUNSUPPORTED = 6, /* valid, but outside what this build supports  */
  TRSGD_EBADINDEX = 7     /* debug build: a drawn slice index or a fiber
                             column outside its range (replaced by 0)     */
} trsgd_status;

/* Mini-batch distributions of Sec. 3.2: uniform, leverage-based (Lemma
 * lev_est), Euclidean-based (Lemma euc_est) and optimal (Theorem variance,
 * Eq. optimal_prob). */
typedef enum {
  TRSGD_DIST_UNIFORM = 0,
  TRSGD_DIST_LEVERAGE = 1,
  TRSGD_DIST_EUCLIDEAN = 2,
  TRSGD_DIST_OPTIMAL = 3
} trsgd_dist;

/* Search direction: p = -g (Algorithm 3, TR-BRSGD) or p = -g h^{-1}
 * (Eq. scaledsg_direction, TR-ScaledBRSGD). */
typedef enum { TRSGD_PLAIN = 0, TRSGD_SCALED = 1 } trsgd_variant;

/* Step rule: fixed alpha (Eq. update_brsgd) or AdaGrad (Remark after
 * Algorithm 3). */
typedef enum { TRSGD_STEP_FIXED = 0, TRSGD_STEP_ADAGRAD = 1 } trsgd_steprule;

/* Arithmetic of the step.  FP64: cores, X and all arithmetic in double.
 * FP32: cores and X in float, FP32 arithmetic (the two contractions: see
 * trsgd_fp32_units).  BF16_MIXED: cores in float,
 * the sampled fibers stored in bfloat16, tensor-core contractions with FP32
 * accumulation.  The scaled variant's Gram matrix is reduced, factorised and
 * applied in FP64 for FP64 cores and in double-float arithmetic (a float
 * pair, about 48 significant bits, on the FP32 pipes) for float cores; the
 * relative-error reduction is FP64 in every mode. */
typedef enum { TRSGD_FP64 = 0, TRSGD_FP32 = 1, TRSGD_BF16_MIXED = 2 } trsgd_prec;

typedef enum { TRSGD_DTYPE_F64 = 0, TRSGD_DTYPE_F32 = 1, TRSGD_DTYPE_BF16 = 2 } trsgd_dtype;

/* Execution path of an iteration.
 * CLUSTER: one fused persistent kernel, one thread-block cluster (<= 16 SMs)
 *   per problem, everything on chip (R_n <= 16, R_n R_{n+1} <= 256, scaled
 *   variant R_n R_{n+1} <= 128); batched problems, every distribution.
 * GRID: a short sequence of kernels over the whole GPU per iteration, the
 *   residual and gradient contractions on the tensor cores (tcgen05, BF16
 *   operands; FP32 as three BF16 pieces per operand); one problem, uniform
 *   sampling, plain and scaled variants, FP32 / BF16-mixed, R_n <= 32,
 *   R_n R_{n+1} <= 512.  The scaled variant's Gram matrix is formed on the
 *   tensor cores from three BF16 pieces of Z (FP32 accuracy in either
 *   mode), then factored and applied in double-float arithmetic.
 * AUTO: CLUSTER when the problem fits it, else GRID. */
typedef enum { TRSGD_PATH_AUTO = 0, TRSGD_PATH_CLUSTER = 1, TRSGD_PATH_GRID = 2 } trsgd_path;

/* Units of the FP32 mode's two contractions, the residual G_n Z^T and the
 * gradient (E D) Z of Eq. S_gradient.
 * PIECES: the tensor cores (tcgen05, FP32 accumulation in tensor memory),
 *   every operand held as three BF16 pieces that sum to its FP32 value (each
 *   piece the rounding of what the previous ones left) and the six piece
 *   products of total order <= 2 accumulated: a dropped product is below
 *   2^-23 of the term, about one FP32 rounding.  The cluster path takes it
 *   when its shared-memory layout holds the pieces (R_n R_{n+1} and the
 *   samples per CTA <= 256, one chunk of 128 rows of G_n at a time), else
 *   the FMA units.  The grid path always uses it.
 * FMA: the FP32 FMA units only (cluster path; the grid path is then not
 *   taken, TRSGD_EUNSUPPORTED if requested).
 * The other modes ignore the field (FP64: FMA units; BF16_MIXED: two pieces
 * for the residual, one for the gradient) but it must hold one of the two
 * values. */
typedef enum { TRSGD_FP32_PIECES = 0, TRSGD_FP32_FMA = 1 } trsgd_fp32_units;

/* One TR problem (Algorithm 3's arguments plus the stopping-free part of the
 * configuration). */
typedef struct {
  int32_t N;                       /* tensor order, 2..TRSGD_MAX_ORDER       */
  int32_t dist;                    /* trsgd_dist                             */
  int64_t I[TRSGD_MAX_ORDER];      /* dims I_1..I_N                          */
  int64_t R[TRSGD_MAX_ORDER];      /* TR ranks R_1..R_N (R_{N+1} = R_1)      */
  int64_t J;                       /* |F_n|, samples per step (>= 1)         */
  int64_t J_H;                     /* |H_n| for the scaled variant; 0: H = F */
  int32_t variant;                 /* trsgd_variant                          */
  int32_t rule;                    /* trsgd_steprule                         */
  int32_t prec;                    /* trsgd_prec                             */
  int32_t x_dtype;                 /* trsgd_dtype of the caller's X          */
  double alpha;                    /* fixed step alpha                       */
  double eta, b, eps;              /* AdaGrad eta, b, epsilon                */
  double damping;                  /* eta^t of the damped preconditioner     */
  uint64_t seed;                   /* Philox key of this problem             */
  int32_t path;                    /* trsgd_path                             */
  int32_t fp32_units;              /* trsgd_fp32_units, FP32 mode            */
} trsgd_config;

typedef struct trsgd_handle trsgd_handle;

/* Create a solver for `nproblems` independent TR problems stepped together
 * (nproblems > 1 is the batched mode: one thread-block cluster per problem in
 * one persistent launch).
 *   cfg        host array [nproblems] of configurations.
 *   X_dev      host array [nproblems] of device pointers to each X (dtype
 *              cfg.x_dtype, i_1 fastest).  Read during init only: the
 *              library keeps its own mode-major copies (one per mode, rows =
 *              mode-n fibers, padded to 16 bytes).
 *   cores_dev  host array of device pointers, problem p's N_p cores
 *              consecutively (problem 0 first); G_{n(2)} layout, dtype
 *              double for TRSGD_FP64 and float otherwise.  Borrowed for the
 *              handle's lifetime and updated in place by every step.  For
 *              float cores of plain problems the library also keeps each
 *              core as BF16 operand pieces (three: 6 bytes per entry, rows
 *              padded to 128 and columns to 16); every step launch rebuilds
 *              them from the cores first, so the caller may change the cores
 *              between calls.
 *   stream     the stream every later call of this handle enqueues on.
 *   out        receives the handle.
 * Synchronising (it builds the mode-major copies and distribution tables).
 * Returns EINVAL for a malformed configuration, EUNSUPPORTED for a valid one
 * this build does not run, ENOMEM/ECUDA on device failures. */
trsgd_status trsgd_init(const trsgd_config *cfg, int32_t nproblems,
                        const void *const *X_dev, void *const *cores_dev,
                        void *stream, trsgd_handle **out);

/* One iteration (Algorithm 3: mode draw, Algorithm 2 sampling, Eq. S_gradient,
 * optional Eq. scaledsg_direction, step rule, update of G_n) of every problem
 * at iteration counter t (the Philox counter; iterations are a pure function
 * of (seed, t) and the current cores).  Enqueued on the handle's stream;
 * does not synchronise. */
trsgd_status trsgd_step(trsgd_handle *h, int64_t t);

/* Iterations t0 .. t0+T-1 (T >= 0) as persistent launches of `chunk` steps
 * each (chunk <= 0: all T in one launch).  With tol > 0 or max_seconds > 0
 * it synchronises every `chunk` steps, evaluates the RSE of problem 0
 * against Xref_dev (NULL: the X given to init) and stops once RSE <= tol or
 * the elapsed device time exceeds max_seconds (Sec. 4 stopping criteria).
 * *steps_done and *rse_out (nullable) receive the iterations run and the
 * last RSE (-1 if none).  Synchronising. */
trsgd_status trsgd_run(trsgd_handle *h, int64_t t0, int64_t T, int64_t chunk,
                       double tol, double max_seconds, const void *Xref_dev,
                       int64_t *steps_done, double *rse_out);

/* Iterations c .. c+T-1 (1 <= T <= 2^20; T = 0 does nothing), where c is a
 * device-resident iteration counter of the handle (0 after init), followed
 * by c += T on the device.  No host-side iteration number is involved, so
 * the call can be recorded in a CUDA graph (stream capture of the handle's
 * stream) and each replay continues the sequence where the last one ended;
 * the iterates are bit-identical to trsgd_run from the same t.  Enqueued on
 * the handle's stream; does not synchronise.  TRSGD_EUNSUPPORTED for the
 * optimal distribution (its tables are built for a mode drawn on the host).
 * trsgd_set_counter enqueues c = t (also capturable).  The whole-GPU path
 * (TRSGD_PATH_GRID) draws the mode on the host and returns EUNSUPPORTED. */
trsgd_status trsgd_step_counter(trsgd_handle *h, int64_t T);
trsgd_status trsgd_set_counter(trsgd_handle *h, int64_t t);

/* RSE = ||TR(G) - X_ref||_F / ||X_ref||_F (Sec. 4) of problem `problem`,
 * reduced in FP64.  Xref_dev: a tensor of the problem's dims in the cores'
 * dtype (double for TRSGD_FP64, float otherwise), or NULL for the X given to
 * init when that X has the cores' dtype (TRSGD_EUNSUPPORTED for a BF16 X).
 * Synchronising; *out receives the value. */
trsgd_status trsgd_rel_error(trsgd_handle *h, int32_t problem,
                             const void *Xref_dev, double *out);

/* Relative error without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc or
 * cudaFree, for example code whose device memory is owned entirely by another
 * allocator (a framework's caching pool or a fixed per-process budget), or a
 * latency-sensitive caller that cannot accept the implicit device
 * synchronisation an allocation or free may cause.  It needs no handle.
 *   Same result as trsgd_rel_error: RSE = ||TR(G) - X_ref||_F / ||X_ref||_F,
 *   reduced in FP64 in a fixed order.  N, I, R, dtype (F64 or F32,
 *   for the cores and X_ref) and cores_dev as in trsgd_reconstruct; Xref_dev
 *   a tensor of dims I (i_1 fastest); out_dev receives one double on the
 *   device.  Enqueued on `stream`, no synchronisation.
 * Scratch: one pair of FP64 partial sums per tile of 64 columns of X_[1],
 *   held in a fixed array inside the library (1 MiB on every GPU that loads
 *   the library, kept until the process exits).  Sizes beyond it, i.e.
 *   prod_{k>1} I_k > 4,194,304, return TRSGD_EINVAL; ranks above 16, or
 *   R_1 R_2 too large for the tiles' shared memory, return
 *   TRSGD_EUNSUPPORTED; a failed launch returns TRSGD_ECUDA.  Every call
 *   overwrites the entries it uses, so nothing
 *   needs clearing, but all calls share the array: calls that can overlap on
 *   the GPU (different streams without ordering between them) race and must
 *   be serialised by the caller.
 * The first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) invalidates the kept address: do not call this entry
 * point after one.  No cudaMalloc, cudaFree or allocating library routine is
 * called. */
trsgd_status trsgd_rel_error_static(int32_t N, const int64_t *I, const int64_t *R, int32_t dtype,
                                    const void *const *cores_dev, const void *Xref_dev,
                                    double *out_dev, void *stream);

/* Full reconstruction X = TR({G_n}) (element formula of the Introduction,
 * evaluated as X_[1] = G_{1(2)} (G^{!=1}_{[2]})^T).  dtype applies to the
 * cores and to X; X_dev receives prod(I) elements, i_1 fastest.  Enqueued on
 * `stream`. */
trsgd_status trsgd_reconstruct(int32_t N, const int64_t *I, const int64_t *R,
                               int32_t dtype, const void *const *cores_dev,
                               void *X_dev, void *stream);

/* Sampled TR loss and its adjoint for every core (FP32):
 *   L = 1/2 sum_j w_j || X_S(:, j) - G_{n(2)} Z(j, :)^T ||^2,
 * Z = G^{!=n}_{[2]}(F, :) built from idx (Algorithm 2), X_S given.
 *   idx_dev  int32 [J][N] slice indices (entry n ignored).
 *   XS_dev   float [J][I_n], fiber j contiguous.
 *   w_dev    float [J] sample weights.
 *   grads_dev (nullable) host array [N] of device pointers receiving dL/dG_k
 *            in the G_{k(2)} layout (overwritten); NULL: loss only.
 *   loss_dev float [1] receives L.
 * The adjoint of core k != n is accumulated per sample from prefix and
 * suffix slice products of the chain (product rule on the trace).  The
 * per-sample terms go to a stream-ordered scratch (cudaMallocAsync, freed
 * on the stream) and are added in increasing j: the results are
 * bit-reproducible. */
trsgd_status trsgd_sampled_loss_grad(int32_t N, const int64_t *I, const int64_t *R,
                                     int32_t n, int64_t J, const int32_t *idx_dev,
                                     const float *XS_dev, const float *w_dev,
                                     const float *const *cores_dev,
                                     float *const *grads_dev, float *loss_dev,
                                     void *stream);

/* Record the intermediates of every following step of problem 0 (mode n,
 * idx, p_F, Z, E, g, direction p, preconditioner h) for readback with
 * trsgd_get_debug.  on = 0 stops recording. */
trsgd_status trsgd_set_debug(trsgd_handle *h, int32_t on);

/* Failure-path testing of the fused kernel: the number of polls of every
 * bounded mbarrier wait (tensor-core completion, bulk fiber copies) before it
 * latches TRSGD_ETIMEOUT.  A timed-out wait is followed by a second wait of
 * the default length that drains the outstanding operation, and the launch
 * runs to its end (its CTAs leave together); the host reads TRSGD_ETIMEOUT
 * at the next synchronising call.  polls = 0 restores the default (2^22);
 * a negative value makes every first try time out.  Applies to every problem
 * of the handle.  Synchronising. */
trsgd_status trsgd_set_wait_limit(trsgd_handle *h, int64_t polls);

/* Index checks of the debug build (the library compiled with -DTRSGD_DEBUG,
 * _lib/libtrsgd_debug.so): every drawn slice index i_k (Algorithm 2) is
 * checked against [0, I_k) and every fiber column of X_[n] against
 * [0, prod_{k != n} I_k) before anything is read with it; a violation
 * latches TRSGD_EBADINDEX in the device status word (read by the next
 * synchronising call) and the index is replaced by 0, so no access leaves
 * its buffer and nothing traps.  This call replaces the upper bound of the
 * check on core k's indices by `bound` (1 <= bound <= I_k; 0 restores I_k)
 * for every problem of the handle, so that the reporting path can be
 * exercised with indices that are valid for the memory they address; the
 * draws themselves do not change.  Synchronising.  TRSGD_EINVAL for a null
 * handle, k outside [0, N) or bound outside [0, I_k]; TRSGD_EUNSUPPORTED in
 * the product build, which has no checks compiled in. */
trsgd_status trsgd_debug_index_bound(trsgd_handle *h, int32_t k, int64_t bound);

typedef enum {
  TRSGD_DBG_MODE = 0,   /* int32 [1]                                   */
  TRSGD_DBG_IDX = 1,    /* int32 [J][N], entry n = -1                  */
  TRSGD_DBG_PF = 2,     /* double [J]                                  */
  TRSGD_DBG_Z = 3,      /* core dtype [J][R_n R_{n+1}]                 */
  TRSGD_DBG_E = 4,      /* core dtype [J][I_n]  (E = G Z^T - X_S)^T    */
  TRSGD_DBG_G = 5,      /* core dtype [I_n][R_n R_{n+1}]  g            */
  TRSGD_DBG_P = 6,      /* core dtype [I_n][R_n R_{n+1}]  direction p  */
  TRSGD_DBG_H = 7       /* double [Q][Q] damped preconditioner h       */
} trsgd_debug_item;

/* Copy one recorded intermediate of the last recorded step into host memory
 * (at most `bytes`; *written receives the bytes copied).  Synchronising. */
trsgd_status trsgd_get_debug(trsgd_handle *h, int32_t item, void *out_host,
                             size_t bytes, size_t *written);

/* AdaGrad state of problem p, core k (sum of squared directions, core dtype,
 * G_{k(2)} layout): copy out (dir = 0) or in (dir = 1), for checkpointing.
 * Synchronising. */
trsgd_status trsgd_adagrad_state(trsgd_handle *h, int32_t problem, int32_t core,
                                 void *host, size_t bytes, int32_t dir);

/* Launch shape picked for the step kernel: cluster size (CTAs per problem)
 * and threads per CTA.  set: 0 = query into *cluster / *threads, 1 = force
 * these values (validated; 0 keeps the current one).  trsgd_autotune times
 * the candidate shapes on scratch copies of the cores and keeps the fastest
 * (synchronising; the cores are left unchanged).  On the whole-GPU path the
 * query returns cluster 0 and threads 256, setting returns EUNSUPPORTED and
 * trsgd_autotune does nothing. */
trsgd_status trsgd_launch_shape(trsgd_handle *h, int32_t set, int32_t *cluster,
                                int32_t *threads);
trsgd_status trsgd_autotune(trsgd_handle *h, int32_t steps_per_trial);

/* Sample-sharded iteration: data parallelism over the samples of
 * Eq. S_gradient (and of Eq. S_hessian for the scaled variant), whose
 * estimators are sums over samples.  Every rank holds the same X and the
 * same cores, draws the same mode and the same Philox counters for
 * iteration t, and takes a disjoint range of the |F| (and |H|) samples; the
 * ranks exchange their FP32 partial sums once per iteration and all apply the
 * same update.  Whole-GPU path only (TRSGD_EUNSUPPORTED otherwise).
 *
 * The samples of a batch fall into split units (a multiple of 256 samples,
 * fixed by the problem and the device); one partial is one unit's sum
 * (gelems = I_n R_n R_{n+1} floats for the gradient, helems =
 * (R_n R_{n+1})^2 for the Gram; a Gram unit is the gradient's unit over a
 * power of two, so a rank's gradient units hold whole Gram units).  trsgd_shard_plan deals the units of
 * iteration t to `world` ranks in contiguous runs (rank r gets units
 * [r U / world, (r+1) U / world) of U); a rank may get none.
 *   trsgd_shard_plan    host-only; fills *out for rank `rank` of `world`.
 *   trsgd_step_partial  writes this rank's partials, then zeros up to
 *                       gsplits_max (hsplits_max) partials, into gpart_dev
 *                       (hpart_dev, scaled only; else may be NULL).  Async.
 *   trsgd_step_apply    sums gsplits partials of gparts_dev (and hsplits of
 *                       hparts_dev) in increasing index, then the direction,
 *                       step rule and update of G_n.  Pass the ranks'
 *                       buffers gathered in rank order (an all-gather): the
 *                       zero padding leaves every sum unchanged, so the
 *                       result is bit-identical for every world size (and to
 *                       trsgd_step(t) on one device, except where that runs
 *                       the fused BF16 kernel, whose sums take another
 *                       order), and identical on every rank.  Async.
 * The buffers are caller device memory of gsplits_max * gelems (per rank) or
 * world * gsplits_max * gelems (gathered) floats. */
typedef struct {
  int32_t mode;                     /* n of iteration t                        */
  int64_t j0, j1;                   /* this rank's samples of F                */
  int64_t h0, h1;                   /* this rank's samples of H (J_H > 0)      */
  int64_t gunit, hunit;             /* samples per gradient / Gram partial     */
  int64_t gsplits, hsplits;         /* partials this rank computes             */
  int64_t gsplits_max, hsplits_max; /* the largest count over the ranks        */
  int64_t gelems, helems;           /* floats per partial                      */
} trsgd_shard;

trsgd_status trsgd_shard_plan(trsgd_handle *h, int64_t t, int32_t rank, int32_t world, trsgd_shard *out);
trsgd_status trsgd_step_partial(trsgd_handle *h, int64_t t, const trsgd_shard *plan, float *gpart_dev,
                                float *hpart_dev);
trsgd_status trsgd_step_apply(trsgd_handle *h, int64_t t, const float *gparts_dev, int64_t gsplits,
                              const float *hparts_dev, int64_t hsplits);

/* Number of iteration kernels enqueued by this handle so far (the fused
 * kernel counts once per launch of any number of iterations; the whole-GPU
 * path launches per iteration: G_n's pieces, the samples, one transpose per
 * kept piece of Z, the residual, the gradient and the update; the scaled
 * variant replaces the update by the Gram, its factorisation and the
 * direction, plus the H batch's samples and transposes when J_H > 0; BF16
 * operands with the plain direction and R_n R_{n+1} <= 448: G_n's pieces,
 * the samples and one fused kernel). */
int64_t trsgd_launch_count(const trsgd_handle *h);

/* One iteration of the full-gradient methods the paper compares against
 * (Sec. 3), on problem 0 of the handle, every core from the same iterate:
 *   grad_n = G_{n(2)} Gamma_n - M_n,  Gamma_n = Z^T Z,  M_n = X_[n] Z,
 *   Z = G^{!=n}_{[2]} (Eq. gradient);
 *   scaled = 0 (TR-GD):       G_{n(2)} <- G_{n(2)} - alpha grad_n;
 *   scaled = 1 (TR-ScaledGD): G_{n(2)} <- G_{n(2)} - alpha grad_n
 *                             (Gamma_n + damping I)^{-1} (Eq. scaled_gd).
 * Z is formed in full (J_n x R_n R_{n+1}, device scratch allocated at the
 * first call), M_n and Gamma_n by passes over Z and the mode-major copy of X
 * with fixed-order sums (deterministic), the factor of Gamma_n + damping I in
 * FP64 (the damping grows on failure as for the scaled step, then
 * TRSGD_ENUMERIC).  FP64 and FP32 problems with uniform sampling, R_n <= 16,
 * scaled R_n R_{n+1} <= 128; else TRSGD_EUNSUPPORTED; alpha, damping finite,
 * damping >= 0, scaled 0 or 1, else TRSGD_EINVAL.  Asynchronous on the
 * handle's stream; device errors are latched as for trsgd_step. */
trsgd_status trsgd_gd_step(trsgd_handle *h, int32_t scaled, double alpha, double damping);

/* BF16 pieces per tensor-core operand of the residual and gradient
 * contractions in the handle's current launch shape: 0 = the FMA units (FP64;
 * FP32 with TRSGD_FP32_FMA or where the pieces do not fit the cluster's shared
 * memory), 3 = FP32 on pieces (either path), 2 = the cluster path's
 * BF16-mixed mode, 1 = the whole-GPU path's BF16-mixed mode.  -1 for a null
 * handle.  Pure host query. */
int32_t trsgd_tensor_pieces(const trsgd_handle *h);

/* Measured arithmetic peak of one unit of the current device, for the
 * roofline fractions of kernels that run on it.  The paper has no
 * counterpart.  unit 0: FP32 fused multiply-add, 1: FP64 fused multiply-add.
 * A warm-up launch, then a timed launch (CUDA events on `stream`) of 8
 * independent FMA chains per thread, 8 CTAs of 256 threads per SM, `iters`
 * rounds of 16 FMAs per chain; *flops_per_s receives 2 flop per FMA over the
 * timed launch.  Synchronising. */
trsgd_status trsgd_probe_peak(int32_t unit, int64_t iters, void *stream, double *flops_per_s);

void trsgd_destroy(trsgd_handle *h);
const char *trsgd_status_string(trsgd_status s);

#ifdef __cplusplus
}
#endif
#endif /* TRSGD_H */
