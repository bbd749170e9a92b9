/*
 * spamm.h -- C ABI of the GB300 (sm_103a) norm-pruned block SpAMM library.
 *
 * Method: arXiv 2103.13042, "Accelerating Sparse Approximate Matrix
 * Multiplication on GPUs".  For square N x N FP32 matrices A, B, a leaf size
 * b and a threshold tau >= 0 it computes (Section 2.1 problem statement,
 * alpha = 1, beta = 0)
 *
 *     C[i,j] = sum over k with ||A[i,k]||_F * ||B[k,j]||_F >= tau of A[i,k] B[k,j]
 *
 * where X[i,k] is the b x b leaf block starting at row i*b, column k*b
 * (Section 3 notation; matrices are zero padded to a multiple of b), and the
 * norms are the Frobenius norms of Eq. 2.  The flat leaf-level test is the
 * GPU re-design of Section 3.1, equivalent to the recursive test of
 * Algorithm 1.  A block product is skipped iff its norm product is < tau:
 * a tie is multiplied and a NaN product is never skipped.
 *
 * Conventions for every entry point:
 *  - Matrices are FP32, row-major, leading dimension n, in DEVICE memory
 *    owned by the caller.  A, B and C must not alias.  Every pointer must be
 *    16-byte aligned (SPAMM_ERR_INVALID_ARG otherwise).
 *  - bd = ceil(n / leaf).  Norm maps are FP64 bd x bd row-major device arrays.
 *  - leaf is 32, 64 or 128 (SPAMM_ERR_UNSUPPORTED otherwise); n >= 1.
 *  - tau must be >= 0 and not NaN; +infinity skips every finite product.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *    calls are asynchronous on it unless stated; errors found on the host are
 *    returned before anything is enqueued; launch failures return
 *    SPAMM_ERR_CUDA.  Device-side checks (bounds, bounded waits) latch a code
 *    in a device status word that spamm_last_device_status reads.
 *  - Nothing aborts or throws.  The library never reads host memory that the
 *    caller did not pass.
 */
#ifndef SPAMM_H
#define SPAMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPAMM_OK = 0,
  SPAMM_ERR_INVALID_ARG = 1,   /* bad size, NaN/negative tau, NULL or misaligned pointer */
  SPAMM_ERR_UNSUPPORTED = 2,   /* leaf or precision not implemented for this shape */
  SPAMM_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  SPAMM_ERR_NO_MEMORY = 4,     /* workspace too small or device allocation failed */
  SPAMM_ERR_TIMEOUT = 5,       /* a bounded device wait ran out (status word) */
  SPAMM_ERR_DEVICE_FAULT = 6   /* a device-side bounds check failed (status word) */
} spamm_status_t;

/* Arithmetic of the block products (Section 3.3 multiplies in FP32 on SIMT
 * and in FP16 on tensor cores; the others extend that):
 *  FP32        FP32 operands, FP32 FMA accumulation on the SIMT cores.
 *  TF32X3      tensor cores, each operand split hi + lo in TF32, three
 *              products hi*hi + hi*lo + lo*hi, FP32 accumulation.
 *  BF16, FP16  tensor cores; every leaf block scaled by a power of two
 *              2^-e (e = frexp exponent of its max |entry|) and rounded to
 *              nearest-even; FP32 accumulation; the product is rescaled by
 *              2^(ea + eb).
 *  *_SPLIT     as BF16/FP16, plus the lo parts on the dominant triples
 *              (see spamm_plan's target_rel_err). */
typedef enum {
  SPAMM_FP32 = 0,
  SPAMM_TF32X3 = 1,
  SPAMM_BF16 = 2,
  SPAMM_FP16 = 3,
  SPAMM_BF16_SPLIT = 4,
  SPAMM_FP16_SPLIT = 5
} spamm_precision_t;

/* Plan statistics (Section 3.5.1 valid multiplications, Section 3.5.2 valid
 * ratio, and the skipped-product bounds):
 *   survivors      S, number of multiplied leaf triples
 *   valid_ratio    S / bd^3
 *   skipped_bound1 sum over skipped triples of ||A_ik|| ||B_kj||
 *   skipped_bound2 sqrt(sum over tiles of (sum over skipped k of the product)^2);
 *                  ||AB - C||_F <= skipped_bound2 <= skipped_bound1 (exact arithmetic)
 *   norm_a, norm_b ||A||_F, ||B||_F recovered from the norm maps
 *   max_tile_survivors  largest per-tile count (kmax)
 *   nonempty_tiles tiles with at least one survivor
 *   flag_exponent  split modes: triples with floor(log2(p/(|A||B|))) >= this get hi+lo
 *   flagged        number of such triples */
typedef struct {
  int64_t survivors;
  int64_t nonempty_tiles;
  int64_t flagged;
  double valid_ratio;
  double skipped_bound1;
  double skipped_bound2;
  double norm_a;
  double norm_b;
  int32_t leaf;
  int32_t bd;
  int32_t max_tile_survivors;
  int32_t flag_exponent;
} spamm_stats_t;

typedef struct spamm_plan_s* spamm_plan_t;

/* ---------------------------------------------------------------------------
 * spamm_normmap -- Get-norm step (Section 3.2, Eq. 2).
 *   X        device, FP32 n x n row-major (ld = n), 16-byte aligned.
 *   normmap  device, FP64 [bd * bd] row-major: normmap[I*bd+K] = ||X[I,K]||_F
 *            over the zero-padded block.  Written completely.
 * Squares are formed exactly (FP32 products split by FMA), accumulated in
 * compensated double-FP32 groups and combined in FP64, so the result is
 * within 3e-13 relative of the exactly rounded norm (NaN entries give NaN;
 * an infinite entry gives NaN or +Inf, both of which survive every test).
 * Asynchronous on `stream`; allocates the device status word on first use.
 * Errors: SPAMM_ERR_INVALID_ARG (n < 1, null or misaligned pointer),
 * _UNSUPPORTED (leaf not 32/64/128, or ceil(n / leaf) > 1024), _CUDA
 * (launch failure).  Device
 * waits are bounded: if one expires, SPAMM_ERR_TIMEOUT is latched in the
 * status word (spamm_last_device_status) and the unfinished norms are NaN.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_normmap(const float* X, int64_t n, int32_t leaf, double* normmap,
                             void* stream);

/* spamm_normmap_pair: the norm maps of both operands of a product (A and B,
 * both n x n as for spamm_normmap) in one launch, their block rows dealt to
 * the same persistent grid: the same values as two spamm_normmap calls, one
 * launch tail instead of two.  normA and normB must differ. */
spamm_status_t spamm_normmap_pair(const float* A, const float* B, int64_t n, int32_t leaf,
                                  double* normA, double* normB, void* stream);

/* ---------------------------------------------------------------------------
 * Plans -- the pair test and work-queue build (Algorithm 2's bitmap and
 * map_offset, built once for all output tiles).
 *
 * spamm_plan_workspace_size: device bytes a plan for (n, leaf, precision)
 *   needs; the worst case (every triple surviving) is provisioned.
 * spamm_plan_create: allocates the plan.  `workspace` (device, 256-byte
 *   aligned, >= the size above) is used when non-NULL and stays owned by the
 *   caller; with NULL the library allocates and frees it itself.  Blocking
 *   only when it allocates.  The plan belongs to the current device.
 * spamm_plan_destroy: frees the plan (synchronises the device first).
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_plan_workspace_size(int64_t n, int32_t leaf, spamm_precision_t precision,
                                         size_t* bytes);
spamm_status_t spamm_plan_create(spamm_plan_t* plan, int64_t n, int32_t leaf,
                                 spamm_precision_t precision, void* workspace, size_t ws_bytes);
spamm_status_t spamm_plan_destroy(spamm_plan_t plan);

/* spamm_plan_set_schedule: the tile order of the plan's later multiplies
 *   (square and general plans): 0, the default (most survivors first, fixed
 *   interleave of the persistent CTAs); SPAMM_BATCH_DYNAMIC (32-tile chunks
 *   from a global counter); SPAMM_BATCH_GROUPS (groups of four tiles of a
 *   block row sharing each staged A block -- SPAMM_BF16 and SPAMM_FP16 at
 *   leaf 128 with alpha = 1, beta = 0 and no output norm map; other calls
 *   keep the per-tile order).  Every schedule gives the same bits.  Host-side
 *   only.  SPAMM_ERR_INVALID_ARG for a NULL plan or another value. */
spamm_status_t spamm_plan_set_schedule(spamm_plan_t plan, int32_t schedule);

/* ---------------------------------------------------------------------------
 * spamm_plan -- evaluate the skip rule of Algorithm 1 / Algorithm 2 for every
 * leaf triple (i, k, j) and build per-output-tile work queues.
 *   normA, normB  device FP64 [bd*bd] norm maps from spamm_normmap.
 *   tau           threshold; skip iff normA[i,k] * normB[k,j] < tau (FP64).
 *   target_rel_err split modes only: the relative error ||C - AB||_F /
 *                 (||A||_F ||B||_F) the caller aims for.  Triples get the
 *                 hi+lo product from the largest relative norm product
 *                 down until the hi-only bound of the rest fits half of
 *                 (target * ||A|| ||B|| - skipped_bound2).  Ignored otherwise.
 * The decision is taken in FP32 on a mantissa/exponent form and re-taken in
 * FP64 whenever the FP32 value lies within 2^-20 relative of tau, so it is
 * exactly the FP64 test for the given norm maps.  Survivors of a tile are
 * listed in increasing k.  Asynchronous; the plan may be executed by
 * spamm_multiply once this returns.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_plan(spamm_plan_t plan, const double* normA, const double* normB,
                          double tau, double target_rel_err, void* stream);

/* spamm_plan_stats: copies the plan's statistics to *stats (host).  Blocks
 * until the plan's work on `stream` is done. */
spamm_status_t spamm_plan_stats(spamm_plan_t plan, spamm_stats_t* stats, void* stream);

/* spamm_plan_export: copies the work queues to host arrays for inspection.
 *   tile_ptr  host int32 [bd*bd + 1] (may be NULL): CSR offsets, tile t = i*bd + j
 *   k_idx     host uint16 [survivors] (may be NULL): surviving k of each tile in
 *             increasing order; bit 15 set marks a split (hi+lo) triple.
 *   cap       capacity of k_idx in entries (SPAMM_ERR_NO_MEMORY if too small).
 * Blocks until the plan's work on `stream` is done. */
spamm_status_t spamm_plan_export(spamm_plan_t plan, int32_t* tile_ptr, uint16_t* k_idx,
                                 int64_t cap, void* stream);

/* ---------------------------------------------------------------------------
 * spamm_multiply -- the multiplication step (Section 3.3, Algorithm 2 /
 * Algorithm 3) over the plan's work queues:
 *   C[i,j] = sum over listed k of A[i,k] B[k,j], every tile written (beta = 0;
 *   tiles without survivors become zeros).
 *   A, B  device FP32 n x n (ld = n); C device FP32 n x n, written completely.
 * The precision is the plan's.  Tensor-core modes first round the blocks the
 * plan uses into plan-owned operand buffers.  Asynchronous.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_multiply(spamm_plan_t plan, const float* A, const float* B, float* C,
                              void* stream);

/* ---------------------------------------------------------------------------
 * spamm_plan_multiply -- spamm_plan followed by spamm_multiply in one call
 * (same arguments, same results).  Knowing C while planning lets the zeros of
 * the tiles without survivors be written as soon as the survivor counts are
 * known, overlapped with the rest of the plan and the multiply.
 * Asynchronous.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_plan_multiply(spamm_plan_t plan, const double* normA, const double* normB,
                                   double tau, double target_rel_err, const float* A,
                                   const float* B, float* C, void* stream);

/* ---------------------------------------------------------------------------
 * The general form -- Section 2 states the problem as C = alpha A B + beta C
 * for general A, B, C before fixing alpha = 1, beta = 0 and square operands:
 *
 *   C = alpha * sum over surviving k of A[i,k] B[k,j]  +  beta * C
 *
 * with A m x k, B k x n, C m x n, each row-major with its own leading
 * dimension, zero padded to whole leaf blocks: block grids bm x bk (A),
 * bk x bn (B), bm x bn (C), bm = ceil(m / leaf) and so on.  The skip rule is
 * the square one, triple by triple (skip iff normA[i,k] normB[k,j] < tau).
 * beta = 0 does not read C (NaN there does not propagate); tiles without
 * survivors become beta * C (left untouched at beta = 1).
 *
 * spamm_normmap_rect: the Eq. 2 norm map of a rows x cols operand (leading
 *   dimension ld >= cols, 16-byte aligned) into normmap [ceil(rows/leaf) *
 *   ceil(cols/leaf)], row-major; accuracy and errors as spamm_normmap.
 * spamm_plan_workspace_size_general / spamm_plan_create_general: a plan for
 *   the shape (m, k, n); arguments otherwise as for the square calls.
 *   Limits: ceil(k / leaf) <= 1024, bm * bn <= 2^22, bm * bk * bn < 2^31,
 *   every dimension <= 2^24 (SPAMM_ERR_UNSUPPORTED beyond).  spamm_plan,
 *   spamm_plan_band, spamm_plan_stats (its bd field holds bm),
 *   spamm_plan_export (tiles t = i * bn + j), spamm_tau_for_valid_ratio,
 *   spamm_norm_histogram and spamm_tau_predict take such a plan with normA
 *   [bm * bk] and normB [bk * bn]; spamm_multiply takes it with leading
 *   dimensions k, n, n, alpha = 1 and beta = 0.
 * spamm_multiply_general: the multiply over the plan's queues with leading
 *   dimensions lda >= k, ldb >= n, ldc >= n, alpha and beta (finite).  A, B
 *   and C are device FP32, 16-byte aligned; C may not overlap A or B.
 *   normC (device FP64 [bm * bn], 16-byte aligned, may be NULL) receives C's
 *   norm map as stored (||C[I,J]||_F of the written FP32 tile, the same
 *   accuracy as spamm_normmap), computed in the multiply's epilogue: the next
 *   product of a chain (matrix powers) plans from it without a norm pass over
 *   C.  Works on square plans too.  Asynchronous.
 * spamm_plan_multiply_general: spamm_plan followed by spamm_multiply_general
 *   in one call (the tiles without survivors are written as soon as the
 *   survivor counts are known).  Asynchronous.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_normmap_rect(const float* X, int64_t rows, int64_t cols, int64_t ld,
                                  int32_t leaf, double* normmap, void* stream);
spamm_status_t spamm_plan_workspace_size_general(int64_t m, int64_t k, int64_t n, int32_t leaf,
                                                 spamm_precision_t precision, size_t* bytes);
spamm_status_t spamm_plan_create_general(spamm_plan_t* plan, int64_t m, int64_t k, int64_t n,
                                         int32_t leaf, spamm_precision_t precision,
                                         void* workspace, size_t ws_bytes);
spamm_status_t spamm_multiply_general(spamm_plan_t plan, const float* A, int64_t lda,
                                      const float* B, int64_t ldb, float* C, int64_t ldc,
                                      float alpha, float beta, double* normC, void* stream);
spamm_status_t spamm_plan_multiply_general(spamm_plan_t plan, const double* normA,
                                           const double* normB, double tau, double target_rel_err,
                                           const float* A, int64_t lda, const float* B,
                                           int64_t ldb, float* C, int64_t ldc, float alpha,
                                           float beta, double* normC, void* stream);

/* ---------------------------------------------------------------------------
 * Error measures (Eq. 5): E = AB - SpAMM(A, B, tau).
 * spamm_frobenius_diff: *out = ||X - Y||_F over `count` FP32 entries
 *   (Y may be NULL for ||X||_F).  FP64 accumulation of exact FP32 squares.
 *   X, Y device; out host.  Blocks until done.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_frobenius_diff(const float* X, const float* Y, int64_t count, double* out,
                                    void* stream);

/* ---------------------------------------------------------------------------
 * spamm_multiply_fp32_noalloc -- the whole FP32 product (norm maps, plan,
 * SIMT multiply, identical arithmetic to spamm_normmap + spamm_plan +
 * spamm_multiply with SPAMM_FP32) without any device allocation.  The paper
 * has no counterpart: this serves callers that cannot allocate device memory
 * where they call it (a host framework whose pool already holds the device
 * memory, a plugin host that forbids allocation, a loop that cannot take
 * the synchronisation an allocation may bring).
 *   A, B, C   device FP32 n x n (ld = n), 16-byte aligned, C written completely.
 *   n, leaf   ceil(n / leaf) must be <= 64 (n <= 2048 at leaf 32, 4096 at 64,
 *             8192 at 128); larger sizes return SPAMM_ERR_UNSUPPORTED and
 *             enqueue nothing.
 *   tau       as for spamm_plan.
 * Its scratch is a 1 MiB array in the library's device memory (static, one
 * per device, kept until the process exits).  The first call on a device
 * looks that array up with cudaGetSymbolAddress; under lazy module loading
 * (the CUDA default) that is also when the library's device code is loaded
 * onto the device, so that one call may allocate driver memory for the
 * module and synchronise.  Make it at set-up (n = 1 is enough), before any
 * stream capture on that device.  The address is kept per CUDA context (by
 * the context's unique id): after cudaDeviceReset the next call looks it up
 * again.  Every call on a device shares the array and leaves its contents
 * behind; calls that overlap on the GPU race on it and must be serialised by
 * the caller.  A bounded wait of its norm maps that runs out latches
 * SPAMM_ERR_TIMEOUT in this entry point's own static status word, which
 * spamm_last_device_status reads and clears along with the library's.
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_multiply_fp32_noalloc(const float* A, const float* B, float* C, int64_t n,
                                           int32_t leaf, double tau, void* stream);

/* ---------------------------------------------------------------------------
 * Batches -- many independent products of uneven n (each one exactly the
 * product spamm_normmap + spamm_plan + spamm_multiply would give it alone,
 * with its own tau, statistics and bounds) run as ONE launch of each kernel:
 * one norm-map launch over both operands of every instance, one plan over
 * all triples of all instances, one rounding launch and one persistent
 * multiply whose work queue holds every non-empty output tile of the batch,
 * most survivors first.  The paper plans one product at a time (Section 3);
 * the batch is the serving form of the same rule.
 *
 * spamm_problem_t: one instance.  A, B, C device FP32 n x n (ld = n),
 *   16-byte aligned; C is written completely and may overlap no A, B or C of
 *   the batch.  tau as for spamm_plan.
 * spamm_batch_workspace_size / spamm_batch_create: the shapes (n[count]),
 *   leaf and precision are fixed at creation; pointers and tau may change on
 *   every run.  `workspace` as for spamm_plan_create.  flags:
 *   SPAMM_BATCH_GRAPH captures the launches of the first run into a CUDA
 *   graph and replays it on later runs (the instance table is re-uploaded,
 *   from pinned host memory, only when it changed).  SPAMM_BATCH_DYNAMIC
 *   makes the persistent multiply take its tiles in 32-tile chunks from a
 *   global counter instead of a fixed interleave.  SPAMM_BATCH_GROUPS (not
 *   with SPAMM_BATCH_DYNAMIC) multiplies the output tiles in groups of four
 *   consecutive tiles of a block row, staging each A_ik once for all tiles of
 *   the group that keep k: fewer staged bytes per product on dense-ish skip
 *   sets.  It takes effect for SPAMM_BF16 and SPAMM_FP16 at leaf 128; other
 *   configurations run the per-tile schedule.  The results equal those of
 *   the per-tile schedules bit for bit.  SPAMM_BATCH_TIMING
 *   records events around the three phases of every run (runs are then
 *   enqueued directly, never from the graph) for spamm_batch_timings.
 *   Creation allocates host staging memory and blocks.
 * spamm_batch_run: enqueues the whole batch on `stream` (asynchronous).
 *   target_rel_err as for spamm_plan (split modes only).
 * spamm_batch_stats: per-instance statistics into stats[count]; blocks.
 * spamm_batch_export: host copies of one instance's norm maps (FP64
 *   [bd*bd] each) and work queues (as spamm_plan_export); every pointer may
 *   be NULL; blocks.
 * spamm_batch_timings: ms[4] = device time of the norm maps, the plan, the
 *   operand rounding (0 for FP32) and the multiply of the last run
 *   (SPAMM_BATCH_TIMING only; the zero-fill of empty tiles runs beside the
 *   last three); blocks.
 * spamm_batch_autotune: times every candidate configuration on the given
 *   problems and returns the fastest in *best: leaf 64 and 128 (32, 64 and
 *   128 for FP32) times the static and dynamic multiply schedules (and the
 *   grouped one for BF16 and FP16 at leaf 128), each
 *   with graph replay, median of `reps` timed runs after two untimed ones.
 *   results[*nresults] (both may be NULL) receives every candidate, ms < 0
 *   for one that did not fit in memory; *nresults is set to the number of
 *   candidates.  Every candidate writes the C buffers (different leaves give
 *   different skip sets): run the chosen configuration afterwards.
 *   Allocates and blocks.
 * spamm_multiply_batched: create + run + stats (if non-NULL) + destroy, for a
 *   one-off batch; allocates and blocks.
 * spamm_batch_destroy: synchronises the device and frees the batch.
 * ------------------------------------------------------------------------- */
typedef struct {
  const float* A;
  const float* B;
  float* C;
  int64_t n;
  double tau;
} spamm_problem_t;

typedef struct spamm_batch_s* spamm_batch_t;

#define SPAMM_BATCH_GRAPH 1
#define SPAMM_BATCH_DYNAMIC 2
#define SPAMM_BATCH_TIMING 4
#define SPAMM_BATCH_GROUPS 8

typedef struct {
  int32_t leaf;
  int32_t flags;   /* SPAMM_BATCH_* flags of the configuration */
  float ms;        /* median time of one run, < 0 if the candidate could not run */
} spamm_tune_t;

spamm_status_t spamm_batch_workspace_size(const int64_t* n, int32_t count, int32_t leaf,
                                          spamm_precision_t precision, size_t* bytes);
spamm_status_t spamm_batch_create(spamm_batch_t* batch, const int64_t* n, int32_t count,
                                  int32_t leaf, spamm_precision_t precision, int32_t flags,
                                  void* workspace, size_t ws_bytes);
spamm_status_t spamm_batch_run(spamm_batch_t batch, const spamm_problem_t* problems,
                               double target_rel_err, void* stream);
spamm_status_t spamm_batch_stats(spamm_batch_t batch, spamm_stats_t* stats, void* stream);
spamm_status_t spamm_batch_export(spamm_batch_t batch, int32_t index, double* normA,
                                  double* normB, int32_t* tile_ptr, uint16_t* k_idx, int64_t cap,
                                  void* stream);
spamm_status_t spamm_batch_timings(spamm_batch_t batch, float* ms);
spamm_status_t spamm_batch_autotune(const spamm_problem_t* problems, int32_t count,
                                    spamm_precision_t precision, double target_rel_err,
                                    int32_t reps, void* stream, spamm_tune_t* best,
                                    spamm_tune_t* results, int32_t* nresults);
spamm_status_t spamm_multiply_batched(const spamm_problem_t* problems, int32_t count, int32_t leaf,
                                      spamm_precision_t precision, double target_rel_err,
                                      spamm_stats_t* stats, void* stream);
spamm_status_t spamm_batch_destroy(spamm_batch_t batch);

/* ---------------------------------------------------------------------------
 * Band plans -- the error measurement behind tau selection.
 * spamm_plan_band: as spamm_plan (FP32 precision only in meaning, any plan
 *   accepted), but lists the triples with tau_lo <= p < tau_hi (p the norm
 *   product, both tests exact in FP64; a NaN product is left out).  With C
 *   the product over that band, AB - SpAMM(A, B, tau_hi) = C + (AB -
 *   SpAMM(A, B, tau_lo)): against a reference tau_lo whose skipped bound is
 *   negligible, ||C||_F is the pruning error at tau_hi without forming AB.
 *   Only survivors, nonempty_tiles and max_tile_survivors of the statistics
 *   are meaningful for a band plan.  tau_hi >= tau_lo >= 0, not NaN.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_plan_band(spamm_plan_t plan, const double* normA, const double* normB,
                               double tau_lo, double tau_hi, void* stream);

/* ---------------------------------------------------------------------------
 * spamm_tau_for_valid_ratio -- the paper's search for a customised accuracy
 * (Section 3.5.2): tau whose valid ratio S / bd^3 is within `tol` of
 * `target_ratio`.  ave = mean norm product over all bd^3 triples (closed
 * form sum_k colsum_A(k) rowsum_B(k) / bd^3); the interval [0, k ave] is
 * widened (k = 1, 2, ...) until its end gives a ratio <= target, the first
 * probe is min(ave, k ave), then bisection until within tol or max_probes
 * probes.  Each probe is the counting half of a plan (no queues).  Outputs
 * (host): *tau, and *ratio / *probes when non-NULL.  Blocks.  The plan's
 * buffers are used: plan again (spamm_plan) afterwards.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_tau_for_valid_ratio(spamm_plan_t plan, const double* normA,
                                         const double* normB, double target_ratio, double tol,
                                         int32_t max_probes, double* tau, double* ratio,
                                         int32_t* probes, void* stream);

/* ---------------------------------------------------------------------------
 * Learned tau.  The paper picks tau by a search for a target valid ratio
 * (Section 3.5.2); here a small network maps the distribution of the norm
 * products and a target relative error ||C - AB||_F / (||A||_F ||B||_F) to
 * tau in one forward pass.
 *
 * Features: the 64-bin histogram of r = p / (||A||_F ||B||_F) over all bd^3
 * triples (p = normA[i,k] normB[k,j] in FP64, ||.||_F from the norm maps),
 * bin t = min(63, max(0, floor(-log2 r))), r = 0 or NaN in bin 63, +Inf in
 * bin 0, each bin divided by bd^3; then log10(target).  Network: FP32,
 * Linear(65,64) - GELU - Linear(64,64) - GELU - Linear(64,1) with exact
 * GELU 0.5 z (1 + erf(z / sqrt 2)); output y = log10(tau / (||A|| ||B||)).
 * Parameters: one device FP32 array of 8449 values: W1 (64 x 65, row-major,
 * y = W x + b), b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1).
 *
 * spamm_norm_histogram: the raw bin counts (host int64[64]) for the plan's
 *   shape; blocks.
 * spamm_tau_predict: the predicted tau (host) for a target in (0, inf);
 *   blocks.  It uses the plan's buffers: plan again (spamm_plan) afterwards.
 * spamm_batch_tau_predict: per instance of a batch (norm maps of the given
 *   A and B computed on the way; C and tau of the problems are not read),
 *   targets and taus host arrays of `count`; blocks.
 * spamm_mlp_param_count: 8449.
 * spamm_mlp_forward: y[count] = network(X[count][65]); all device pointers.
 * spamm_mlp_grad: gradient (device [8449]) and value (device [1]) of the
 *   pinball loss mean_s rho_q(y_true[s] - y[s]), rho_q(r) = max(q r,
 *   (q - 1) r), over count samples; 0 < quantile < 1.
 * spamm_mlp_adam: one Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected
 *   with step number t >= 1) on device weights with device moments m, v.
 * spamm_mlp_train: `steps` Adam steps (numbers t0 + 1 ...); step s uses the
 *   samples idx[s * batch .. (s + 1) * batch) (device int32) of X / y_true;
 *   loss_hist (device [steps], may be NULL) receives each step's loss.  One
 *   CTA runs the whole loop with the weights on chip.
 * All are asynchronous unless stated.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_norm_histogram(spamm_plan_t plan, const double* normA, const double* normB,
                                    int64_t* counts, void* stream);
spamm_status_t spamm_tau_predict(spamm_plan_t plan, const double* normA, const double* normB,
                                 double target_rel_err, const float* weights, double* tau,
                                 void* stream);
spamm_status_t spamm_batch_tau_predict(spamm_batch_t batch, const spamm_problem_t* problems,
                                       const double* targets, const float* weights,
                                       double* taus, void* stream);
spamm_status_t spamm_mlp_param_count(int32_t* count);
spamm_status_t spamm_mlp_forward(const float* weights, const float* X, int32_t count, float* y,
                                 void* stream);
spamm_status_t spamm_mlp_grad(const float* weights, const float* X, const float* y_true,
                              int32_t count, float quantile, float* grad, float* loss,
                              void* stream);
spamm_status_t spamm_mlp_adam(float* weights, const float* grad, float* m, float* v, int32_t t,
                              float lr, void* stream);
spamm_status_t spamm_mlp_train(float* weights, float* m, float* v, int32_t t0, const float* X,
                               const float* y_true, const int32_t* idx, int32_t steps,
                               int32_t batch, float lr, float quantile, float* loss_hist,
                               void* stream);

/* ---------------------------------------------------------------------------
 * Choosing tau for a target error -- the arbiter and fallback of the learned
 * tau.  The paper searches tau for a valid ratio (Section 3.5.2); these
 * calls choose it for the pruning error of Eq. 5 relative to the operands,
 * e(tau) = ||AB - SpAMM(A, B, tau)||_F / (||A||_F ||B||_F), without forming AB.
 * All use the plan's buffers (plan again with spamm_plan afterwards) and block.
 * Square plans only (SPAMM_ERR_UNSUPPORTED for a plan of the general form).
 *
 * spamm_tau_certify: *tau_ref = the largest tau = ||A|| ||B|| 10^x, x found
 *   by 36 bisection steps over [-60, 0], whose skipped bound2 is <=
 *   ref_rel ||A|| ||B|| (so ||AB - SpAMM(tau_ref)||_F <= ref_rel ||A|| ||B||);
 *   0 when ||A|| ||B|| is 0 or not finite.  *norm_ab (may be NULL) =
 *   ||A||_F ||B||_F from the norm maps.  ref_rel in (0, inf).
 * spamm_tau_error: *err = e(tau) up to ref_rel: 0 when tau <= tau_ref, else
 *   ||C_band||_F / (||A|| ||B||), C_band the FP32 product over the triples with
 *   tau_ref <= p < tau (a band plan and the SIMT multiply into `scratch`).
 *   A, B device FP32 n x n as for spamm_multiply; scratch device FP32 n x n,
 *   16-byte aligned, aliasing neither, overwritten.
 * spamm_tau_select: tau for target_rel_err in (0, inf).  tau_ref is
 *   certified at ref_rel = 1e-11.  With `weights` (device FP32 [8449], the
 *   network of spamm_tau_predict) the predicted tau is checked once with
 *   spamm_tau_error and returned if e <= target.  Otherwise (a miss, or
 *   weights == NULL) bisection on e: lo = 0, hi = target ||A|| ||B||; if e(hi)
 *   <= target, hi moves up by factors of 10 while admissible, else down by
 *   factors of 10 until an admissible tau is found; then hi := sqrt(lo hi) or
 *   lo := sqrt(lo hi) until hi / lo <= 1.01, at most 40 evaluations of e in
 *   all.  *tau = the largest admissible tau tested (0 if none), *evals
 *   (may be NULL) = evaluations of e including the network's check,
 *   *achieved (may be NULL) = e(*tau).
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_tau_certify(spamm_plan_t plan, const double* normA, const double* normB,
                                 double ref_rel, double* tau_ref, double* norm_ab, void* stream);
spamm_status_t spamm_tau_error(spamm_plan_t plan, const double* normA, const double* normB,
                               const float* A, const float* B, double tau, double tau_ref,
                               float* scratch, double* err, void* stream);
spamm_status_t spamm_tau_select(spamm_plan_t plan, const double* normA, const double* normB,
                                const float* A, const float* B, double target_rel_err,
                                const float* weights, float* scratch, double* tau,
                                int32_t* evals, double* achieved, void* stream);

/* ---------------------------------------------------------------------------
 * spamm_peak_rates -- measured peak rates of this GPU, the denominators of
 * roofline fractions for which no library routine gives one.  The paper has
 * no counterpart (it quotes no hardware rates).  tflops (host double[5]):
 *   [0] FP32 FFMA on the SIMT cores, [1] FP64 DFMA, [2] BF16, [3] FP16 and
 *   [4] TF32 dense tcgen05 MMA with FP32 accumulation (one CTA per SM issuing
 *   back-to-back 128 x N x K MMAs on operands resident in shared memory, the
 *   better of N = 128 and 256).  Each is the second of two launches, timed
 *   with events.  Allocates a small buffer, takes tens of milliseconds and
 *   blocks; SPAMM_ERR_TIMEOUT if an MMA launch did not complete in time.
 * ------------------------------------------------------------------------- */
spamm_status_t spamm_peak_rates(double* tflops, void* stream);

/* ---------------------------------------------------------------------------
 * Status helpers.
 * spamm_status_string: static description of a status code.
 * spamm_last_device_status: reads and clears the library's device status word
 *   for the current device, and the static one of spamm_multiply_fp32_noalloc
 *   once that entry point has run in the current context (0 = clean, else a
 *   spamm_status_t; the library's word first when both are set).  Blocks.
 * ------------------------------------------------------------------------- */
const char* spamm_status_string(spamm_status_t status);
spamm_status_t spamm_last_device_status(void* stream, int32_t* code);

/* spamm_selftest_bounded_wait: runs the bounded wait routines of the
 *   tensor-core multiply (one thread) and of the norm map (a whole warp) on an
 *   mbarrier phase that nothing completes, with the given limit (1 us .. 1 s).
 *   Each wait gives up, raises its abort flag and latches SPAMM_ERR_TIMEOUT in
 *   the device status word (read it with spamm_last_device_status); returns
 *   SPAMM_OK when all of that happened for both, *elapsed_ns (may be NULL) =
 *   the shorter of the two waits.  Blocks.  No part of the GPU is left waiting. */
spamm_status_t spamm_selftest_bounded_wait(int64_t limit_ns, int64_t* elapsed_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPAMM_H */
