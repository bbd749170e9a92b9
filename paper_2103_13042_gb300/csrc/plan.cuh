// Device-side plan state shared by the plan and multiply kernels.
//
// Every kernel works on a table of SpAMM instances (one entry for a single
// product, many for a batch).  An instance is the general product of
// Section 2, C = alpha * SpAMM(A, B) + beta * C, with A m x kd, B kd x n and
// C m x n (row-major, leading dimensions lda, ldb, ldc), zero padded to whole
// leaf blocks: block grids bm x bk (A), bk x bn (B) and bm x bn (C).  The
// square product of the rest of the paper is m = kd = n, alpha = 1, beta = 0.
// Instance i owns bm_i * bn_i output tiles, numbered globally from tile0_i
// (the sum over the instances before it), bm_i * bk_i blocks of A from ablk0_i
// and bk_i * bn_i blocks of B from bblk0_i (block (I, K) of A is
// ablk0 + I * bk + K, block (K, J) of B is bblk0 + K * bn + J).  Its
// surviving k indices live in k_idx slots from kidx0_i = sum of bm * bk * bn
// of the instances before it.  All instances of a table share one leaf size.
#pragma once

#include "common.cuh"

namespace spamm {

// The threshold in the form the pair test uses (built on the host).
struct TauScreen {
  double tau;
  float m_lo, m_hi;
  int32_t e;
  int all;   // tau == 0: every triple survives
  int none;  // tau == +Inf: only non-finite products survive
};

TauScreen make_tau_screen(double tau);

// Bins of the log2 histogram of relative norm products (tau prediction).
constexpr int kHistBins = 64;

// Longest-first buckets of the multiply's tile order: key = floor(log2 c) + 1
// for a tile with c >= 1 survivors (c <= 1024: keys 1 .. 11), largest first;
// inside a bucket the tiles keep the plan's enumeration order.
constexpr int kOrderKeys = 12;

// Per-instance statistics; `ticket` and the bins are cleared before each plan.
struct PlanDevice {
  double norm_a, norm_b, inv_ab;
  double bound1, bound2, valid_ratio;
  long long survivors, flagged;
  int max_tile, nonempty, flag_exp;
  int ne_base;                              // non-empty tiles of the instances before this one
  unsigned int hist[kHistBins];             // norm-product histogram (tau prediction)
  int key_tot[kOrderKeys];                  // non-empty tiles per order bucket
  int key_base[kOrderKeys];                 // first slot of this instance in each bucket
  unsigned int ticket;                      // prep CTAs of this instance that have finished
  double bin_sum[kFlagBins];                // surviving products per relative binade
  unsigned long long bin_cnt[kFlagBins];
};

// Batch-wide state of the longest-first order (cleared before each plan).
struct BatchDevice {
  int hist[kMaxBd + 2];     // non-empty tiles per survivor count, over all instances
  int cursor[kMaxBd + 2];   // next slot of each count's bucket in `order`
  int nonempty;             // non-empty tiles over all instances
  unsigned int ticket;      // finalize CTAs that have finished
  int mul_ticket;           // next slot of `order` to hand out (dynamic multiply schedule)
  int need_count;           // entries of the needed-block list
};

// Multiply schedules: CTAs walk the longest-first order with a fixed
// interleave (static) or take 32-slot chunks from a global counter (dynamic);
// or (tensor modes, leaf 128) take groups of four tiles of one block row that
// share their A operands (groups).
enum Schedule { kScheduleStatic = 0, kScheduleDynamic = 1, kScheduleGroups = 2 };

// Tiles per group of the grouped multiply: one block row, kGroupTiles
// consecutive block columns.
constexpr int kGroupTiles = 4;

// Extended-range FP32 sum: value = m * 2^e with an integer exponent.
struct ExtSum {
  float m;
  int e;
};

// One SpAMM instance.
struct Inst {
  const float* A;
  const float* B;
  float* C;
  const double* nA;     // norm maps: A [bm * bk], B [bk * bn], row-major
  const double* nB;
  double* nC;           // C's norm map [bm * bn], written by the multiply when non-null
  int64_t m, kd, n;     // C is m x n, A is m x kd, B is kd x n
  int64_t lda, ldb, ldc;
  int bm, bk, bn;       // block grids
  float alpha, beta;    // C = alpha * sum + beta * C; beta = 0: the old C is not read
  int split;            // 1: BF16/FP16 split mode (dominant triples get hi+lo)
  int quant;            // 1: the multiply rounds operands (build the needed-block list)
  int64_t tile0;        // first global output tile
  int64_t ablk0;        // first global block of A
  int64_t bblk0;        // first global block of B
  int64_t kidx0;        // first k_idx slot
  int64_t mask0;        // first word of the survivor bitmask (bm * bn * ceil(bk / 32) words)
  int64_t grp0;         // first global tile group (bm * ceil(bn / kGroupTiles) groups)
  int prep0;            // first CTA of this instance in the prep grid
  int count0;           // first CTA of this instance in the count and fill grids
  double target_rel;    // split modes: relative error target
  double c1;            // split modes: hi-only error coefficient 2u + u^2
  TauScreen T;
  TauScreen T_hi;       // band plans: triples with p >= T_hi.tau are left out too
  int band;             // 1: multiply only tau <= p < T_hi.tau
  int pad_;
  PlanDevice* pd;
};

// The instance table a kernel reads: a device array, or one instance passed
// by value (then `table` is null).
struct InstRef {
  const Inst* table;
  Inst one;
  int count;
  int any_split, any_band;   // some instance uses split flags / a band (host-side dispatch)
  int any_norm_out;          // some instance writes an output norm map (nC)
  int any_scaled;            // some instance has alpha != 1 or beta != 0
  __device__ __forceinline__ const Inst& at(int i) const { return table ? table[i] : one; }
};

// Largest i with key(i) <= v over a non-decreasing key (0 for a single instance).
template <typename Key>
__device__ __forceinline__ int find_inst(const InstRef& r, int64_t v, Key key) {
  if (r.count <= 1) return 0;
  int lo = 0, hi = r.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (key(r.at(mid)) <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int inst_of_tile(const InstRef& r, int64_t g) {
  return find_inst(r, g, [](const Inst& x) { return x.tile0; });
}
__device__ __forceinline__ int inst_of_ablk(const InstRef& r, int64_t g) {
  return find_inst(r, g, [](const Inst& x) { return x.ablk0; });
}
__device__ __forceinline__ int inst_of_bblk(const InstRef& r, int64_t g) {
  return find_inst(r, g, [](const Inst& x) { return x.bblk0; });
}
__device__ __forceinline__ int inst_of_group(const InstRef& r, int64_t g) {
  return find_inst(r, g, [](const Inst& x) { return x.grp0; });
}

// Device buffers of a plan (carved from one workspace allocation).
struct PlanBuffers {
  int64_t tiles;       // sum of bm * bn (output tiles)
  int64_t groups;      // sum of bm * ceil(bn / kGroupTiles) (tile groups)
  int64_t ablks;       // sum of bm * bk (blocks of A)
  int64_t bblks;       // sum of bk * bn (blocks of B)
  int64_t kslots;      // sum of bm * bk * bn
  int prep_ctas;       // prep grid
  int count_ctas;      // count and fill grids
  int max_bk;          // largest bk of the table (the count kernel's shared-memory size)
  Screen* sA;          // [ablks] screen form of normA, row-major per instance
  Screen* sBT;         // [bblks] screen form of normB, transposed per instance (J * bk + K)
  double* part_a;      // [prep_ctas] partial sums of squared norms
  double* part_b;
  long long* part_S;   // [count_ctas] per-CTA partials of the count kernel
  int* part_kmax;
  int* part_ne;
  ExtSum* part_b1;     // sums of skipped relative products
  ExtSum* part_b2;     // sums of their per-tile squares
  int* cta_base;       // [count_ctas] first k_idx slot of the CTA's tiles
  int* ne_cta_base;    // [count_ctas] non-empty tiles of the instance's earlier CTAs
  int* part_keys;      // [count_ctas * kOrderKeys] non-empty tiles of the CTA per bucket
  int* key_cta_base;   // [count_ctas * kOrderKeys] the instance's earlier CTAs' tiles per bucket
  int* cnt;            // [tiles] survivors per tile
  int* tile_beg;       // [tiles] absolute first k_idx slot of the tile
  int* order;          // [tiles] global ids: the non-empty tiles, most survivors first, then
                       // the empty tiles in increasing order
  uint16_t* k_idx;     // [kslots] surviving k per tile, increasing (bit 15: split triple)
  int* tile_inst;      // [tiles] instance of each global output tile
  uint32_t* surv_mask; // survivors of each tile, 32 k per word (tile t = i*bn + j of an instance)
  uint32_t* need_bits; // [words_a + words_b] bit g: block g of A (first part) / B (second) is used
  uint32_t* need_list; // [ablks + bblks] used blocks, each once: g (A) or g | 2^31 (B)
  int64_t need_words_a;   // 32-bit words of the A part of need_bits
  int64_t need_words_b;
  void* norm_part;     // tensor modes with an output norm map: per-tile partial sums
  PlanDevice* pd;      // [instances]; pd, bdev and need_bits are contiguous (one memset)
  BatchDevice* bdev;
};

// Instance of a global output tile.
__device__ __forceinline__ int inst_of(const InstRef& r, const PlanBuffers& b, int64_t g) {
  return r.count <= 1 ? 0 : b.tile_inst[g];
}

// Grid sizes of the plan kernels for one instance.
int prep_ctas_of(const Inst& in);
int count_ctas_of(const Inst& in);

// Sets the shape fields of a square n x n instance (alpha = 1, beta = 0).
void set_square(Inst& in, int64_t n, int leaf);
// Sets the shape fields of C (m x n) = A (m x kd) B (kd x n) with the given
// leading dimensions, alpha and beta.
void set_general(Inst& in, int64_t m, int64_t kd, int64_t n, int64_t lda, int64_t ldb,
                 int64_t ldc, float alpha, float beta, int leaf);

// Fills the layout fields of `insts` (tile0, ablk0, bblk0, kidx0, mask0,
// prep0, count0; the shape fields must be set) and of `b`; carves the buffers
// from `base` when non-null.  Returns the bytes needed.
// `norm_parts`: also provision the per-tile partial sums of the tensor-core
// epilogue's output norm maps.
size_t plan_layout(Inst* insts, int count, PlanBuffers* b, char* base, bool norm_parts = false);

// Host wrapper of a table: `dev_table` holds a device copy (batches) or is
// null (a single instance, passed by value).
InstRef make_ref(const Inst* host_insts, const Inst* dev_table, int count);

cudaError_t run_plan(const InstRef& ref, const PlanBuffers& b, cudaStream_t s);

// run_plan in two halves: the first ends once every tile's survivor count is
// known (cnt), the second builds the queues and the order.
cudaError_t run_plan_count_half(const InstRef& ref, const PlanBuffers& b, cudaStream_t s);
cudaError_t run_plan_queue_half(const InstRef& ref, const PlanBuffers& b, cudaStream_t s);

// The plan's counting half (statistics, survivors per tile; no queues).
cudaError_t run_plan_count(const InstRef& ref, const PlanBuffers& b, cudaStream_t s);

// Clears the statistics, builds the screen forms and norms (as run_plan's
// first step) and the per-instance norm-product histograms (pd[i].hist).
cudaError_t run_histogram(const InstRef& ref, const PlanBuffers& b, cudaStream_t s);

// Norm map of one n x n operand.  `status` (may be null) receives
// SPAMM_ERR_TIMEOUT if a bounded wait of the staged form expires; the norms
// that were not finished are then NaN.
cudaError_t launch_normmap(const float* X, int64_t n, int32_t leaf, double* out, int32_t* status,
                           cudaStream_t s);
// Both n x n operands of a product in one launch (their units dealt together).
cudaError_t launch_normmap_pair(const float* A, const float* B, int64_t n, int32_t leaf,
                                double* outA, double* outB, int32_t* status, cudaStream_t s);
// The same for a rows x cols operand with leading dimension ld.
cudaError_t launch_normmap_rect(const float* X, int64_t rows, int64_t cols, int64_t ld,
                                int32_t leaf, double* out, int32_t* status, cudaStream_t s);

// Norm-map jobs (one per operand of an instance) of the staged norm-map
// kernel: X is rows x cols, row-major with leading dimension ld, 16-byte
// aligned; out is [br * bc].  A job table lists the jobs whose rows are
// 16-byte aligned (vec: ld % 4 == 0) first, then the others; unit0 counts the
// kernel's units (block rows x column windows) from the start of the job's
// part of the table.
struct NormJob {
  const float* X;
  double* out;
  int64_t rows, cols, ld;
  int br, bc, nwin, unit0, vec;
  int lines;   // every row starts on a 128-byte line (X 128-byte aligned, ld % 32 == 0)
};
// Self-test of the norm map's bounded wait (a phase nothing completes).
cudaError_t launch_normmap_wait_selftest(int32_t* status, uint64_t limit_ns, long long* out,
                                         cudaStream_t s);
// Sets br, bc, nwin and lines from X, rows, cols, ld, vec and the leaf;
// returns the job's units.
int normjob_shape(NormJob& j, int leaf);
// Both kinds of jobs (16-byte aligned rows, others); with a side stream and two
// events they run at once, sharing the SMs in proportion to their units.
cudaError_t launch_normmap_jobs(const NormJob* dev_jobs, int n_vec, int units_vec, int n_other,
                                int units_other, int leaf, int32_t* status, cudaStream_t s,
                                cudaStream_t side = nullptr, cudaEvent_t fork = nullptr,
                                cudaEvent_t join = nullptr);

cudaError_t launch_multiply_simt(const InstRef& ref, const PlanBuffers& b, int leaf,
                                 int schedule, cudaStream_t s);

// Per-tile partial sums of squares of the tensor-core epilogue (output norm
// maps): one per epilogue warp of a tile, merged by launch_norm_out_finish.
constexpr int kMaxEpiWarps = 8;
struct NormPart {
  float hi, lo;
  int e, pad_;
};

// Learned tau (FP32 network, 8449 parameters).
int mlp_param_count();
cudaError_t launch_mlp_forward(const float* W, const float* X, int count, float* Y,
                               cudaStream_t s);
cudaError_t launch_mlp_grad(const float* W, const float* X, const float* Y, int count, float q,
                            float* grad, float* loss, cudaStream_t s);
cudaError_t launch_mlp_adam(float* W, const float* grad, float* m, float* v, int t, float lr,
                            cudaStream_t s);
cudaError_t launch_mlp_train(float* W, float* m, float* v, int t0, const float* X, const float* Y,
                             const int* idx, int steps, int batch, float lr, float q,
                             float* loss_hist, cudaStream_t s);
// tau[i] (and the 65 features, when feats is non-null) of every instance
// from pd[i].hist, pd[i].norm_a/b and Inst::target_rel.
cudaError_t launch_tau_from_hist(const InstRef& ref, const float* W, float* feats, double* tau,
                                 cudaStream_t s);

cudaError_t launch_frobenius_diff(const float* X, const float* Y, int64_t count, double* partials,
                                  int nparts, double* out, cudaStream_t s);

}  // namespace spamm
