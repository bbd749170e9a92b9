// Device-side plan state shared by the plan and multiply kernels.
#pragma once

#include "common.cuh"

namespace spamm {

// Scalars the plan kernels produce (one per plan, in device memory).  The
// members from `hist` on are accumulators cleared at the start of every plan.
struct PlanDevice {
  double norm_a, norm_b, inv_ab;
  double bound1, bound2, valid_ratio;
  long long survivors, flagged;
  int max_tile, nonempty, flag_exp, pad_;
  int cursor[kMaxBd + 2];                   // next longest-first slot per survivor count
  int hist[kMaxBd + 2];                     // number of tiles per survivor count (>= 1)
  unsigned int ticket;                      // prep CTAs that have finished
  unsigned int pad2_;
  double bin_sum[kFlagBins];                // surviving products per relative binade
  unsigned long long bin_cnt[kFlagBins];
};

// Extended-range FP32 sum: value = m * 2^e with an integer exponent.
struct ExtSum {
  float m;
  int e;
};

// Device buffers of one plan (carved from one workspace allocation).
struct PlanBuffers {
  int bd;
  Screen* sA;          // [bd*bd] screen form of normA, row-major
  Screen* sBT;         // [bd*bd] screen form of normB, transposed (j-major)
  double* part_a;      // per-CTA partial sums (prep)
  double* part_b;
  long long* part_S;   // per-CTA partials (count)
  int* part_kmax;
  int* part_ne;
  ExtSum* part_b1;     // per-CTA sums of skipped relative products
  ExtSum* part_b2;     // per-CTA sums of their squares per tile
  int* cta_base;       // per count-CTA: first k_idx slot of its tiles
  int* cta_ebase;      // per count-CTA: empty tiles before its tiles
  int* cnt;            // [bd*bd] survivors per tile
  int* tile_ptr;       // [bd*bd + 1] CSR offsets
  int* order;          // [bd*bd] tiles, most survivors first, empty tiles last
  uint16_t* k_idx;     // [bd^3] surviving k per tile (bit 15: split triple)
  uint8_t* needA;      // [bd*bd] 1 if block A[i,k] takes part in some surviving triple
  uint8_t* needB;      // [bd*bd] 1 if block B[k,j] takes part in some surviving triple
  PlanDevice* pd;
};

cudaError_t run_plan(PlanBuffers& b, const double* nA, const double* nB, double tau,
                     double target_rel, int split, double c1, cudaStream_t s);
int64_t plan_part_count(int bd);

// Carves the plan buffers for a bd x bd grid out of `base` (NULL: size only);
// returns the bytes needed (256-byte aligned pieces).
size_t plan_layout(int bd, PlanBuffers* b, char* base);

cudaError_t launch_normmap(const float* X, int64_t n, int32_t leaf, double* out, cudaStream_t s);

cudaError_t launch_multiply_simt(const PlanBuffers& b, const float* A, const float* B, float* C,
                                 int64_t n, int32_t leaf, cudaStream_t s);

cudaError_t launch_frobenius_diff(const float* X, const float* Y, int64_t count, double* partials,
                                  int nparts, double* out, cudaStream_t s);

}  // namespace spamm
