// Layout constants shared by the operand rounding and tensor-core multiply kernels.
#pragma once

#include "plan.cuh"
#include "tc.cuh"

namespace spamm {

// Operand images of one plan: per leaf block a K-major, 128-byte swizzled
// image (hi, and lo in split modes) plus the block's power-of-two exponent.
struct OperandImages {
  uint8_t* a_hi;
  uint8_t* a_lo;
  uint8_t* b_hi;
  uint8_t* b_lo;
  int32_t* ea;   // [ablks] per block of A
  int32_t* eb;   // [bblks] per block of B
};

template <uint32_t FMT, int LEAF>
struct TcLayout {
  static constexpr int kElt = FMT == tc::kFmtTF32 ? 4 : 2;      // bytes per element
  static constexpr int kKc = 128 / kElt;                        // K elements per 128-byte row
  static constexpr int kNch = LEAF / kKc;                       // 128-byte chunks per block row
  static constexpr uint32_t kChunkBytes = LEAF * 128;           // one chunk of one block
  static constexpr uint32_t kBlockBytes = kChunkBytes * kNch;   // = LEAF * LEAF * kElt
  static constexpr int kLoShift = FMT == tc::kFmtBF16 ? 8 : 11; // lo part scaled by 2^kLoShift
};

// Waits of the persistent tensor-core multiplies: 2 s is a safety net, never
// hit normally; 100 ms for the drain after an abort.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 100000000ull;

// Bounded wait that also returns when another role raised the abort flag.
__device__ __forceinline__ bool wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        int32_t* status, uint64_t limit_ns = kWaitLimitNs) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = tc::globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0) {
      if (*abort_flag) return false;
      if (tc::globaltimer_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicExch(status, (int32_t)SPAMM_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// One MMA of the format's kind (kind::tf32 or kind::f16).
template <uint32_t FMT>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accumulate) {
  if constexpr (FMT == tc::kFmtTF32) tc::mma_tf32(d, a, b, id, accumulate);
  else tc::mma_f16(d, a, b, id, accumulate);
}

// Operand images are indexed by the global block number (ablk0 + I * bk + K
// for A, bblk0 + K * bn + J for B).
cudaError_t launch_quantize(spamm_precision_t prec, int leaf, const InstRef& ref,
                            const PlanBuffers& b, const OperandImages& img, cudaStream_t s);

cudaError_t launch_multiply_tc(spamm_precision_t prec, int leaf, const InstRef& ref,
                               const PlanBuffers& b, const OperandImages& img, int32_t* status,
                               int schedule, cudaStream_t s);

// The grouped multiply (groups of four tiles of a block row sharing their A
// operands): leaf 128, BF16 or FP16, alpha = 1, beta = 0, no output norm map.
bool multiply_tc_groups_supported(spamm_precision_t prec, int leaf, const InstRef& ref);
cudaError_t launch_multiply_tc_groups(spamm_precision_t prec, const InstRef& ref,
                                      const PlanBuffers& b, const OperandImages& img,
                                      int32_t* status, cudaStream_t s);

// Writes every tile without survivors, of every instance: beta * C (zeros at
// beta = 0; the tile's norm into nC when set).  Reads the plan's empty-tile
// list: after the whole plan.
cudaError_t launch_zero_empty_tiles(const InstRef& ref, const PlanBuffers& b, int leaf,
                                    cudaStream_t s);

// Output norm maps of the tensor-core multiply: merges the epilogue's per-tile
// partial sums into each instance's nC (after launch_multiply_tc).
cudaError_t launch_norm_out_finish(const InstRef& ref, const PlanBuffers& b, int leaf,
                                   cudaStream_t s);

// Self-test of the multiply's bounded wait on a phase that never completes.
cudaError_t launch_wait_selftest(int32_t* status, uint64_t limit_ns, long long* out,
                                 cudaStream_t s);

// The same from the per-tile counts alone: may run as soon as the plan's
// counting half has finished.
cudaError_t launch_zero_empty_tiles_scan(const InstRef& ref, const PlanBuffers& b, int leaf,
                                         cudaStream_t s);

}  // namespace spamm
