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
  int32_t* ea;   // [bd*bd]
  int32_t* eb;   // [bd*bd]
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

// Operand images are indexed by the global block number (tile0 + I * bd + K).
cudaError_t launch_quantize(spamm_precision_t prec, int leaf, const InstRef& ref,
                            const PlanBuffers& b, const OperandImages& img, cudaStream_t s);

cudaError_t launch_multiply_tc(spamm_precision_t prec, int leaf, const InstRef& ref,
                               const PlanBuffers& b, const OperandImages& img, int32_t* status,
                               int schedule, cudaStream_t s);

// Writes zeros to every tile without survivors, of every instance (reads the
// plan's empty-tile list: after the whole plan).
cudaError_t launch_zero_empty_tiles(const InstRef& ref, const PlanBuffers& b, int leaf,
                                    cudaStream_t s);

// Self-test of the multiply's bounded wait on a phase that never completes.
cudaError_t launch_wait_selftest(int32_t* status, uint64_t limit_ns, long long* out,
                                 cudaStream_t s);

// The same from the per-tile counts alone: may run as soon as the plan's
// counting half has finished.
cudaError_t launch_zero_empty_tiles_scan(const InstRef& ref, const PlanBuffers& b, int leaf,
                                         cudaStream_t s);

}  // namespace spamm
