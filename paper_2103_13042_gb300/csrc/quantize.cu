// Operand rounding for the tensor-core multiply (spec mixed precision on
// top of the paper's FP16 tensor-core kernel, Section 3.3 / Algorithm 3).
//
// For every leaf block that some surviving triple uses (the plan's list of
// needed blocks) one CTA finds e = frexp exponent of its largest magnitude,
// scales by 2^-e (exact), rounds to nearest-even in the operand format (hi)
// and, in split modes, rounds the exact residual scaled by 2^s_lo (lo).  The result is written directly as the K-major, 128-byte
// swizzled image the MMA reads: chunk c of a block holds K elements
// [c*kc, (c+1)*kc) (kc = 128 bytes / element size) for every row, 128 bytes
// per row, 16-byte pieces XOR-swizzled by (row mod 8).  A blocks keep their
// rows; B blocks are transposed (image row n = column n of the block).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc.cuh"
#include "tc_common.cuh"

namespace spamm {
namespace {


// Round to nearest even, keeping 10 explicit significand bits (TF32), on the
// IEEE bit pattern; NaN/Inf pass through unchanged.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0xfffu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xffffe000u);
}

template <uint32_t FMT>
__device__ __forceinline__ float round_op(float x) {
  if constexpr (FMT == tc::kFmtBF16) return __bfloat162float(__float2bfloat16_rn(x));
  else if constexpr (FMT == tc::kFmtF16) return __half2float(__float2half_rn(x));
  else return round_tf32(x);
}

template <uint32_t FMT>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (FMT == tc::kFmtBF16) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
  } else {
    const uint32_t lo = __half_as_ushort(__float2half_rn(a));
    const uint32_t hi = __half_as_ushort(__float2half_rn(b));
    return lo | (hi << 16);
  }
}

// Loads X[r][c] of a rows x cols matrix with leading dimension ld, 0 outside it.
__device__ __forceinline__ float ld_or_zero(const float* X, int64_t rows, int64_t cols,
                                            int64_t ld, int64_t r, int64_t c) {
  return (r < rows && c < cols) ? __ldg(X + r * ld + c) : 0.0f;
}

// One CTA per used leaf block (the plan's needed-block list), one pass: each
// thread owns UNITS / kThreads 16-byte pieces of the image (unit u = image
// row u / PPR, piece u % PPR; consecutive threads take consecutive pieces, so
// a warp's stores cover whole 128-byte rows), loads their source values into
// registers (all loads of a thread issued before any use), the CTA reduces the
// block's largest magnitude, then every thread scales, rounds and stores.
// A B block's image is its transpose: when the block is whole and its rows are
// 16-byte aligned, the CTA first copies it row by row (float4, coalesced) into
// shared memory with one float of padding per row and the threads gather their
// image pieces from there (a column read straight from global memory touches
// one cache line per lane: 0.22 -> 0.17 ms on the near-sparse N = 8192 leaf-128
// rounding); other B blocks are read by columns (for them the staging was
// slower).  Threads per CTA: 256 at leaf 64, 512 at leaf 128 (32 values per
// thread at most).
template <int LEAF>
constexpr int q_threads() { return LEAF == 128 ? 512 : 256; }
// Resident CTAs per SM the register allocation is held to: the rounding is
// bound by the HBM reads in flight.  Leaf 64: eight CTAs beat six (batch
// rounding 0.96 -> 0.85 ms).  Leaf 128: two CTAs (64 registers); one CTA
// (up to 128 registers) measured 2.79 -> 4.0 ms at N = 32768 and three spill
// (3.42 ms).  TF32 images hold twice the pieces.
template <uint32_t FMT, int LEAF>
constexpr int q_min_blocks() {
  return LEAF == 128 ? 2 : (FMT == tc::kFmtTF32 ? 6 : 8);
}

template <uint32_t FMT, int LEAF, bool SPLIT>
__global__ void __launch_bounds__(q_threads<LEAF>(), (q_min_blocks<FMT, LEAF>()))
    quantize_kernel(InstRef R, PlanBuffers Bf, OperandImages img) {
  constexpr int kThreads = q_threads<LEAF>();
  using L = TcLayout<FMT, LEAF>;
  constexpr int KC = L::kKc;                 // K elements per 128-byte chunk row
  constexpr int PER16 = 16 / L::kElt;        // elements per 16-byte piece
  constexpr int PPR = LEAF / PER16;          // pieces per image row
  constexpr int UNITS = LEAF * PPR;          // pieces per block image
  constexpr int U = UNITS / kThreads;        // pieces per thread
  static_assert(UNITS % kThreads == 0, "whole pieces per thread");
  __shared__ float s_max[kThreads / 32];
  extern __shared__ float s_blk[];   // [LEAF][LEAF + 1]: one B block, row-major
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = Bf.bdev->need_count;
  const float lo_scale = (float)(1 << L::kLoShift);

  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const uint32_t ent = Bf.need_list[idx];
    const bool isB = (ent >> 31) != 0;
    const int64_t blk = (int64_t)(ent & 0x7fffffffu);   // global block number of A or of B
    const Inst& in = R.at(isB ? inst_of_bblk(R, blk) : inst_of_ablk(R, blk));
    // A block (I, K): rows of A, K along its columns; B block (K, J): K along its rows
    const int64_t lb = blk - (isB ? in.bblk0 : in.ablk0);
    const int64_t gcols = isB ? in.bn : in.bk;                 // blocks per row of the grid
    const int64_t rows = isB ? in.kd : in.m, cols = isB ? in.n : in.kd;
    const int64_t ld = isB ? in.ldb : in.lda;                  // leading dimension
    const float* __restrict__ X = isB ? in.B : in.A;
    const int64_t r0 = (lb / gcols) * LEAF, c0 = (lb % gcols) * LEAF;
    const bool full = r0 + LEAF <= rows && c0 + LEAF <= cols;
    const bool vec = full && (ld & 3) == 0;

    if (isB && vec) {   // stage the block row-major (float4, coalesced), then read it
                        // transposed; the previous block's pieces were read before the
                        // loop's closing barrier
      constexpr int F4 = LEAF / 4;   // float4 per block row
      for (int t = tid; t < LEAF * F4; t += kThreads) {
        const int rr = t / F4, c4 = t - rr * F4;
        const float4 v = __ldg(reinterpret_cast<const float4*>(X + (r0 + rr) * ld + c0) + c4);
        float* d = s_blk + rr * (LEAF + 1) + 4 * c4;
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
      }
      __syncthreads();
    }
    float x[U][PER16];
#pragma unroll
    for (int r = 0; r < U; ++r) {
      const int u = tid + r * kThreads;
      const int row = u / PPR, k0 = (u % PPR) * PER16;
      if (!isB) {   // image row = block row, K along the block's columns
        const float* src = X + (r0 + row) * ld + c0 + k0;
        if (vec) {
#pragma unroll
          for (int q = 0; q < PER16; q += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src + q));
            x[r][q] = v.x; x[r][q + 1] = v.y; x[r][q + 2] = v.z; x[r][q + 3] = v.w;
          }
        } else if (full) {
#pragma unroll
          for (int q = 0; q < PER16; ++q) x[r][q] = __ldg(src + q);
        } else {
#pragma unroll
          for (int q = 0; q < PER16; ++q) x[r][q] = ld_or_zero(X, rows, cols, ld, r0 + row, c0 + k0 + q);
        }
      } else if (vec) {   // image row = block column, K along the block's rows (staged)
#pragma unroll
        for (int q = 0; q < PER16; ++q) x[r][q] = s_blk[(k0 + q) * (LEAF + 1) + row];
      } else if (full) {
#pragma unroll
        for (int q = 0; q < PER16; ++q) x[r][q] = __ldg(X + (r0 + k0 + q) * ld + c0 + row);
      } else {
#pragma unroll
        for (int q = 0; q < PER16; ++q) x[r][q] = ld_or_zero(X, rows, cols, ld, r0 + k0 + q, c0 + row);
      }
    }
    // largest magnitude of the block (NaN ignored, as fmaxf does)
    float mx = 0.0f;
#pragma unroll
    for (int r = 0; r < U; ++r)
#pragma unroll
      for (int q = 0; q < PER16; ++q) mx = fmaxf(mx, fabsf(x[r][q]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) s_max[warp] = mx;
    __syncthreads();
    mx = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, s_max[w]);
    int ex = 0;
    if (mx > 0.0f && mx <= 3.402823466e38f) frexpf(mx, &ex);
    // BF16 and TF32 have FP32's exponent range: the scaling only has to keep
    // products and sums inside it, so e is rounded up to a multiple of 32
    // (scaled maximum in [2^-33, 1)).  The roundings are those of the exact
    // exponent for every entry above 2^-94 of the block's maximum (hi parts)
    // and above 2^-80 (lo parts of the split modes), and
    // the blocks of a tile mostly share one exponent sum: the multiply's runs
    // (one accumulator pass per change of the sum) stay long.  FP16 keeps the
    // exact exponent: its range is the constraint.
    if constexpr (FMT != tc::kFmtF16) ex = ((ex + 31) >> 5) << 5;
    if (tid == 0) (isB ? img.eb : img.ea)[blk] = ex;
    // 2^-ex as a float when it is a normal number (the usual case), else ldexpf
    const bool pow2_ok = ex >= -126 && ex <= 126;
    const float scale = pow2_ok ? __int_as_float((127 - ex) << 23) : 1.0f;

    uint8_t* hi_img = (isB ? img.b_hi : img.a_hi) + blk * (int64_t)L::kBlockBytes;
    uint8_t* lo_img = SPLIT ? (isB ? img.b_lo : img.a_lo) + blk * (int64_t)L::kBlockBytes : nullptr;
#pragma unroll
    for (int r = 0; r < U; ++r) {
      const int u = tid + r * kThreads;
      const int row = u / PPR, k0 = (u % PPR) * PER16;
      float hv[PER16], lv[PER16];
#pragma unroll
      for (int q = 0; q < PER16; ++q) {
        const float sc = pow2_ok ? __fmul_rn(x[r][q], scale) : ldexpf(x[r][q], -ex);
        const float h = round_op<FMT>(sc);
        hv[q] = h;
        if constexpr (SPLIT) lv[q] = round_op<FMT>(__fmul_rn(__fsub_rn(sc, h), lo_scale));
      }
      uint4 ph, pl;
      if constexpr (FMT == tc::kFmtTF32) {
        ph = make_uint4(__float_as_uint(hv[0]), __float_as_uint(hv[1]), __float_as_uint(hv[2]),
                        __float_as_uint(hv[3]));
        if constexpr (SPLIT)
          pl = make_uint4(__float_as_uint(lv[0]), __float_as_uint(lv[1]), __float_as_uint(lv[2]),
                          __float_as_uint(lv[3]));
      } else {
        ph = make_uint4(pack2<FMT>(hv[0], hv[1]), pack2<FMT>(hv[2], hv[3]),
                        pack2<FMT>(hv[4], hv[5]), pack2<FMT>(hv[6], hv[7]));
        if constexpr (SPLIT)
          pl = make_uint4(pack2<FMT>(lv[0], lv[1]), pack2<FMT>(lv[2], lv[3]),
                          pack2<FMT>(lv[4], lv[5]), pack2<FMT>(lv[6], lv[7]));
      }
      const uint32_t off = (uint32_t)(k0 / KC) * (LEAF * 128) + tc::sw128_offset(row, (k0 % KC) / PER16);
      *reinterpret_cast<uint4*>(hi_img + off) = ph;
      if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo_img + off) = pl;
    }
    __syncthreads();   // s_max and s_blk are rewritten for the next block
  }
}

template <uint32_t FMT, int LEAF, bool SPLIT>
cudaError_t launch_q(const InstRef& ref, const PlanBuffers& b, const OperandImages& img,
                     cudaStream_t s) {
  constexpr size_t kBlkSmem = (size_t)LEAF * (LEAF + 1) * sizeof(float);
  static int wave[64] = {};   // resident CTAs per device (occupancy x SMs)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (wave[dev] == 0) {
    int sms = 0, per_sm = 0;
    e = cudaFuncSetAttribute(quantize_kernel<FMT, LEAF, SPLIT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlkSmem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, quantize_kernel<FMT, LEAF, SPLIT>,
                                                        q_threads<LEAF>(), kBlkSmem);
    if (e != cudaSuccess) return e;
    wave[dev] = sms * std::max(1, per_sm);
  }
  // the list length is known on the device only: one full wave of CTAs
  const int64_t cap = b.ablks + b.bblks;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cap, (int64_t)wave[dev]));
  return launch_pdl(quantize_kernel<FMT, LEAF, SPLIT>, dim3(grid), dim3(q_threads<LEAF>()),
                    kBlkSmem, s, ref, b, img);
}

}  // namespace

cudaError_t launch_quantize(spamm_precision_t prec, int leaf, const InstRef& ref,
                            const PlanBuffers& b, const OperandImages& img, cudaStream_t s) {
  const bool l64 = leaf == 64;
  switch (prec) {
    case SPAMM_BF16:
      return l64 ? launch_q<tc::kFmtBF16, 64, false>(ref, b, img, s)
                 : launch_q<tc::kFmtBF16, 128, false>(ref, b, img, s);
    case SPAMM_FP16:
      return l64 ? launch_q<tc::kFmtF16, 64, false>(ref, b, img, s)
                 : launch_q<tc::kFmtF16, 128, false>(ref, b, img, s);
    case SPAMM_BF16_SPLIT:
      return l64 ? launch_q<tc::kFmtBF16, 64, true>(ref, b, img, s)
                 : launch_q<tc::kFmtBF16, 128, true>(ref, b, img, s);
    case SPAMM_FP16_SPLIT:
      return l64 ? launch_q<tc::kFmtF16, 64, true>(ref, b, img, s)
                 : launch_q<tc::kFmtF16, 128, true>(ref, b, img, s);
    case SPAMM_TF32X3:
      return l64 ? launch_q<tc::kFmtTF32, 64, true>(ref, b, img, s)
                 : launch_q<tc::kFmtTF32, 128, true>(ref, b, img, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spamm
