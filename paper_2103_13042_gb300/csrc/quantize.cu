// Operand rounding for the tensor-core multiply (spec mixed precision on
// top of the paper's FP16 tensor-core kernel, Section 3.3 / Algorithm 3).
//
// For every leaf block that some surviving triple uses (the plan's need flags)
// one CTA stages the FP32 block in shared memory, finds e = frexp exponent of
// its largest magnitude, scales by 2^-e (exact), rounds to nearest-even in the
// operand format (hi) and, in split modes, rounds the exact residual scaled by
// 2^s_lo (lo).  The result is written directly as the K-major, 128-byte
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

constexpr int kThreads = 256;
constexpr int kChunk = 64;   // candidate blocks per need-flag scan (two warps)

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

template <uint32_t FMT, int LEAF, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
    quantize_kernel(InstRef R, PlanBuffers Bf, OperandImages img) {
  using L = TcLayout<FMT, LEAF>;
  constexpr int ELT = L::kElt, KC = L::kKc, NCH = L::kNch;
  constexpr int PER16 = 16 / ELT;                 // elements per 16-byte piece
  constexpr int UNITS = NCH * LEAF * 8;           // 16-byte pieces per block image
  extern __shared__ float tile[];                 // [LEAF][LEAF + 1]
  __shared__ float warp_max[kThreads / 32];
  __shared__ int s_list[kChunk];
  const int64_t tiles = Bf.tiles;      // global blocks of A (and of B)
  const uint8_t* __restrict__ needA = Bf.needA;
  const uint8_t* __restrict__ needB = Bf.needB;
  const float lo_scale = (float)(1 << L::kLoShift);

  // Candidates (A blocks, then B blocks) in chunks of kChunk: the first two
  // warps read one need flag each, thread 0 lists the needed ones in order,
  // then the CTA rounds them one block at a time.
  const int64_t nchunks = (2 * tiles + kChunk - 1) / kChunk;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    if (threadIdx.x < kChunk) {
      const int64_t cand = chunk * kChunk + threadIdx.x;
      bool need = false;
      if (cand < 2 * tiles) need = cand >= tiles ? needB[cand - tiles] != 0 : needA[cand] != 0;
      s_list[threadIdx.x] = need ? 1 : 0;
    }
    __syncthreads();
    // compact (kChunk entries; thread 0 is enough and keeps the order)
    __shared__ int s_total;
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int q = 0; q < kChunk; ++q)
        if (s_list[q]) s_list[tot++] = q;
      s_total = tot;
    }
    __syncthreads();
    const int total = s_total;
  for (int li = 0; li < total; ++li) {
    const int64_t w = chunk * kChunk + s_list[li];
    const bool isB = w >= tiles;
    const int64_t blk = isB ? w - tiles : w;      // global block number
    const Inst& in = R.at(inst_of_tile(R, blk));
    const int64_t n = in.n, lb = blk - in.tile0;
    const int bd = in.bd;
    const float* X = isB ? in.B : in.A;
    const int64_t r0 = (lb / bd) * LEAF, c0 = (lb % bd) * LEAF;

    // stage the block (zero outside the matrix) and its largest magnitude;
    // all loads are issued before the first shared-memory store
    constexpr int PER_T = LEAF * LEAF / kThreads;
    float vals[PER_T];
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int e = threadIdx.x + q * kThreads;
      const int64_t gr = r0 + e / LEAF, gc = c0 + e % LEAF;
      vals[q] = (gr < n && gc < n) ? __ldg(X + gr * n + gc) : 0.0f;
    }
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int e = threadIdx.x + q * kThreads;
      tile[(e / LEAF) * (LEAF + 1) + e % LEAF] = vals[q];
      mx = fmaxf(mx, fabsf(vals[q]));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x / 32] = mx;
    __syncthreads();
    mx = 0.0f;
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) mx = fmaxf(mx, warp_max[q]);
    int e = 0;
    if (mx > 0.0f && mx <= 3.402823466e38f) frexpf(mx, &e);
    if (threadIdx.x == 0) (isB ? img.eb : img.ea)[blk] = e;

    uint8_t* hi_img = (isB ? img.b_hi : img.a_hi) + blk * (int64_t)L::kBlockBytes;
    uint8_t* lo_img = SPLIT ? (isB ? img.b_lo : img.a_lo) + blk * (int64_t)L::kBlockBytes : nullptr;
    for (int u = threadIdx.x; u < UNITS; u += kThreads) {
      const int piece = u % 8, row = (u / 8) % LEAF, ch = u / (8 * LEAF);
      float hv[PER16], lv[PER16];
#pragma unroll
      for (int q = 0; q < PER16; ++q) {
        const int k = ch * KC + piece * PER16 + q;
        const float x = isB ? tile[k * (LEAF + 1) + row] : tile[row * (LEAF + 1) + k];
        const float s = ldexpf(x, -e);
        const float h = round_op<FMT>(s);
        hv[q] = h;
        if constexpr (SPLIT) lv[q] = round_op<FMT>(__fmul_rn(__fsub_rn(s, h), lo_scale));
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
      const uint32_t off = ch * (LEAF * 128) + tc::sw128_offset(row, piece);
      *reinterpret_cast<uint4*>(hi_img + off) = ph;
      if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo_img + off) = pl;
    }
    __syncthreads();   // the tile is reused by the next block
  }
    __syncthreads();   // s_list / s_total are rewritten by the next chunk
  }
}

template <uint32_t FMT, int LEAF, bool SPLIT>
cudaError_t launch_q(const InstRef& ref, const PlanBuffers& b, const OperandImages& img,
                     cudaStream_t s) {
  const size_t smem = (size_t)LEAF * (LEAF + 1) * sizeof(float);
  cudaFuncSetAttribute(quantize_kernel<FMT, LEAF, SPLIT>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, quantize_kernel<FMT, LEAF, SPLIT>,
                                                kThreads, smem);
  const int64_t chunks = (2 * b.tiles + kChunk - 1) / kChunk;
  const int grid =
      (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)sms * std::max(1, per_sm)));
  quantize_kernel<FMT, LEAF, SPLIT><<<grid, kThreads, smem, s>>>(ref, b, img);
  return cudaPeekAtLastError();
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
