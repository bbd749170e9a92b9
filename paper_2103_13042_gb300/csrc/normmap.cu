// Get-norm step (Section 3.2, Eq. 2): normmap[I*bd+K] = ||X[I,K]||_F.
//
// GB300 design.  A single streaming pass over X: a CTA covers one block-row
// strip (leaf rows) and a window of columns; each thread owns a fixed column
// slot (a float4 when n % 4 == 0, else one float) and walks the strip's rows,
// so every warp load is a contiguous row segment (512 or 128 bytes), loads
// are streamed (evict-first) and eight rows of loads are in flight per group.
// FP64 arithmetic runs at 1/72 of the FP32 rate on this part, so every group
// of 32 entries is scaled by a power of two (no FP32 underflow of tiny
// squares), squared exactly with FMA and accumulated as an unevaluated FP32
// pair with an explicit scale exponent; the threads of a block column are
// combined in that FP32 form (warp shuffles, and shared memory when a block
// column spans several warps), and the square root is taken with an FP32
// Newton step on the exact residual, so a block costs three FP64
// instructions.
#include "plan.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void merge_from(SumSq& a, float h, float l, int e) {
  if (e == kSumSqEmpty) {
    if (h != h) a.hi = h;   // NaN from an otherwise empty partner
  } else {
    sumsq_merge(a, h, l, e);
  }
}

// One CTA: block row I, column window wx of X (kThreads * VEC columns).
template <int VEC, int LEAF>
__device__ __forceinline__ void norm_strip(const float* __restrict__ X, int64_t n, int bd,
                                           double* __restrict__ out, int I, int64_t wx) {
  constexpr int kCols = kThreads * VEC;               // columns per CTA window
  constexpr int kThreadsPerBlockCol = LEAF / VEC;     // threads sharing one output
  constexpr int kRowsPerGroup = 32 / VEC;             // rows per 32-entry group
  const int64_t col0 = wx * kCols + (int64_t)threadIdx.x * VEC;
  const int64_t row0 = (int64_t)I * LEAF;
  const int64_t row1 = (n < row0 + LEAF) ? n : row0 + LEAF;
  const bool active = col0 < n;

  SumSq ss = sumsq_empty();
  if (active) {
    const float* p = X + row0 * n + col0;
    for (int64_t r = row0; r < row1; r += kRowsPerGroup) {
      const int rows = (int)((row1 - r) < kRowsPerGroup ? (row1 - r) : kRowsPerGroup);
      float v[32];
#pragma unroll
      for (int q = 0; q < kRowsPerGroup; ++q) {
        if (q < rows) {
          if constexpr (VEC == 4) {
            const float4 t = __ldcs(reinterpret_cast<const float4*>(p + (int64_t)q * n));
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
          } else {
            v[q] = __ldcs(p + (int64_t)q * n);
          }
        } else {
#pragma unroll
          for (int c = 0; c < VEC; ++c) v[VEC * q + c] = 0.0f;
        }
      }
      sumsq_group<32>(ss, v);
      p += (int64_t)kRowsPerGroup * n;
    }
  }

  // combine the threads of a block column in the FP32-pair form
  if constexpr (kThreadsPerBlockCol <= 32) {
#pragma unroll
    for (int off = kThreadsPerBlockCol / 2; off > 0; off >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
      const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
      const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
      merge_from(ss, h, l, e);
    }
    if ((threadIdx.x % kThreadsPerBlockCol) == 0 && active)
      out[(int64_t)I * bd + col0 / LEAF] = sumsq_sqrt(ss);
  } else {
    __shared__ SumSq warp_sum[kThreads / 32];
    ss = sumsq_warp_sum(ss);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x / 32] = ss;
    __syncthreads();
    constexpr int kWarpsPerBlockCol = kThreadsPerBlockCol / 32;
    if ((threadIdx.x % kThreadsPerBlockCol) == 0 && active) {
      SumSq s = warp_sum[threadIdx.x / 32];
#pragma unroll
      for (int w = 1; w < kWarpsPerBlockCol; ++w) {
        const SumSq o = warp_sum[threadIdx.x / 32 + w];
        merge_from(s, o.hi, o.lo, o.e);
      }
      out[(int64_t)I * bd + col0 / LEAF] = sumsq_sqrt(s);
    }
  }
}

template <int VEC, int LEAF>
__global__ void __launch_bounds__(kThreads, 4)
    normmap_kernel(const float* __restrict__ X, int64_t n, int bd, double* __restrict__ out) {
  norm_strip<VEC, LEAF>(X, n, bd, out, blockIdx.y, blockIdx.x);
}

// Batched form: one CTA per (job, block row, window); a job is one operand of
// one instance, aligned (float4) or not.
template <int LEAF>
__global__ void __launch_bounds__(kThreads)
    normmap_batched_kernel(const NormJob* __restrict__ jobs, int njobs) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].cta0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const NormJob jb = jobs[lo];
  const int64_t local = (int64_t)blockIdx.x - jb.cta0;
  const int64_t windows = (jb.n + kThreads * (jb.vec ? 4 : 1) - 1) / (kThreads * (jb.vec ? 4 : 1));
  const int I = (int)(local / windows);
  const int64_t wx = local % windows;
  if (jb.vec) norm_strip<4, LEAF>(jb.X, jb.n, jb.bd, jb.out, I, wx);
  else norm_strip<1, LEAF>(jb.X, jb.n, jb.bd, jb.out, I, wx);
}

template <int VEC, int LEAF>
cudaError_t launch(const float* X, int64_t n, int bd, double* out, cudaStream_t s) {
  constexpr int kCols = kThreads * VEC;
  dim3 grid((unsigned)((n + kCols - 1) / kCols), (unsigned)bd);
  normmap_kernel<VEC, LEAF><<<grid, kThreads, 0, s>>>(X, n, bd, out);
  return cudaPeekAtLastError();
}

}  // namespace

cudaError_t launch_normmap(const float* X, int64_t n, int32_t leaf, double* out,
                           cudaStream_t s) {
  const int bd = (int)num_blocks(n, leaf);
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  switch (leaf) {
    case 32: return vec ? launch<4, 32>(X, n, bd, out, s) : launch<1, 32>(X, n, bd, out, s);
    case 64: return vec ? launch<4, 64>(X, n, bd, out, s) : launch<1, 64>(X, n, bd, out, s);
    case 128: return vec ? launch<4, 128>(X, n, bd, out, s) : launch<1, 128>(X, n, bd, out, s);
    default: return cudaErrorInvalidValue;
  }
}

int normjob_ctas(const NormJob& j) {
  const int64_t cols = kThreads * (j.vec ? 4 : 1);
  return (int)(((j.n + cols - 1) / cols) * j.bd);
}

cudaError_t launch_normmap_jobs(const NormJob* dev_jobs, int njobs, int total_ctas, int leaf,
                                cudaStream_t s) {
  if (total_ctas <= 0) return cudaSuccess;
  switch (leaf) {
    case 32: normmap_batched_kernel<32><<<total_ctas, kThreads, 0, s>>>(dev_jobs, njobs); break;
    case 64: normmap_batched_kernel<64><<<total_ctas, kThreads, 0, s>>>(dev_jobs, njobs); break;
    case 128: normmap_batched_kernel<128><<<total_ctas, kThreads, 0, s>>>(dev_jobs, njobs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaPeekAtLastError();
}

}  // namespace spamm
