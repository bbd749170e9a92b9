// Error measures (Eq. 5): ||X - Y||_F (or ||X||_F) with FP64-grade accuracy.
//
// Each difference d = x - y is formed in FP32 and its rounding error dl kept
// (TwoSum); groups of 32 differences are scaled by a power of two, squared
// exactly with FMA and accumulated as a scaled FP32 pair (plus the 2 d dl
// cross terms), so tiny differences do not underflow and FP64 (1/72 of the
// FP32 rate here) is used once per thread.
// A grid-stride pass writes one FP64 partial per CTA; a one-CTA pass adds them.
#include "plan.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
    diff_partial_kernel(const float* __restrict__ X, const float* __restrict__ Y, int64_t count,
                        double* __restrict__ partials) {
  SumSq ss = sumsq_empty();
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  while (e < count) {
    float d[32], dl[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int64_t idx = e + (int64_t)q * stride;
      d[q] = 0.f;
      dl[q] = 0.f;
      if (idx < count) {
        const float x = __ldcs(X + idx);
        if (Y != nullptr) two_sum(x, -__ldcs(Y + idx), d[q], dl[q]);
        else d[q] = x;
      }
    }
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) mx = fmaxf(mx, fabsf(d[q]));
    if (mx != 0.f) {
      const int g = group_exponent(mx);
      const float sc = pow2f(-g);
      float hi = 0.f, lo = 0.f, cross = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float ds = __fmul_rn(d[q], sc);
        dw_add_square(ds, hi, lo);
        cross = __fmaf_rn(2.0f * ds, __fmul_rn(dl[q], sc), cross);
      }
      sumsq_merge(ss, hi, __fadd_rn(lo, cross), g);
    } else {
      bool nan = false;
#pragma unroll
      for (int q = 0; q < 32; ++q) nan |= (d[q] != d[q]);
      if (nan) {
        ss.hi = __int_as_float(0x7fffffff);
        ss.e = 0;
      }
    }
    e += 32 * stride;
  }
  double acc = sumsq_value(ss);
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double ws[kThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += ws[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void sum_sqrt_kernel(const double* __restrict__ partials, int nparts,
                                double* __restrict__ out) {
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) a += partials[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(s[0]);
}

}  // namespace

cudaError_t launch_frobenius_diff(const float* X, const float* Y, int64_t count, double* partials,
                                  int nparts, double* out, cudaStream_t s) {
  diff_partial_kernel<<<nparts, kThreads, 0, s>>>(X, Y, count, partials);
  sum_sqrt_kernel<<<1, kThreads, 0, s>>>(partials, nparts, out);
  return cudaPeekAtLastError();
}

}  // namespace spamm
