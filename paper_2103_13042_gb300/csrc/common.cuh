// Shared device/host helpers of the SpAMM library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spamm.h"

#define SPAMM_CUDA_TRY(call)                                   \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return SPAMM_ERR_CUDA;              \
  } while (0)

#define SPAMM_LAUNCH_CHECK()                                   \
  do {                                                         \
    if (cudaPeekAtLastError() != cudaSuccess) {                \
      (void)cudaGetLastError();                                \
      return SPAMM_ERR_CUDA;                                   \
    }                                                          \
  } while (0)

namespace spamm {

constexpr int kMaxBd = 1024;          // k indices are stored in 10 bits of a uint16
constexpr uint16_t kSplitFlag = 0x8000;
constexpr int kFlagBinMin = -200;     // relative products below 2^-200 share one bin
constexpr int kFlagBins = 202;        // bins -200 .. 1

inline int64_t num_blocks(int64_t n, int32_t leaf) { return (n + leaf - 1) / leaf; }

// Device status word of the current device (defined in api.cu).
int32_t* device_status_word();

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel of the plan -> rounding -> multiply
// chain is launched while its predecessor in the stream still runs (its CTAs
// are placed and set up early); it calls pdl_wait() before anything else, which
// returns once the predecessor grid has completed and its writes are visible.
// Every kernel so launched waits unconditionally at its top, so completion
// stays transitive along the chain.  pdl_trigger() lets the successor launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, FMA-based TwoProd) in FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (hi, lo) += x^2 with x^2 split exactly and the pair renormalised afterwards.
// Relative error of each step <= 2u^2 for non-negative terms (u = 2^-24).
__device__ __forceinline__ void dw_add_square(float x, float& hi, float& lo) {
  float p = __fmul_rn(x, x);
  float pe = __fmaf_rn(x, x, -p);
  float s, e;
  two_sum(hi, p, s, e);
  float t = __fadd_rn(lo, __fadd_rn(e, pe));
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// ---------------------------------------------------------------------------
// Sum of squares with a moving power-of-two scale: value = (hi + lo) * 4^e.
// Squares of FP32 entries below 2^-63 underflow in FP32, so every group of
// entries is first scaled by 2^-g (g = exponent of the group's largest
// magnitude; exact), squared exactly, and merged into the running pair after
// aligning the two scales.  Contributions smaller than 2^-90 of the running
// sum are dropped (far below the 2^-43 accuracy target).
// ---------------------------------------------------------------------------
constexpr int kSumSqEmpty = -100000;

struct SumSq {
  float hi, lo;
  int e;
};

__device__ __forceinline__ SumSq sumsq_empty() { return SumSq{0.0f, 0.0f, kSumSqEmpty}; }

// 2^k as a normal FP32 for -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// Scale exponent of a group from its largest magnitude (NaN ignored, Inf kept).
__device__ __forceinline__ int group_exponent(float max_abs) {
  const int ef = (int)((__float_as_uint(max_abs) >> 23) & 0xffu);
  const int g = ef - 127;                 // max_abs in [2^g, 2^(g+1)); -127 when subnormal
  return g > 126 ? 126 : g;
}

// acc += (hi + lo) * 4^g.
__device__ __forceinline__ void sumsq_merge(SumSq& acc, float hi, float lo, int g) {
  if (!(hi != 0.0f || lo != 0.0f)) {
    if (hi != hi || lo != lo) acc.hi = hi + lo;  // keep NaN
    return;
  }
  if (acc.e == kSumSqEmpty) {
    acc.hi = hi;
    acc.lo = lo;
    acc.e = g;
    return;
  }
  int d = acc.e - g;
  if (d < 0) {  // the group dominates: rescale the accumulator
    if (-2 * d > 90) {
      acc.hi = hi;
      acc.lo = lo;
      acc.e = g;
      return;
    }
    const float f = pow2f(2 * d);
    acc.hi *= f;
    acc.lo *= f;
    acc.e = g;
  } else if (d > 0) {
    if (2 * d > 90) return;
    const float f = pow2f(-2 * d);
    hi *= f;
    lo *= f;
  }
  float s, e;
  two_sum(acc.hi, hi, s, e);
  const float t = __fadd_rn(__fadd_rn(acc.lo, lo), e);
  acc.hi = __fadd_rn(s, t);
  acc.lo = __fsub_rn(t, __fsub_rn(acc.hi, s));
}

// acc += a partner's sum (hi, lo) * 4^e that may be empty (e == kSumSqEmpty;
// a NaN there still propagates).
__device__ __forceinline__ void sumsq_merge_any(SumSq& acc, float h, float l, int e) {
  if (e == kSumSqEmpty) {
    if (h != h) acc.hi = h;
  } else {
    sumsq_merge(acc, h, l, e);
  }
}

// Exact-squares sum of one group of N entries into acc.
//
// The running pair starts at B = 2 fl((scaled max)^2), so every square p
// satisfies p < hi (also after a renormalisation, which moves hi by far less
// than B / 2) and Fast2Sum gives the exact error of hi + p in 3 operations;
// the errors and the low halves of the squares go into lo, and (hi, lo) is
// renormalised every 8 entries.  B is removed with one TwoSum at the end.
// Every group is scaled (its largest magnitude to [1, 2)), so a group's pair
// lies in [1, 34) of its unit 4^g and an accumulator's hi stays within a few
// binades of its unit: sumsq_merge's exponent test then drops only terms far
// below 2^-43 of the sum.  (Leaving groups of moderate magnitude unscaled would
// break that: an unscaled pair may be as small as 2^-60, and a scaled group
// 2^-98 below its unit would be dropped at a relative size of 2^-38.)
template <int N>
__device__ __forceinline__ void sumsq_group(SumSq& acc, const float (&v)[N]) {
  float mx = 0.0f;
#pragma unroll
  for (int q = 0; q < N; ++q) mx = fmaxf(mx, fabsf(v[q]));
  if (mx == 0.0f) {
    bool nan = false;
#pragma unroll
    for (int q = 0; q < N; ++q) nan |= (v[q] != v[q]);
    if (nan) {
      acc.hi = __int_as_float(0x7fffffff);
      acc.e = 0;
    }
    return;
  }
  const int g = group_exponent(mx);
  const float sc = pow2f(-g);
  const float ms = __fmul_rn(mx, sc);
  const float pB = 2.0f * __fmul_rn(ms, ms);   // the starting value B (a float)
  float hi = pB, lo = 0.0f;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const float x = __fmul_rn(v[q], sc);
    const float p = __fmul_rn(x, x);
    const float pe = __fmaf_rn(x, x, -p);
    const float s = __fadd_rn(hi, p);
    const float e = __fsub_rn(p, __fsub_rn(s, hi));   // exact: hi >= p
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
    if ((q & 7) == 7) {   // renormalise: |hi| >= |lo|
      const float t = __fadd_rn(hi, lo);
      lo = __fsub_rn(lo, __fsub_rn(t, hi));
      hi = t;
    }
  }
  // remove the starting value B
  float s, e;
  two_sum(hi, -pB, s, e);
  lo = __fadd_rn(lo, e);
  hi = __fadd_rn(s, lo);
  lo = __fsub_rn(lo, __fsub_rn(hi, s));
  sumsq_merge(acc, hi, lo, g);
}

// sqrt of the accumulated value, returned in FP64, with FP32 arithmetic and
// three FP64 instructions (the FP64 pipe is narrow on this part).  With
// S = (hi + lo) 4^e: r0 = sqrtf(hi); one Newton step on the exact residual
// hi + lo - r0^2 (r0^2 split exactly by FMA) gives r0 + c within ~2^-47 of
// sqrt(hi + lo); the result is (r0 + c) 2^e, converted and added in FP64.
__device__ __forceinline__ double sumsq_sqrt(const SumSq& a) {
  if (a.e == kSumSqEmpty) return (double)a.hi;   // 0, or NaN
  const float hi = a.hi, lo = a.lo;
  if (!(hi > 0.0f) || !(hi <= 3.402823466e38f)) return sqrt(ldexp((double)hi + (double)lo, 2 * a.e));
  const float r0 = sqrtf(hi);
  const float sq = __fmul_rn(r0, r0);
  const float sq_e = __fmaf_rn(r0, r0, -sq);            // r0^2 = sq + sq_e exactly
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(hi, sq), sq_e), lo);
  const float c = __fdiv_rn(d, __fmul_rn(2.0f, r0));
  const double r = (double)r0 + (double)c;               // the FP64 work
  // scale by 2^e on the bit pattern (the result stays a normal double)
  return __longlong_as_double(__double_as_longlong(r) + ((long long)a.e << 52));
}

// The accumulated value in FP64.
__device__ __forceinline__ double sumsq_value(const SumSq& a) {
  if (a.e == kSumSqEmpty) return (double)a.hi;   // 0, or NaN
  return ldexp((double)a.hi + (double)a.lo, 2 * a.e);
}

// ---------------------------------------------------------------------------
// Mantissa/exponent form of a non-negative FP64 value for the FP32 pre-screen:
//   x = m * 2^e, m in [0.5, 1] rounded to FP32.  kind: 0 finite > 0, 1 zero,
//   2 non-finite (Inf or NaN).
// ---------------------------------------------------------------------------
struct Screen {
  float m;
  int32_t e;
};

constexpr int32_t kZeroExp = -100000;      // zero: never survives a positive tau
constexpr int32_t kNonFiniteExp = 100000;  // Inf/NaN: always survives

__device__ __forceinline__ Screen make_screen(double x) {
  Screen s;
  if (!(x == x) || isinf(x)) {
    s.m = 1.0f;
    s.e = kNonFiniteExp;
  } else if (x == 0.0) {
    s.m = 0.0f;
    s.e = kZeroExp;
  } else {
    int e;
    double m = frexp(x, &e);
    s.m = __double2float_rn(m);  // in [0.5, 1]
    s.e = e;
  }
  return s;
}

}  // namespace spamm
