// Peak-rate microkernels: the denominators of the roofline fractions that a
// library GEMM cannot provide.  FP32 FFMA and FP64 DFMA issue rates of the
// SIMT cores (independent FMA chains in every thread of a full grid), and
// tcgen05 MMA rates of one CTA per SM whose single issuing thread sends
// back-to-back 128 x N x K MMAs (BF16 or FP16 operands with kind::f16, TF32
// with kind::tf32, FP32 accumulators in tensor memory) on operands resident in
// shared memory, so neither memory nor the epilogue limits the rate.  The
// paper has no counterpart: it quotes no hardware rates.
#include <vector>

#include "plan.cuh"
#include "tc.cuh"

namespace spamm {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_peak_kernel(float x, float y, int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = (float)(threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = __fmaf_rn(a[q], x, y);
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 1234.5678f) sink[0] = s;   // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(256) dfma_peak_kernel(double x, double y, int iters,
                                                        double* sink) {
  double a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = (double)(threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = __fma_rn(a[q], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 1234.5678) sink[0] = s;
}

// One CTA per SM, 128 threads.  Shared memory: the A image (128 rows of 128
// bytes) and the B image (N rows), zeroed, 1024-byte aligned; a completion
// barrier.  ok[blockIdx.x] = 1 when the issued MMAs completed within the limit.
template <uint32_t FMT, int N>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int iters, int* ok) {
  constexpr int M = 128;
  constexpr uint32_t kIdesc = tc::idesc(FMT, M, N);
  constexpr uint32_t kABytes = M * 128, kBBytes = N * 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + kABytes + kBBytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(done + 1);
  for (uint32_t i = threadIdx.x; i < (kABytes + kBBytes) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    tc::mbar_init(done, 1);
    tc::fence_mbarrier_init();
  }
  const int warp = threadIdx.x / 32;
  if (warp == 0) {
    tc::tmem_alloc(slot, (uint32_t)N);
    tc::tmem_relinquish();
  }
  // the zeroed operands are read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  if (threadIdx.x == 0) {
    const uint64_t da = tc::sdesc_k_sw128(tc::smem_u32(smem));
    const uint64_t db = tc::sdesc_k_sw128(tc::smem_u32(smem + kABytes));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {   // four 32-byte K steps of the 128-byte rows
        if constexpr (FMT == tc::kFmtTF32) tc::mma_tf32(tmem, da + 2u * ks, db + 2u * ks, kIdesc, 1u);
        else tc::mma_f16(tmem, da + 2u * ks, db + 2u * ks, kIdesc, 1u);
      }
    }
    tc::mma_commit(done);
    ok[blockIdx.x] = tc::mbar_wait(done, 0u, 2000000000ull) ? 1 : 0;   // 2 s at most
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)N);
  }
}

template <uint32_t FMT, int N>
cudaError_t launch_mma_peak(int sms, int iters, int* ok, cudaStream_t s) {
  // more than half of an SM's shared memory: one CTA per SM
  const size_t need = 128 * 128 + N * 128 + 64 + 1024;
  const size_t smem = need > 120 * 1024 ? need : 120 * 1024;
  cudaError_t e = cudaFuncSetAttribute(mma_peak_kernel<FMT, N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mma_peak_kernel<FMT, N><<<sms, 128, smem, s>>>(iters, ok);
  return cudaPeekAtLastError();
}

}  // namespace
}  // namespace spamm

using namespace spamm;

extern "C" spamm_status_t spamm_peak_rates(double* tflops, void* stream) {
  if (!tflops) return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  SPAMM_CUDA_TRY(cudaGetDevice(&dev));
  SPAMM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, (size_t)sms * sizeof(int) + 64) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_NO_MEMORY;
  }
  int* ok = static_cast<int*>(scratch);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  spamm_status_t st = SPAMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SPAMM_ERR_CUDA;
  // times one launch (after one untimed launch of the same work); ms out
  auto timed = [&](auto launch, float* ms) -> bool {
    if (launch() != cudaSuccess) return false;
    if (cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return false;
    return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
  };
  const int simt_blocks = sms * 8, simt_iters = 1 << 16;
  const double simt_flops = 2.0 * kChains * (double)simt_iters * simt_blocks * 256;
  float ms = 0.0f;
  // [0] FP32 FFMA, [1] FP64 DFMA
  if (st == SPAMM_OK) {
    float* sink = reinterpret_cast<float*>(ok + sms);
    if (!timed([&] {
          ffma_peak_kernel<<<simt_blocks, 256, 0, s>>>(1.0000001f, 1e-7f, simt_iters, sink);
          return cudaPeekAtLastError();
        }, &ms))
      st = SPAMM_ERR_CUDA;
    else
      tflops[0] = simt_flops / (ms * 1e-3) / 1e12;
  }
  if (st == SPAMM_OK) {
    double* sink = reinterpret_cast<double*>(reinterpret_cast<char*>(ok + sms) + 16);
    if (!timed([&] {
          dfma_peak_kernel<<<simt_blocks, 256, 0, s>>>(1.0000001, 1e-7, simt_iters / 16, sink);
          return cudaPeekAtLastError();
        }, &ms))
      st = SPAMM_ERR_CUDA;
    else
      tflops[1] = simt_flops / 16.0 / (ms * 1e-3) / 1e12;
  }
  // [2] BF16, [3] FP16 (kind::f16, K = 16 per MMA), [4] TF32 (kind::tf32, K = 8), each the
  // better of N = 128 and N = 256
  const int mma_iters = 8192;
  struct Case { int idx; int fmt; int n; double k; };
  const Case cases[] = {{2, (int)tc::kFmtBF16, 128, 16}, {2, (int)tc::kFmtBF16, 256, 16},
                        {3, (int)tc::kFmtF16, 128, 16},  {3, (int)tc::kFmtF16, 256, 16},
                        {4, (int)tc::kFmtTF32, 128, 8},  {4, (int)tc::kFmtTF32, 256, 8}};
  for (int q = 2; q < 5; ++q) tflops[q] = 0.0;
  for (const Case& c : cases) {
    if (st != SPAMM_OK) break;
    auto launch = [&]() -> cudaError_t {
      if (c.fmt == (int)tc::kFmtBF16)
        return c.n == 128 ? launch_mma_peak<tc::kFmtBF16, 128>(sms, mma_iters, ok, s)
                          : launch_mma_peak<tc::kFmtBF16, 256>(sms, mma_iters, ok, s);
      if (c.fmt == (int)tc::kFmtF16)
        return c.n == 128 ? launch_mma_peak<tc::kFmtF16, 128>(sms, mma_iters, ok, s)
                          : launch_mma_peak<tc::kFmtF16, 256>(sms, mma_iters, ok, s);
      return c.n == 128 ? launch_mma_peak<tc::kFmtTF32, 128>(sms, mma_iters, ok, s)
                        : launch_mma_peak<tc::kFmtTF32, 256>(sms, mma_iters, ok, s);
    };
    if (!timed(launch, &ms)) {
      st = SPAMM_ERR_CUDA;
      break;
    }
    std::vector<int> h((size_t)sms);
    if (cudaMemcpy(h.data(), ok, (size_t)sms * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = SPAMM_ERR_CUDA;
      break;
    }
    for (int v : h)
      if (v != 1) st = SPAMM_ERR_TIMEOUT;
    const double flops = 2.0 * 128.0 * c.n * c.k * 4.0 * mma_iters * sms;
    const double r = flops / (ms * 1e-3) / 1e12;
    if (r > tflops[c.idx]) tflops[c.idx] = r;
  }
  if (st == SPAMM_ERR_CUDA) (void)cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  return st;
}
