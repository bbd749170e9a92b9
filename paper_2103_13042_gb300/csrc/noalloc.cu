// spamm_multiply_fp32_noalloc: a whole FP32 SpAMM call (norm maps, pair-test
// plan, SIMT multiply) that performs no device allocation.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// a product -- for example a library running under a host framework whose
// memory pool has already reserved the device memory, a plugin whose host
// forbids device allocations, or a latency-sensitive loop that cannot afford
// the implicit device-wide synchronisation a cudaMalloc/cudaFree may cause.
// Everything the call needs beyond A, B and C lives in the file-scope device
// array below, which every GPU that loads this library keeps until the
// process exits.
//
// Contract:
//  - The scratch holds the plan of at most kNoAllocMaxBd x kNoAllocMaxBd leaf
//    blocks (ceil(n / leaf) <= 64: n <= 2048 at leaf 32, 4096 at leaf 64,
//    8192 at leaf 128); larger problems are rejected with
//    SPAMM_ERR_UNSUPPORTED before anything is enqueued.
//  - The first call on a device looks the array's device address up with
//    cudaGetSymbolAddress (once per device, with that device current).  Make
//    that first call before any stream capture on the device.
//  - All calls on a device share the one array and it keeps whatever the last
//    call left there; each call rewrites every piece it reads and clears its
//    own accumulators.  Calls whose work overlaps on the GPU (two streams, or
//    two host threads) race on the array and give wrong results: serialise them.
#include <mutex>

#include "tc_common.cuh"

namespace spamm {
namespace {

constexpr int kNoAllocMaxBd = 64;
constexpr size_t kNoAllocBytes = size_t(1) << 20;   // 1 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace spamm

using namespace spamm;

extern "C" spamm_status_t spamm_multiply_fp32_noalloc(const float* A, const float* B, float* C,
                                                       int64_t n, int32_t leaf, double tau,
                                                       void* stream) {
  if (n < 1 || !A || !B || !C) return SPAMM_ERR_INVALID_ARG;
  if (leaf != 32 && leaf != 64 && leaf != 128) return SPAMM_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
       reinterpret_cast<uintptr_t>(C)) & 15u)
    return SPAMM_ERR_INVALID_ARG;
  if (A == C || B == C) return SPAMM_ERR_INVALID_ARG;
  if (tau != tau || tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  const int64_t bd64 = num_blocks(n, leaf);
  if (bd64 > kNoAllocMaxBd) return SPAMM_ERR_UNSUPPORTED;   // beyond the static scratch
  const int bd = (int)bd64;

  // scratch: [normA | normB | plan buffers]
  const size_t norm_bytes = round256((size_t)bd * bd * sizeof(double));
  Inst inst{};
  inst.n = n;
  inst.bd = bd;
  const size_t plan_bytes = plan_layout(&inst, 1, nullptr, nullptr);
  if (2 * norm_bytes + plan_bytes > kNoAllocBytes) return SPAMM_ERR_UNSUPPORTED;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  char* p = static_cast<char*>(base);
  double* nA = reinterpret_cast<double*>(p);
  double* nB = reinterpret_cast<double*>(p + norm_bytes);
  PlanBuffers buf{};
  plan_layout(&inst, 1, &buf, p + 2 * norm_bytes);
  inst.A = A;
  inst.B = B;
  inst.C = C;
  inst.nA = nA;
  inst.nB = nB;
  inst.T = make_tau_screen(tau);
  const InstRef ref = make_ref(&inst, nullptr, 1);

  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_normmap(A, n, leaf, nA, nullptr, s);
  if (e == cudaSuccess) e = launch_normmap(B, n, leaf, nB, nullptr, s);
  if (e == cudaSuccess) e = run_plan(ref, buf, s);
  if (e == cudaSuccess) e = launch_multiply_simt(ref, buf, leaf, kScheduleStatic, s);
  if (e == cudaSuccess) e = launch_zero_empty_tiles(ref, buf, leaf, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}
