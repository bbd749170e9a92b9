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
//    cudaGetSymbolAddress (once per device context, with that device current).
//    Under lazy module loading (the CUDA default) that lookup is also when the
//    library's device code is loaded onto the device, so the first call may
//    allocate driver memory for the module and synchronise: make it (n = 1 is
//    enough) at set-up, before any stream capture on the device.  The address
//    is kept with the context's unique id, so a context that is torn down and
//    created again (cudaDeviceReset) gets a fresh lookup, never a stale address.
//  - Bounded waits of the norm map that run out latch SPAMM_ERR_TIMEOUT in a
//    status word of this file (a second static device variable);
//    spamm_last_device_status reads and clears it with the library's own.
//  - All calls on a device share the one array and it keeps whatever the last
//    call left there; each call rewrites every piece it reads and clears its
//    own accumulators.  Calls whose work overlaps on the GPU (two streams, or
//    two host threads) race on the array and give wrong results: serialise them.
#include <cuda.h>

#include <mutex>

#include "tc_common.cuh"

namespace spamm {
namespace {

constexpr int kNoAllocMaxBd = 64;
constexpr size_t kNoAllocBytes = size_t(1) << 20;   // 1 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static __device__ int32_t g_noalloc_status;   // bounded-wait timeouts of this entry point

constexpr int kMaxDevices = 64;

// The current context's unique id through the driver's cuCtxGetCurrent and
// cuCtxGetId, reached with the runtime's entry-point query (no link against
// the driver library).  0 when it cannot be told.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct CtxApi {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

CtxApi ctx_api() {
  static const CtxApi api = [] {
    CtxApi a;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      a.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      a.get_id = reinterpret_cast<CtxGetIdFn>(f);
    (void)cudaGetLastError();
    return a;
  }();
  return api;
}

unsigned long long current_context_id() {
  const CtxApi api = ctx_api();
  if (!api.get_current || !api.get_id) return 0;
  CUcontext ctx = nullptr;
  if (api.get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  return api.get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

struct Resolved {
  unsigned long long ctx = 0;   // id of the context the addresses belong to
  void* scratch = nullptr;
  int32_t* status = nullptr;
};
Resolved g_resolved[kMaxDevices];
std::mutex g_scratch_mu;

// Device addresses of the scratch array and the status word in the current
// device's context.  Looked up with cudaGetSymbolAddress once per context (the
// host-side names of the two variables are stand-ins, never device addresses);
// when the context id cannot be read, looked up on every call.
cudaError_t resolve(Resolved* out, bool lookup) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  Resolved& r = g_resolved[dev];
  const unsigned long long id = current_context_id();
  if (r.scratch && id != 0 && id == r.ctx) {
    *out = r;
    return cudaSuccess;
  }
  if (!lookup) {   // nothing resolved in this context: the entry point has not run in it
    *out = Resolved{};
    return cudaSuccess;
  }
  void* p = nullptr;
  void* q = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  e = cudaGetSymbolAddress(&q, g_noalloc_status);
  if (e != cudaSuccess) return e;
  // the lookup binds the device's primary context to this thread if none was current
  r.ctx = id != 0 ? id : current_context_id();
  r.scratch = p;
  r.status = static_cast<int32_t*>(q);
  *out = r;
  return cudaSuccess;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

cudaError_t noalloc_take_status(cudaStream_t s, int32_t* code) {
  *code = 0;
  Resolved addr;
  cudaError_t e = resolve(&addr, false);
  if (e != cudaSuccess || !addr.status) return e;
  e = cudaMemcpyAsync(code, addr.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(addr.status, 0, sizeof(int32_t), s);
  return e;
}

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
  set_square(inst, n, leaf);
  const size_t plan_bytes = plan_layout(&inst, 1, nullptr, nullptr);
  if (2 * norm_bytes + plan_bytes > kNoAllocBytes) return SPAMM_ERR_UNSUPPORTED;

  Resolved addr;
  if (resolve(&addr, true) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  char* p = static_cast<char*>(addr.scratch);
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
  cudaError_t e = launch_normmap(A, n, leaf, nA, addr.status, s);
  if (e == cudaSuccess) e = launch_normmap(B, n, leaf, nB, addr.status, s);
  if (e == cudaSuccess) e = run_plan(ref, buf, s);
  if (e == cudaSuccess) e = launch_multiply_simt(ref, buf, leaf, kScheduleStatic, s);
  if (e == cudaSuccess) e = launch_zero_empty_tiles(ref, buf, leaf, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}
