// Host-side engine shared by single plans and batches: one workspace holding
// the plan buffers and operand images of a table of instances, plus the
// streams and events of the multiply.
#pragma once

#include <vector>

#include "plan.cuh"
#include "tc_common.cuh"

namespace spamm {

struct Engine {
  int32_t leaf = 0;
  spamm_precision_t precision = SPAMM_FP32;
  int device = 0;
  void* base = nullptr;        // workspace
  bool owns = false;           // allocated by the library
  std::vector<Inst> insts;     // host copy of the instance table (layout fields filled)
  PlanBuffers buf{};
  OperandImages img{};         // tensor-core modes only
  double* tau_dev = nullptr;   // [instances] predicted tau
  float* feat_dev = nullptr;   // [instances * 65] network inputs of the last prediction
  size_t extra_bytes = 0;      // caller-defined area at the start of the workspace
  int schedule = kScheduleStatic;
  cudaStream_t side = nullptr; // zero-fill of empty tiles runs here, overlapped
  cudaEvent_t fork = nullptr, join = nullptr;
};

bool is_tensor_mode(spamm_precision_t p);
bool has_lo(spamm_precision_t p);
bool uses_split_flags(spamm_precision_t p);   // BF16/FP16 split: flag budget in the plan
double hi_unit(spamm_precision_t p);

// Bytes of the workspace for `insts` (bd fields set) with `extra` bytes in
// front; fills the layout of `insts`, `buf` and `img` when `base` is non-null.
size_t engine_layout(std::vector<Inst>& insts, int leaf, spamm_precision_t prec, size_t extra,
                     PlanBuffers* buf, OperandImages* img, char* base, double** tau = nullptr,
                     float** feat = nullptr);

// Sets up `e` for `insts` (only n and bd read): allocates the workspace when
// `workspace` is null, creates the side stream and events.
spamm_status_t engine_init(Engine& e, std::vector<Inst> insts, int leaf, spamm_precision_t prec,
                           size_t extra, void* workspace, size_t ws_bytes);
spamm_status_t engine_free(Engine& e);

// Enqueues the multiply of every instance of `ref` on `s` (zero-fill of the
// empty tiles forked to the side stream and joined back).
// `after_round` (optional) is recorded on `s` once the operands are rounded
// (tensor modes) or right away (FP32).
cudaError_t engine_multiply(Engine& e, const InstRef& ref, int32_t* status, cudaStream_t s,
                            cudaEvent_t after_round = nullptr);

// Plan and multiply in one sequence; the zero-fill of empty tiles starts as
// soon as the plan's counting half is done.  Optional events after the plan
// and after the rounding.
cudaError_t engine_plan_multiply(Engine& e, const InstRef& ref, int32_t* status, cudaStream_t s,
                                 cudaEvent_t after_plan = nullptr,
                                 cudaEvent_t after_round = nullptr);

void fill_stats(const PlanDevice& h, int leaf, int bd, spamm_stats_t* out);

// Host copy of one instance's work queues as a row-major CSR (tile t = i*bd + j):
// tile_ptr[bd*bd + 1] and k_idx[cap] may be null.  Blocks.
spamm_status_t export_queues(const PlanBuffers& b, const Inst& in, int32_t* tile_ptr,
                             uint16_t* k_idx, int64_t cap, cudaStream_t s);

// Lazily allocated device status word of the current device (tensor-core
// kernels latch timeouts there).
int32_t* device_status_word();

// The no-allocation entry point's own status word on the current device:
// copied to *code (host) and cleared, asynchronously on `s`; *code = 0 when
// that entry point has not run in the current context.
cudaError_t noalloc_take_status(cudaStream_t s, int32_t* code);

}  // namespace spamm

// A single-instance plan (the C ABI's spamm_plan_t).
struct spamm_plan_s {
  int64_t n = 0;       // C is m x n, A m x kd, B kd x n (all n for a square plan)
  int64_t m = 0, kd = 0;
  int32_t bd = 0;      // square plans: blocks per dimension
  bool general = false;
  spamm::Engine eng;
};
