// C ABI of the SpAMM library: argument validation, plan ownership, dispatch.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "plan.cuh"
#include "tc_common.cuh"

using namespace spamm;

struct spamm_plan_s {
  int64_t n = 0;
  int32_t leaf = 0;
  int32_t bd = 0;
  spamm_precision_t precision = SPAMM_FP32;
  int device = 0;
  void* base = nullptr;     // workspace
  bool owns = false;
  PlanBuffers buf{};
  OperandImages img{};      // tensor-core modes only
  cudaStream_t side = nullptr;        // zero-fill of empty tiles runs here, overlapped
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace spamm {

namespace {
constexpr int kMaxDevices = 64;
int32_t* g_status[kMaxDevices] = {};
std::mutex g_status_mu;
constexpr int kReduceParts = 1024;
double* g_reduce[kMaxDevices] = {};   // [kReduceParts + 1] per device
}  // namespace

int32_t* device_status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!g_status[dev]) {
    int32_t* p = nullptr;
    if (cudaMalloc(&p, sizeof(int32_t)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int32_t)) != cudaSuccess) return nullptr;
    g_status[dev] = p;
  }
  return g_status[dev];
}

static double* reduce_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!g_reduce[dev]) {
    double* p = nullptr;
    if (cudaMalloc(&p, (kReduceParts + 1) * sizeof(double)) != cudaSuccess) return nullptr;
    g_reduce[dev] = p;
  }
  return g_reduce[dev];
}

}  // namespace spamm

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool leaf_ok(int32_t leaf) { return leaf == 32 || leaf == 64 || leaf == 128; }
bool precision_ok(spamm_precision_t p) { return p >= SPAMM_FP32 && p <= SPAMM_FP16_SPLIT; }
bool is_split(spamm_precision_t p) {
  return p == SPAMM_BF16_SPLIT || p == SPAMM_FP16_SPLIT || p == SPAMM_TF32X3;
}

// Unit roundoff of the hi part of each precision (for the split-flag budget).
double hi_unit(spamm_precision_t p) {
  switch (p) {
    case SPAMM_BF16:
    case SPAMM_BF16_SPLIT: return std::ldexp(1.0, -8);
    case SPAMM_FP16:
    case SPAMM_FP16_SPLIT:
    case SPAMM_TF32X3: return std::ldexp(1.0, -11);
    default: return 0.0;
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace spamm {

// Lays the plan buffers out in one allocation; returns the total size.
size_t plan_layout(int bd, PlanBuffers* b, char* base) {
  const size_t tiles = (size_t)bd * bd;
  const size_t parts = (size_t)plan_part_count(bd);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  PlanBuffers t{};
  t.bd = bd;
  t.pd = reinterpret_cast<PlanDevice*>(take(sizeof(PlanDevice)));
  t.sA = reinterpret_cast<Screen*>(take(tiles * sizeof(Screen)));
  t.sBT = reinterpret_cast<Screen*>(take(tiles * sizeof(Screen)));
  t.part_a = reinterpret_cast<double*>(take(parts * sizeof(double)));
  t.part_b = reinterpret_cast<double*>(take(parts * sizeof(double)));
  t.part_S = reinterpret_cast<long long*>(take(parts * sizeof(long long)));
  t.part_kmax = reinterpret_cast<int*>(take(parts * sizeof(int)));
  t.part_ne = reinterpret_cast<int*>(take(parts * sizeof(int)));
  t.part_b1 = reinterpret_cast<ExtSum*>(take(parts * sizeof(ExtSum)));
  t.part_b2 = reinterpret_cast<ExtSum*>(take(parts * sizeof(ExtSum)));
  t.cta_base = reinterpret_cast<int*>(take(parts * sizeof(int)));
  t.cta_ebase = reinterpret_cast<int*>(take(parts * sizeof(int)));
  t.cnt = reinterpret_cast<int*>(take(tiles * sizeof(int)));
  t.tile_ptr = reinterpret_cast<int*>(take((tiles + 1) * sizeof(int)));
  t.order = reinterpret_cast<int*>(take(tiles * sizeof(int)));
  t.k_idx = reinterpret_cast<uint16_t*>(take(tiles * (size_t)bd * sizeof(uint16_t)));
  t.needA = reinterpret_cast<uint8_t*>(take(tiles));
  t.needB = reinterpret_cast<uint8_t*>(take(tiles));
  if (b) *b = t;
  return align_up(off, 256);
}

bool is_tensor_mode(spamm_precision_t p) { return p != SPAMM_FP32; }

bool has_lo(spamm_precision_t p) {
  return p == SPAMM_BF16_SPLIT || p == SPAMM_FP16_SPLIT || p == SPAMM_TF32X3;
}

// Operand images of the tensor-core modes, carved after the plan buffers.
size_t images_layout(int bd, int leaf, spamm_precision_t prec, OperandImages* img, char* base) {
  OperandImages t{};
  if (!is_tensor_mode(prec)) {
    if (img) *img = t;
    return 0;
  }
  const size_t tiles = (size_t)bd * bd;
  const size_t blk = (size_t)leaf * leaf * (prec == SPAMM_TF32X3 ? 4 : 2);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  t.a_hi = reinterpret_cast<uint8_t*>(take(tiles * blk));
  t.b_hi = reinterpret_cast<uint8_t*>(take(tiles * blk));
  if (has_lo(prec)) {
    t.a_lo = reinterpret_cast<uint8_t*>(take(tiles * blk));
    t.b_lo = reinterpret_cast<uint8_t*>(take(tiles * blk));
  }
  t.ea = reinterpret_cast<int32_t*>(take(tiles * sizeof(int32_t)));
  t.eb = reinterpret_cast<int32_t*>(take(tiles * sizeof(int32_t)));
  if (img) *img = t;
  return align_up(off, 256);
}

}  // namespace spamm

namespace {

spamm_status_t check_shape(int64_t n, int32_t leaf) {
  if (n < 1) return SPAMM_ERR_INVALID_ARG;
  if (!leaf_ok(leaf)) return SPAMM_ERR_UNSUPPORTED;
  if (num_blocks(n, leaf) > kMaxBd) return SPAMM_ERR_UNSUPPORTED;
  if (n > (int64_t)1 << 20) return SPAMM_ERR_UNSUPPORTED;
  return SPAMM_OK;
}

}  // namespace

extern "C" {

const char* spamm_status_string(spamm_status_t s) {
  switch (s) {
    case SPAMM_OK: return "ok";
    case SPAMM_ERR_INVALID_ARG: return "invalid argument";
    case SPAMM_ERR_UNSUPPORTED: return "unsupported leaf size, precision or shape";
    case SPAMM_ERR_CUDA: return "CUDA runtime error";
    case SPAMM_ERR_NO_MEMORY: return "out of memory or workspace too small";
    case SPAMM_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SPAMM_ERR_DEVICE_FAULT: return "a device-side bounds check failed";
  }
  return "unknown status";
}

spamm_status_t spamm_normmap(const float* X, int64_t n, int32_t leaf, double* normmap,
                             void* stream) {
  spamm_status_t st = check_shape(n, leaf);
  if (st != SPAMM_OK) return st;
  if (!X || !normmap || !aligned16(X) || !aligned16(normmap)) return SPAMM_ERR_INVALID_ARG;
  cudaError_t e = launch_normmap(X, n, leaf, normmap, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_workspace_size(int64_t n, int32_t leaf, spamm_precision_t precision,
                                         size_t* bytes) {
  spamm_status_t st = check_shape(n, leaf);
  if (st != SPAMM_OK) return st;
  if (!precision_ok(precision)) return SPAMM_ERR_INVALID_ARG;
  if (!bytes) return SPAMM_ERR_INVALID_ARG;
  if (is_tensor_mode(precision) && leaf == 32) return SPAMM_ERR_UNSUPPORTED;
  const int bd = (int)num_blocks(n, leaf);
  *bytes = plan_layout(bd, nullptr, nullptr) + images_layout(bd, leaf, precision, nullptr, nullptr);
  return SPAMM_OK;
}

spamm_status_t spamm_plan_create(spamm_plan_t* plan, int64_t n, int32_t leaf,
                                 spamm_precision_t precision, void* workspace, size_t ws_bytes) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  *plan = nullptr;
  spamm_status_t st = check_shape(n, leaf);
  if (st != SPAMM_OK) return st;
  if (!precision_ok(precision)) return SPAMM_ERR_INVALID_ARG;
  if (is_tensor_mode(precision) && leaf == 32) return SPAMM_ERR_UNSUPPORTED;
  const int bd = (int)num_blocks(n, leaf);
  const size_t plan_bytes = plan_layout(bd, nullptr, nullptr);
  const size_t need = plan_bytes + images_layout(bd, leaf, precision, nullptr, nullptr);
  spamm_plan_s* p = new (std::nothrow) spamm_plan_s();
  if (!p) return SPAMM_ERR_NO_MEMORY;
  p->n = n;
  p->leaf = leaf;
  p->bd = bd;
  p->precision = precision;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return SPAMM_ERR_CUDA;
  }
  if (workspace) {
    if (ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
      delete p;
      return ws_bytes < need ? SPAMM_ERR_NO_MEMORY : SPAMM_ERR_INVALID_ARG;
    }
    p->base = workspace;
  } else {
    if (cudaMalloc(&p->base, need) != cudaSuccess) {
      (void)cudaGetLastError();
      delete p;
      return SPAMM_ERR_NO_MEMORY;
    }
    p->owns = true;
  }
  plan_layout(bd, &p->buf, static_cast<char*>(p->base));
  images_layout(bd, leaf, precision, &p->img, static_cast<char*>(p->base) + plan_bytes);
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    if (p->side) cudaStreamDestroy(p->side);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->owns) cudaFree(p->base);
    delete p;
    return SPAMM_ERR_CUDA;
  }
  *plan = p;
  return SPAMM_OK;
}

spamm_status_t spamm_plan_destroy(spamm_plan_t plan) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = SPAMM_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) st = SPAMM_ERR_CUDA;
  if (plan->side) cudaStreamDestroy(plan->side);
  if (plan->fork) cudaEventDestroy(plan->fork);
  if (plan->join) cudaEventDestroy(plan->join);
  if (plan->owns && plan->base) {
    if (cudaFree(plan->base) != cudaSuccess) st = SPAMM_ERR_CUDA;
  }
  delete plan;
  return st;
}

spamm_status_t spamm_plan(spamm_plan_t plan, const double* normA, const double* normB,
                          double tau, double target_rel_err, void* stream) {
  if (!plan || !normA || !normB) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (std::isnan(tau) || tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  const bool split = is_split(plan->precision) && plan->precision != SPAMM_TF32X3;
  if (split && !(target_rel_err >= 0.0)) return SPAMM_ERR_INVALID_ARG;
  const double u = hi_unit(plan->precision);
  cudaError_t e = run_plan(plan->buf, normA, normB, tau, target_rel_err, split ? 1 : 0,
                           2.0 * u + u * u, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_stats(spamm_plan_t plan, spamm_stats_t* stats, void* stream) {
  if (!plan || !stats) return SPAMM_ERR_INVALID_ARG;
  PlanDevice h;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(&h, plan->buf.pd, sizeof(PlanDevice), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
  SPAMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  std::memset(stats, 0, sizeof(*stats));
  stats->survivors = h.survivors;
  stats->nonempty_tiles = h.nonempty;
  stats->flagged = h.flagged;
  stats->valid_ratio = h.valid_ratio;
  stats->skipped_bound1 = h.bound1;
  stats->skipped_bound2 = h.bound2;
  stats->norm_a = h.norm_a;
  stats->norm_b = h.norm_b;
  stats->leaf = plan->leaf;
  stats->bd = plan->bd;
  stats->max_tile_survivors = h.max_tile;
  stats->flag_exponent = h.flag_exp;
  return SPAMM_OK;
}

spamm_status_t spamm_plan_export(spamm_plan_t plan, int32_t* tile_ptr, uint16_t* k_idx,
                                 int64_t cap, void* stream) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t tiles = (int64_t)plan->bd * plan->bd;
  int32_t total = 0;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(&total, plan->buf.tile_ptr + tiles, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  if (tile_ptr)
    SPAMM_CUDA_TRY(cudaMemcpyAsync(tile_ptr, plan->buf.tile_ptr, (tiles + 1) * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, s));
  if (k_idx) {
    if (cap < total) return SPAMM_ERR_NO_MEMORY;
    if (total > 0)
      SPAMM_CUDA_TRY(cudaMemcpyAsync(k_idx, plan->buf.k_idx, (size_t)total * sizeof(uint16_t),
                                     cudaMemcpyDeviceToHost, s));
  }
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

spamm_status_t spamm_multiply(spamm_plan_t plan, const float* A, const float* B, float* C,
                              void* stream) {
  if (!plan || !A || !B || !C) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return SPAMM_ERR_INVALID_ARG;
  if (A == C || B == C) return SPAMM_ERR_INVALID_ARG;
  int32_t* status = nullptr;
  if (plan->precision != SPAMM_FP32) {
    status = device_status_word();
    if (!status) return SPAMM_ERR_NO_MEMORY;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  // empty tiles (zeros, HBM-write bound) on the side stream, overlapped with
  // the rounding and multiply of the non-empty tiles (disjoint parts of C)
  cudaError_t e = cudaEventRecord(plan->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->side, plan->fork, 0);
  if (e == cudaSuccess) e = launch_zero_empty_tiles(plan->buf, C, plan->n, plan->leaf, plan->side);
  if (e == cudaSuccess) e = cudaEventRecord(plan->join, plan->side);
  if (e == cudaSuccess) {
    if (plan->precision == SPAMM_FP32) {
      e = launch_multiply_simt(plan->buf, A, B, C, plan->n, plan->leaf, s);
    } else {
      e = launch_quantize(plan->precision, plan->leaf, A, B, plan->n, plan->bd, plan->buf.needA,
                          plan->buf.needB, plan->img, s);
      if (e == cudaSuccess)
        e = launch_multiply_tc(plan->precision, plan->leaf, plan->buf, plan->img, C, plan->n,
                               status, s);
    }
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->join, 0);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_frobenius_diff(const float* X, const float* Y, int64_t count, double* out,
                                    void* stream) {
  if (!X || !out || count < 0) return SPAMM_ERR_INVALID_ARG;
  double* scratch = reduce_scratch();
  if (!scratch) return SPAMM_ERR_NO_MEMORY;
  cudaStream_t s = (cudaStream_t)stream;
  const int parts = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (count + 2047) / 2048));
  cudaError_t e = launch_frobenius_diff(X, Y, count, scratch, parts, scratch + kReduceParts, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  SPAMM_CUDA_TRY(cudaMemcpyAsync(out, scratch + kReduceParts, sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

spamm_status_t spamm_last_device_status(void* stream, int32_t* code) {
  if (!code) return SPAMM_ERR_INVALID_ARG;
  int32_t* w = device_status_word();
  if (!w) return SPAMM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(code, w, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(int32_t), s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

}  // extern "C"
