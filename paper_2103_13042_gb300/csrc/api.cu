// C ABI of the SpAMM library: argument validation, plan ownership, dispatch.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "engine.cuh"

using namespace spamm;

namespace spamm {

namespace {
constexpr int kMaxDevices = 64;
int32_t* g_status[kMaxDevices] = {};
std::mutex g_status_mu;
constexpr int kReduceParts = 1024;
double* g_reduce[kMaxDevices] = {};   // [kReduceParts + 1] per device

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
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

bool is_tensor_mode(spamm_precision_t p) { return p != SPAMM_FP32; }

bool has_lo(spamm_precision_t p) {
  return p == SPAMM_BF16_SPLIT || p == SPAMM_FP16_SPLIT || p == SPAMM_TF32X3;
}

bool uses_split_flags(spamm_precision_t p) {
  return p == SPAMM_BF16_SPLIT || p == SPAMM_FP16_SPLIT;
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

size_t engine_layout(std::vector<Inst>& insts, int leaf, spamm_precision_t prec, size_t extra,
                     PlanBuffers* buf, OperandImages* img, char* base, double** tau,
                     float** feat) {
  size_t off = align_up(extra, 256);
  PlanBuffers b{};
  const size_t plan_bytes = plan_layout(insts.data(), (int)insts.size(), &b,
                                        base ? base + off : nullptr, is_tensor_mode(prec));
  off += plan_bytes;
  OperandImages t{};
  if (is_tensor_mode(prec)) {
    const size_t na = (size_t)b.ablks, nb = (size_t)b.bblks;
    const size_t blk = (size_t)leaf * leaf * (prec == SPAMM_TF32X3 ? 4 : 2);
    auto take = [&](size_t bytes) {
      off = align_up(off, 256);
      char* p = base ? base + off : nullptr;
      off += bytes;
      return p;
    };
    t.a_hi = reinterpret_cast<uint8_t*>(take(na * blk));
    t.b_hi = reinterpret_cast<uint8_t*>(take(nb * blk));
    if (has_lo(prec)) {
      t.a_lo = reinterpret_cast<uint8_t*>(take(na * blk));
      t.b_lo = reinterpret_cast<uint8_t*>(take(nb * blk));
    }
    t.ea = reinterpret_cast<int32_t*>(take(na * sizeof(int32_t)));
    t.eb = reinterpret_cast<int32_t*>(take(nb * sizeof(int32_t)));
  }
  {
    off = align_up(off, 256);
    if (tau) *tau = base ? reinterpret_cast<double*>(base + off) : nullptr;
    off += insts.size() * sizeof(double);
    off = align_up(off, 256);
    if (feat) *feat = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += insts.size() * 65 * sizeof(float);
  }
  if (buf) *buf = b;
  if (img) *img = t;
  return align_up(off, 256);
}

spamm_status_t engine_init(Engine& e, std::vector<Inst> insts, int leaf, spamm_precision_t prec,
                           size_t extra, void* workspace, size_t ws_bytes) {
  e.leaf = leaf;
  e.precision = prec;
  e.extra_bytes = extra;
  e.insts = std::move(insts);
  const size_t need = engine_layout(e.insts, leaf, prec, extra, nullptr, nullptr, nullptr);
  if (cudaGetDevice(&e.device) != cudaSuccess) return SPAMM_ERR_CUDA;
  if (workspace) {
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return SPAMM_ERR_INVALID_ARG;
    if (ws_bytes < need) return SPAMM_ERR_NO_MEMORY;
    e.base = workspace;
  } else {
    if (cudaMalloc(&e.base, need) != cudaSuccess) {
      (void)cudaGetLastError();
      e.base = nullptr;
      return SPAMM_ERR_NO_MEMORY;
    }
    e.owns = true;
  }
  engine_layout(e.insts, leaf, prec, extra, &e.buf, &e.img, static_cast<char*>(e.base), &e.tau_dev,
                &e.feat_dev);
  if (cudaStreamCreateWithFlags(&e.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    engine_free(e);
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t engine_free(Engine& e) {
  spamm_status_t st = SPAMM_OK;
  if (e.side) cudaStreamDestroy(e.side);
  if (e.fork) cudaEventDestroy(e.fork);
  if (e.join) cudaEventDestroy(e.join);
  e.side = nullptr;
  e.fork = e.join = nullptr;
  if (e.owns && e.base) {
    if (cudaFree(e.base) != cudaSuccess) st = SPAMM_ERR_CUDA;
  }
  e.base = nullptr;
  e.owns = false;
  return st;
}

namespace {

// The multiply of the non-empty tiles (operand rounding first in tensor modes).
cudaError_t multiply_nonempty(Engine& e, const InstRef& ref, int32_t* status, cudaStream_t s,
                              cudaEvent_t after_round) {
  cudaError_t err = cudaSuccess;
  if (e.schedule == kScheduleDynamic)
    err = cudaMemsetAsync(&e.buf.bdev->mul_ticket, 0, sizeof(int), s);
  if (err != cudaSuccess) return err;
  if (e.precision == SPAMM_FP32) {
    if (after_round) err = cudaEventRecord(after_round, s);
    if (err == cudaSuccess) err = launch_multiply_simt(ref, e.buf, e.leaf, e.schedule, s);
  } else {
    err = launch_quantize(e.precision, e.leaf, ref, e.buf, e.img, s);
    if (err == cudaSuccess && after_round) err = cudaEventRecord(after_round, s);
    if (err == cudaSuccess)
      err = launch_multiply_tc(e.precision, e.leaf, ref, e.buf, e.img, status, e.schedule, s);
    if (err == cudaSuccess && ref.any_norm_out) err = launch_norm_out_finish(ref, e.buf, e.leaf, s);
  }
  return err;
}

}  // namespace

cudaError_t engine_multiply(Engine& e, const InstRef& ref, int32_t* status, cudaStream_t s,
                            cudaEvent_t after_round) {
  // empty tiles (zeros, HBM-write bound) on the side stream, overlapped with
  // the rounding and multiply of the non-empty tiles (disjoint parts of C)
  cudaError_t err = cudaEventRecord(e.fork, s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(e.side, e.fork, 0);
  if (err == cudaSuccess) err = launch_zero_empty_tiles(ref, e.buf, e.leaf, e.side);
  if (err == cudaSuccess) err = cudaEventRecord(e.join, e.side);
  if (err == cudaSuccess) err = multiply_nonempty(e, ref, status, s, after_round);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(s, e.join, 0);
  return err;
}

cudaError_t engine_plan_multiply(Engine& e, const InstRef& ref, int32_t* status, cudaStream_t s,
                                 cudaEvent_t after_plan, cudaEvent_t after_round) {
  // the empty tiles are known once the counting half of the plan is done: their
  // zeros (HBM-write bound) overlap the latency-bound rest of the plan, the
  // rounding and the multiply
  cudaError_t err = run_plan_count_half(ref, e.buf, s);
  if (err == cudaSuccess) err = cudaEventRecord(e.fork, s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(e.side, e.fork, 0);
  if (err == cudaSuccess) err = launch_zero_empty_tiles_scan(ref, e.buf, e.leaf, e.side);
  if (err == cudaSuccess) err = cudaEventRecord(e.join, e.side);
  if (err == cudaSuccess) err = run_plan_queue_half(ref, e.buf, s);
  if (err == cudaSuccess && after_plan) err = cudaEventRecord(after_plan, s);
  if (err == cudaSuccess) err = multiply_nonempty(e, ref, status, s, after_round);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(s, e.join, 0);
  return err;
}

void fill_stats(const PlanDevice& h, int leaf, int bd, spamm_stats_t* stats) {
  std::memset(stats, 0, sizeof(*stats));
  stats->survivors = h.survivors;
  stats->nonempty_tiles = h.nonempty;
  stats->flagged = h.flagged;
  stats->valid_ratio = h.valid_ratio;
  stats->skipped_bound1 = h.bound1;
  stats->skipped_bound2 = h.bound2;
  stats->norm_a = h.norm_a;
  stats->norm_b = h.norm_b;
  stats->leaf = leaf;
  stats->bd = bd;
  stats->max_tile_survivors = h.max_tile;
  stats->flag_exponent = h.flag_exp;
}

spamm_status_t export_queues(const PlanBuffers& b, const Inst& in, int32_t* tile_ptr,
                             uint16_t* k_idx, int64_t cap, cudaStream_t s) {
  const int64_t tiles = (int64_t)in.bm * in.bn;
  // per tile: count and absolute first slot (tiles are stored in the plan's
  // enumeration order, not row-major)
  std::vector<int32_t> cnt((size_t)tiles), beg((size_t)tiles);
  SPAMM_CUDA_TRY(cudaMemcpyAsync(cnt.data(), b.cnt + in.tile0, (size_t)tiles * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaMemcpyAsync(beg.data(), b.tile_beg + in.tile0,
                                 (size_t)tiles * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  int64_t total = 0;
  for (int64_t t = 0; t < tiles; ++t) {
    if (tile_ptr) tile_ptr[t] = (int32_t)total;
    total += cnt[(size_t)t];
  }
  if (tile_ptr) tile_ptr[tiles] = (int32_t)total;
  if (k_idx) {
    if (cap < total) return SPAMM_ERR_NO_MEMORY;
    if (total > 0) {
      // the instance's slots are one contiguous range from its first slot
      std::vector<uint16_t> raw((size_t)total);
      SPAMM_CUDA_TRY(cudaMemcpyAsync(raw.data(), b.k_idx + in.kidx0,
                                     (size_t)total * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
      SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
      int64_t o = 0;
      for (int64_t t = 0; t < tiles; ++t) {
        const int64_t src = (int64_t)beg[(size_t)t] - in.kidx0;
        for (int32_t q = 0; q < cnt[(size_t)t]; ++q) k_idx[o++] = raw[(size_t)(src + q)];
      }
    }
  }
  return SPAMM_OK;
}

}  // namespace spamm

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool leaf_ok(int32_t leaf) { return leaf == 32 || leaf == 64 || leaf == 128; }
bool precision_ok(spamm_precision_t p) { return p >= SPAMM_FP32 && p <= SPAMM_FP16_SPLIT; }

spamm_status_t check_shape(int64_t n, int32_t leaf) {
  if (n < 1) return SPAMM_ERR_INVALID_ARG;
  if (!leaf_ok(leaf)) return SPAMM_ERR_UNSUPPORTED;
  if (num_blocks(n, leaf) > kMaxBd) return SPAMM_ERR_UNSUPPORTED;
  if (n > (int64_t)1 << 20) return SPAMM_ERR_UNSUPPORTED;
  return SPAMM_OK;
}

// General shapes: the inner block count is stored in 10 bits of a k index;
// tile positions, k slots and block numbers are 32-bit on the device.
spamm_status_t check_general(int64_t m, int64_t kd, int64_t n, int32_t leaf) {
  if (m < 1 || kd < 1 || n < 1) return SPAMM_ERR_INVALID_ARG;
  if (!leaf_ok(leaf)) return SPAMM_ERR_UNSUPPORTED;
  const int64_t lim = (int64_t)1 << 24;
  if (m > lim || kd > lim || n > lim) return SPAMM_ERR_UNSUPPORTED;
  const int64_t bm = num_blocks(m, leaf), bk = num_blocks(kd, leaf), bn = num_blocks(n, leaf);
  if (bk > kMaxBd) return SPAMM_ERR_UNSUPPORTED;
  if (bm * bn > ((int64_t)1 << 22)) return SPAMM_ERR_UNSUPPORTED;
  if (bm * bk * bn >= ((int64_t)1 << 31) || bm * bk >= ((int64_t)1 << 31) ||
      bk * bn >= ((int64_t)1 << 31))
    return SPAMM_ERR_UNSUPPORTED;
  return SPAMM_OK;
}

// Bytes spanned by a rows x cols row-major matrix with leading dimension ld.
size_t span_bytes(int64_t rows, int64_t cols, int64_t ld) {
  return (size_t)((rows - 1) * ld + cols) * sizeof(float);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

std::vector<Inst> single_inst(int64_t n, int leaf) {
  std::vector<Inst> v(1);
  v[0] = Inst{};
  set_square(v[0], n, leaf);
  return v;
}

std::vector<Inst> general_inst(int64_t m, int64_t kd, int64_t n, int leaf) {
  std::vector<Inst> v(1);
  v[0] = Inst{};
  set_general(v[0], m, kd, n, kd, n, n, 1.0f, 0.0f, leaf);
  return v;
}

// The plan's instance reset to the square call form: leading dimensions of
// its own shape, alpha = 1, beta = 0, no output norm map.
void square_call(Inst& in) {
  in.lda = in.kd;
  in.ldb = in.n;
  in.ldc = in.n;
  in.alpha = 1.0f;
  in.beta = 0.0f;
  in.nC = nullptr;
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
  int32_t* status = device_status_word();
  if (!status) return SPAMM_ERR_NO_MEMORY;
  cudaError_t e = launch_normmap(X, n, leaf, normmap, status, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_normmap_pair(const float* A, const float* B, int64_t n, int32_t leaf,
                                  double* normA, double* normB, void* stream) {
  spamm_status_t st = check_shape(n, leaf);
  if (st != SPAMM_OK) return st;
  if (!A || !B || !normA || !normB || !aligned16(A) || !aligned16(B) || !aligned16(normA) ||
      !aligned16(normB) || normA == normB)
    return SPAMM_ERR_INVALID_ARG;
  int32_t* status = device_status_word();
  if (!status) return SPAMM_ERR_NO_MEMORY;
  cudaError_t e = launch_normmap_pair(A, B, n, leaf, normA, normB, status, (cudaStream_t)stream);
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
  std::vector<Inst> v = single_inst(n, leaf);
  *bytes = engine_layout(v, leaf, precision, 0, nullptr, nullptr, nullptr);
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
  spamm_plan_s* p = new (std::nothrow) spamm_plan_s();
  if (!p) return SPAMM_ERR_NO_MEMORY;
  p->n = p->m = p->kd = n;
  p->bd = (int)num_blocks(n, leaf);
  st = engine_init(p->eng, single_inst(n, leaf), leaf, precision, 0, workspace, ws_bytes);
  if (st != SPAMM_OK) {
    delete p;
    return st;
  }
  *plan = p;
  return SPAMM_OK;
}

spamm_status_t spamm_plan_set_schedule(spamm_plan_t plan, int32_t schedule) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  switch (schedule) {
    case 0: plan->eng.schedule = kScheduleStatic; return SPAMM_OK;
    case SPAMM_BATCH_DYNAMIC: plan->eng.schedule = kScheduleDynamic; return SPAMM_OK;
    case SPAMM_BATCH_GROUPS: plan->eng.schedule = kScheduleGroups; return SPAMM_OK;
    default: return SPAMM_ERR_INVALID_ARG;
  }
}

spamm_status_t spamm_plan_destroy(spamm_plan_t plan) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = SPAMM_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) st = SPAMM_ERR_CUDA;
  if (engine_free(plan->eng) != SPAMM_OK) st = SPAMM_ERR_CUDA;
  delete plan;
  return st;
}

spamm_status_t spamm_plan(spamm_plan_t plan, const double* normA, const double* normB,
                          double tau, double target_rel_err, void* stream) {
  if (!plan || !normA || !normB) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (std::isnan(tau) || tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  const bool split = uses_split_flags(e.precision);
  if (split && !(target_rel_err >= 0.0)) return SPAMM_ERR_INVALID_ARG;
  const double u = hi_unit(e.precision);
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  in.T = make_tau_screen(tau);
  in.split = split ? 1 : 0;
  in.quant = is_tensor_mode(e.precision) ? 1 : 0;
  in.target_rel = split ? target_rel_err : 0.0;
  in.c1 = split ? 2.0 * u + u * u : 0.0;
  cudaError_t err = run_plan(make_ref(e.insts.data(), nullptr, 1), e.buf, (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_stats(spamm_plan_t plan, spamm_stats_t* stats, void* stream) {
  if (!plan || !stats) return SPAMM_ERR_INVALID_ARG;
  PlanDevice h;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(&h, plan->eng.buf.pd, sizeof(PlanDevice), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
  SPAMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  fill_stats(h, plan->eng.leaf, plan->eng.insts[0].bm, stats);
  return SPAMM_OK;
}

spamm_status_t spamm_plan_export(spamm_plan_t plan, int32_t* tile_ptr, uint16_t* k_idx,
                                 int64_t cap, void* stream) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  return export_queues(plan->eng.buf, plan->eng.insts[0], tile_ptr, k_idx, cap,
                       (cudaStream_t)stream);
}

spamm_status_t spamm_multiply(spamm_plan_t plan, const float* A, const float* B, float* C,
                              void* stream) {
  if (!plan || !A || !B || !C) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return SPAMM_ERR_INVALID_ARG;
  if (A == C || B == C) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  int32_t* status = nullptr;
  if (e.precision != SPAMM_FP32) {
    status = device_status_word();
    if (!status) return SPAMM_ERR_NO_MEMORY;
  }
  Inst& in = e.insts[0];
  square_call(in);
  in.A = A;
  in.B = B;
  in.C = C;
  cudaError_t err = engine_multiply(e, make_ref(e.insts.data(), nullptr, 1), status,
                                    (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_multiply(spamm_plan_t plan, const double* normA, const double* normB,
                                   double tau, double target_rel_err, const float* A,
                                   const float* B, float* C, void* stream) {
  if (!plan || !normA || !normB || !A || !B || !C) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return SPAMM_ERR_INVALID_ARG;
  if (A == C || B == C) return SPAMM_ERR_INVALID_ARG;
  if (std::isnan(tau) || tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  const bool split = uses_split_flags(e.precision);
  if (split && !(target_rel_err >= 0.0)) return SPAMM_ERR_INVALID_ARG;
  int32_t* status = nullptr;
  if (e.precision != SPAMM_FP32) {
    status = device_status_word();
    if (!status) return SPAMM_ERR_NO_MEMORY;
  }
  const double u = hi_unit(e.precision);
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  in.T = make_tau_screen(tau);
  in.band = 0;
  in.split = split ? 1 : 0;
  in.quant = is_tensor_mode(e.precision) ? 1 : 0;
  in.target_rel = split ? target_rel_err : 0.0;
  in.c1 = split ? 2.0 * u + u * u : 0.0;
  square_call(in);
  in.A = A;
  in.B = B;
  in.C = C;
  cudaError_t err = engine_plan_multiply(e, make_ref(e.insts.data(), nullptr, 1), status,
                                         (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_normmap_rect(const float* X, int64_t rows, int64_t cols, int64_t ld,
                                  int32_t leaf, double* normmap, void* stream) {
  spamm_status_t st = check_general(rows, 1, cols, leaf);
  if (st != SPAMM_OK) return st;
  if (ld < cols) return SPAMM_ERR_INVALID_ARG;
  if (!X || !normmap || !aligned16(X) || !aligned16(normmap)) return SPAMM_ERR_INVALID_ARG;
  int32_t* status = device_status_word();
  if (!status) return SPAMM_ERR_NO_MEMORY;
  cudaError_t e = launch_normmap_rect(X, rows, cols, ld, leaf, normmap, status,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_workspace_size_general(int64_t m, int64_t k, int64_t n, int32_t leaf,
                                                 spamm_precision_t precision, size_t* bytes) {
  spamm_status_t st = check_general(m, k, n, leaf);
  if (st != SPAMM_OK) return st;
  if (!precision_ok(precision) || !bytes) return SPAMM_ERR_INVALID_ARG;
  if (is_tensor_mode(precision) && leaf == 32) return SPAMM_ERR_UNSUPPORTED;
  std::vector<Inst> v = general_inst(m, k, n, leaf);
  *bytes = engine_layout(v, leaf, precision, 0, nullptr, nullptr, nullptr);
  return SPAMM_OK;
}

spamm_status_t spamm_plan_create_general(spamm_plan_t* plan, int64_t m, int64_t k, int64_t n,
                                         int32_t leaf, spamm_precision_t precision,
                                         void* workspace, size_t ws_bytes) {
  if (!plan) return SPAMM_ERR_INVALID_ARG;
  *plan = nullptr;
  spamm_status_t st = check_general(m, k, n, leaf);
  if (st != SPAMM_OK) return st;
  if (!precision_ok(precision)) return SPAMM_ERR_INVALID_ARG;
  if (is_tensor_mode(precision) && leaf == 32) return SPAMM_ERR_UNSUPPORTED;
  spamm_plan_s* p = new (std::nothrow) spamm_plan_s();
  if (!p) return SPAMM_ERR_NO_MEMORY;
  p->m = m;
  p->kd = k;
  p->n = n;
  p->bd = 0;
  p->general = true;
  st = engine_init(p->eng, general_inst(m, k, n, leaf), leaf, precision, 0, workspace, ws_bytes);
  if (st != SPAMM_OK) {
    delete p;
    return st;
  }
  *plan = p;
  return SPAMM_OK;
}

namespace {

// Argument checks and instance set-up of the general multiply calls.
spamm_status_t general_call(spamm_plan_t plan, const float* A, int64_t lda, const float* B,
                            int64_t ldb, float* C, int64_t ldc, float alpha, float beta,
                            double* normC) {
  if (!plan || !A || !B || !C) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return SPAMM_ERR_INVALID_ARG;
  if (normC && !aligned16(normC)) return SPAMM_ERR_INVALID_ARG;
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return SPAMM_ERR_INVALID_ARG;
  Inst& in = plan->eng.insts[0];
  if (lda < in.kd || ldb < in.n || ldc < in.n) return SPAMM_ERR_INVALID_ARG;
  const size_t sc = span_bytes(in.m, in.n, ldc);
  if (overlaps(C, sc, A, span_bytes(in.m, in.kd, lda)) ||
      overlaps(C, sc, B, span_bytes(in.kd, in.n, ldb)))
    return SPAMM_ERR_INVALID_ARG;
  in.A = A;
  in.B = B;
  in.C = C;
  in.lda = lda;
  in.ldb = ldb;
  in.ldc = ldc;
  in.alpha = alpha;
  in.beta = beta;
  in.nC = normC;
  return SPAMM_OK;
}

}  // namespace

spamm_status_t spamm_multiply_general(spamm_plan_t plan, const float* A, int64_t lda,
                                      const float* B, int64_t ldb, float* C, int64_t ldc,
                                      float alpha, float beta, double* normC, void* stream) {
  spamm_status_t st = general_call(plan, A, lda, B, ldb, C, ldc, alpha, beta, normC);
  if (st != SPAMM_OK) return st;
  Engine& e = plan->eng;
  int32_t* status = nullptr;
  if (e.precision != SPAMM_FP32) {
    status = device_status_word();
    if (!status) return SPAMM_ERR_NO_MEMORY;
  }
  cudaError_t err = engine_multiply(e, make_ref(e.insts.data(), nullptr, 1), status,
                                    (cudaStream_t)stream);
  square_call(e.insts[0]);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_multiply_general(spamm_plan_t plan, const double* normA,
                                           const double* normB, double tau, double target_rel_err,
                                           const float* A, int64_t lda, const float* B,
                                           int64_t ldb, float* C, int64_t ldc, float alpha,
                                           float beta, double* normC, void* stream) {
  if (!plan || !normA || !normB) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (std::isnan(tau) || tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  const bool split = uses_split_flags(e.precision);
  if (split && !(target_rel_err >= 0.0)) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = general_call(plan, A, lda, B, ldb, C, ldc, alpha, beta, normC);
  if (st != SPAMM_OK) return st;
  int32_t* status = nullptr;
  if (e.precision != SPAMM_FP32) {
    status = device_status_word();
    if (!status) return SPAMM_ERR_NO_MEMORY;
  }
  const double u = hi_unit(e.precision);
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  in.T = make_tau_screen(tau);
  in.band = 0;
  in.split = split ? 1 : 0;
  in.quant = is_tensor_mode(e.precision) ? 1 : 0;
  in.target_rel = split ? target_rel_err : 0.0;
  in.c1 = split ? 2.0 * u + u * u : 0.0;
  cudaError_t err = engine_plan_multiply(e, make_ref(e.insts.data(), nullptr, 1), status,
                                         (cudaStream_t)stream);
  square_call(in);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_plan_band(spamm_plan_t plan, const double* normA, const double* normB,
                               double tau_lo, double tau_hi, void* stream) {
  if (!plan || !normA || !normB) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (std::isnan(tau_lo) || tau_lo < 0.0 || std::isnan(tau_hi) || !(tau_hi >= tau_lo))
    return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  in.T = make_tau_screen(tau_lo);
  in.T_hi = make_tau_screen(tau_hi);
  in.band = 1;
  in.split = 0;
  in.quant = is_tensor_mode(e.precision) ? 1 : 0;
  in.target_rel = 0.0;
  in.c1 = 0.0;
  cudaError_t err = run_plan(make_ref(e.insts.data(), nullptr, 1), e.buf, (cudaStream_t)stream);
  in.band = 0;
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_tau_for_valid_ratio(spamm_plan_t plan, const double* normA,
                                         const double* normB, double target_ratio, double tol,
                                         int32_t max_probes, double* tau, double* ratio,
                                         int32_t* probes, void* stream) {
  if (!plan || !normA || !normB || !tau) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (!(target_ratio >= 0.0 && target_ratio <= 1.0) || !(tol >= 0.0) || max_probes < 1)
    return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  const int bm = e.insts[0].bm, bk = e.insts[0].bk, bn = e.insts[0].bn;
  const cudaStream_t s = (cudaStream_t)stream;
  // ave = mean of nA[i,k] nB[k,j] over all bm bk bn triples
  //     = sum_k colsum_A(k) rowsum_B(k) / (bm bk bn)
  std::vector<double> ha((size_t)bm * bk), hb((size_t)bk * bn);
  SPAMM_CUDA_TRY(cudaMemcpyAsync(ha.data(), normA, ha.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaMemcpyAsync(hb.data(), normB, hb.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  double acc = 0.0;
  for (int k = 0; k < bk; ++k) {
    double col = 0.0, row = 0.0;
    for (int i = 0; i < bm; ++i) col += ha[(size_t)i * bk + k];
    for (int j = 0; j < bn; ++j) row += hb[(size_t)k * bn + j];
    acc += col * row;
  }
  const double cube = (double)bm * bk * bn;
  const double ave = acc / cube;
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  in.band = 0;
  in.split = 0;
  in.quant = 0;
  auto valid_ratio = [&](double t, double* out) -> spamm_status_t {
    in.T = make_tau_screen(t);
    cudaError_t err = run_plan_count(make_ref(e.insts.data(), nullptr, 1), e.buf, s);
    if (err != cudaSuccess) {
      (void)cudaGetLastError();
      return SPAMM_ERR_CUDA;
    }
    long long surv = 0;
    SPAMM_CUDA_TRY(cudaMemcpyAsync(&surv, &e.buf.pd->survivors, sizeof(long long),
                                   cudaMemcpyDeviceToHost, s));
    SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = (double)surv / cube;
    return SPAMM_OK;
  };
  // Section 3.5.2: widen [0, k ave] until its upper end gives at most the
  // target ratio, probe ave, then bisect until within tol
  double vr = 0.0;
  int k = 1;
  for (;;) {
    spamm_status_t st = valid_ratio(k * ave, &vr);
    if (st != SPAMM_OK) return st;
    if (!(vr > target_ratio) || k >= 1000000) break;
    ++k;
  }
  double lo = 0.0, hi = k * ave;
  double t = ave < hi ? ave : hi;
  spamm_status_t st = valid_ratio(t, &vr);
  if (st != SPAMM_OK) return st;
  int n = 1;
  while (std::fabs(vr - target_ratio) > tol && n < max_probes) {
    if (vr > target_ratio) lo = t;
    else hi = t;
    t = 0.5 * (lo + hi);
    st = valid_ratio(t, &vr);
    if (st != SPAMM_OK) return st;
    ++n;
  }
  *tau = t;
  if (ratio) *ratio = vr;
  if (probes) *probes = n;
  return SPAMM_OK;
}

spamm_status_t spamm_norm_histogram(spamm_plan_t plan, const double* normA, const double* normB,
                                    int64_t* counts, void* stream) {
  if (!plan || !normA || !normB || !counts) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err = run_histogram(make_ref(e.insts.data(), nullptr, 1), e.buf, s);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  PlanDevice h;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(&h, e.buf.pd, sizeof(PlanDevice), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int b = 0; b < kHistBins; ++b) counts[b] = (int64_t)h.hist[b];
  return SPAMM_OK;
}

spamm_status_t spamm_tau_predict(spamm_plan_t plan, const double* normA, const double* normB,
                                 double target_rel_err, const float* weights, double* tau,
                                 void* stream) {
  if (!plan || !normA || !normB || !weights || !tau) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(normA) || !aligned16(normB)) return SPAMM_ERR_INVALID_ARG;
  if (!(target_rel_err > 0.0) || std::isinf(target_rel_err)) return SPAMM_ERR_INVALID_ARG;
  Engine& e = plan->eng;
  Inst& in = e.insts[0];
  in.nA = normA;
  in.nB = normB;
  const double keep = in.target_rel;
  in.target_rel = target_rel_err;
  const cudaStream_t s = (cudaStream_t)stream;
  const InstRef ref = make_ref(e.insts.data(), nullptr, 1);
  cudaError_t err = run_histogram(ref, e.buf, s);
  if (err == cudaSuccess) err = launch_tau_from_hist(ref, weights, e.feat_dev, e.tau_dev, s);
  in.target_rel = keep;
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  SPAMM_CUDA_TRY(cudaMemcpyAsync(tau, e.tau_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

spamm_status_t spamm_mlp_param_count(int32_t* count) {
  if (!count) return SPAMM_ERR_INVALID_ARG;
  *count = mlp_param_count();
  return SPAMM_OK;
}

spamm_status_t spamm_mlp_forward(const float* weights, const float* X, int32_t count, float* y,
                                 void* stream) {
  if (!weights || count < 0 || (count > 0 && (!X || !y))) return SPAMM_ERR_INVALID_ARG;
  cudaError_t err = launch_mlp_forward(weights, X, count, y, (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_mlp_grad(const float* weights, const float* X, const float* y_true,
                              int32_t count, float quantile, float* grad, float* loss,
                              void* stream) {
  if (!weights || !X || !y_true || !grad || !loss || count < 1) return SPAMM_ERR_INVALID_ARG;
  if (!(quantile > 0.0f && quantile < 1.0f)) return SPAMM_ERR_INVALID_ARG;
  cudaError_t err = launch_mlp_grad(weights, X, y_true, count, quantile, grad, loss,
                                    (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_mlp_adam(float* weights, const float* grad, float* m, float* v, int32_t t,
                              float lr, void* stream) {
  if (!weights || !grad || !m || !v || t < 1 || !(lr > 0.0f)) return SPAMM_ERR_INVALID_ARG;
  cudaError_t err = launch_mlp_adam(weights, grad, m, v, t, lr, (cudaStream_t)stream);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_mlp_train(float* weights, float* m, float* v, int32_t t0, const float* X,
                               const float* y_true, const int32_t* idx, int32_t steps,
                               int32_t batch, float lr, float quantile, float* loss_hist,
                               void* stream) {
  if (!weights || !m || !v || !X || !y_true || !idx || t0 < 0 || steps < 0 || batch < 1)
    return SPAMM_ERR_INVALID_ARG;
  if (!(quantile > 0.0f && quantile < 1.0f) || !(lr > 0.0f)) return SPAMM_ERR_INVALID_ARG;
  cudaError_t err = launch_mlp_train(weights, m, v, t0, X, y_true, idx, steps, batch, lr,
                                     quantile, loss_hist, (cudaStream_t)stream);
  if (err != cudaSuccess) {
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

spamm_status_t spamm_selftest_bounded_wait(int64_t limit_ns, int64_t* elapsed_ns,
                                           void* stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000LL) return SPAMM_ERR_INVALID_ARG;
  int32_t* status = device_status_word();
  if (!status) return SPAMM_ERR_NO_MEMORY;
  const cudaStream_t s = (cudaStream_t)stream;
  long long* out = nullptr;
  if (cudaMalloc(&out, 6 * sizeof(long long)) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_NO_MEMORY;
  }
  long long h[6] = {0, 0, 0, 0, 0, 0};
  // the multiply's wait (one thread) and the norm map's warp-wide wait
  cudaError_t err = launch_wait_selftest(status, (uint64_t)limit_ns, out, s);
  if (err == cudaSuccess) err = launch_normmap_wait_selftest(status, (uint64_t)limit_ns, out + 3, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(out);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  if (elapsed_ns) *elapsed_ns = h[2] < h[5] ? h[2] : h[5];
  // both waits must have given up and raised their abort flags
  return (h[0] == 1 && h[1] == 1 && h[3] == 1 && h[4] == 1) ? SPAMM_OK : SPAMM_ERR_DEVICE_FAULT;
}

spamm_status_t spamm_last_device_status(void* stream, int32_t* code) {
  if (!code) return SPAMM_ERR_INVALID_ARG;
  int32_t* w = device_status_word();
  if (!w) return SPAMM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t other = 0;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(code, w, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(int32_t), s));
  SPAMM_CUDA_TRY(noalloc_take_status(s, &other));   // the no-allocation entry point's word
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  if (*code == 0) *code = other;
  return SPAMM_OK;
}

}  // extern "C"
