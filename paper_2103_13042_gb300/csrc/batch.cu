// Batched SpAMM: many independent instances of uneven n in one pass of each
// kernel (one norm-map launch over both operands of every instance, one plan,
// one rounding launch and one persistent multiply over the global tile
// queue), optionally replayed from a captured CUDA graph.
//
// The paper runs one product at a time (its Section 3.4 spreads a single
// product over GPUs); this is the serving form of the same method: every
// instance keeps its own tau, norm maps, statistics and skipped-product
// bounds, exactly as if it were planned alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "engine.cuh"

using namespace spamm;

struct spamm_batch_s {
  Engine eng;
  int32_t count = 0;
  int32_t flags = 0;
  std::vector<int64_t> n;
  double* normA = nullptr;       // [tiles] norm maps, instance i at tile0_i
  double* normB = nullptr;
  NormJob* jobs_dev = nullptr;   // [2 * count], followed by the Inst table
  Inst* insts_dev = nullptr;     // [count]
  size_t table_bytes = 0;        // jobs + insts (one upload)
  size_t insts_offset = 0;       // offset of the Inst table inside it
  int n_vec_jobs = 0;            // norm-map jobs with 16-byte aligned rows (listed first)
  int units_vec = 0, units_other = 0;
  std::vector<int> job_slot;     // table slot of job 2 i + op (op 0: A, 1: B)
  std::vector<int> job_unit0;    // its first unit in its part of the table
  void* staging = nullptr;       // pinned host copy of the tables being uploaded
  std::vector<char> last;        // tables of the previous upload
  bool uploaded_once = false;
  cudaEvent_t upload_done = nullptr;
  int32_t* status = nullptr;
  cudaStream_t main = nullptr;   // graph launches run here
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t phase[5] = {};     // SPAMM_BATCH_TIMING: start, after norms, plan, rounding, multiply
  bool timed = false;            // a timed run has been enqueued
};

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

spamm_status_t check_shapes(const int64_t* n, int32_t count, int32_t leaf,
                            spamm_precision_t prec) {
  if (!n || count < 1) return SPAMM_ERR_INVALID_ARG;
  if (leaf != 32 && leaf != 64 && leaf != 128) return SPAMM_ERR_UNSUPPORTED;
  if (prec < SPAMM_FP32 || prec > SPAMM_FP16_SPLIT) return SPAMM_ERR_INVALID_ARG;
  if (prec != SPAMM_FP32 && leaf == 32) return SPAMM_ERR_UNSUPPORTED;
  int64_t tiles = 0, kslots = 0;
  for (int32_t i = 0; i < count; ++i) {
    if (n[i] < 1) return SPAMM_ERR_INVALID_ARG;
    if (n[i] > (int64_t)1 << 20) return SPAMM_ERR_UNSUPPORTED;
    const int64_t bd = num_blocks(n[i], leaf);
    if (bd > kMaxBd) return SPAMM_ERR_UNSUPPORTED;
    tiles += bd * bd;
    kslots += bd * bd * bd;
  }
  // tile ids, k_idx slots and grid sizes are 32-bit on the device
  if (tiles >= ((int64_t)1 << 31) || kslots >= ((int64_t)1 << 31)) return SPAMM_ERR_UNSUPPORTED;
  return SPAMM_OK;
}

std::vector<Inst> shape_table(const int64_t* n, int32_t count, int32_t leaf) {
  std::vector<Inst> v((size_t)count);
  for (int32_t i = 0; i < count; ++i) {
    v[i] = Inst{};
    set_square(v[i], n[i], leaf);
  }
  return v;
}

// Bytes of the area in front of the plan buffers: norm maps and the tables.
size_t batch_extra(const std::vector<Inst>& insts, size_t* norm_bytes, size_t* table_bytes,
                   size_t* insts_offset) {
  int64_t tiles = 0;
  for (const Inst& in : insts) tiles += (int64_t)in.bm * in.bn;
  const size_t nb = align256((size_t)tiles * sizeof(double));
  const size_t jobs = align256(2 * insts.size() * sizeof(NormJob));
  const size_t tb = jobs + insts.size() * sizeof(Inst);
  if (norm_bytes) *norm_bytes = nb;
  if (table_bytes) *table_bytes = tb;
  if (insts_offset) *insts_offset = jobs;
  return 2 * nb + align256(tb);
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

spamm_status_t check_problems(const spamm_batch_s* b, const spamm_problem_t* p) {
  if (!p) return SPAMM_ERR_INVALID_ARG;
  for (int32_t i = 0; i < b->count; ++i) {
    const spamm_problem_t& q = p[i];
    if (q.n != b->n[i]) return SPAMM_ERR_INVALID_ARG;
    if (!q.A || !q.B || !q.C) return SPAMM_ERR_INVALID_ARG;
    if (!aligned16(q.A) || !aligned16(q.B) || !aligned16(q.C)) return SPAMM_ERR_INVALID_ARG;
    if (std::isnan(q.tau) || q.tau < 0.0) return SPAMM_ERR_INVALID_ARG;
  }
  // an output may overlap no input and no other output
  for (int32_t i = 0; i < b->count; ++i) {
    const size_t bytes_i = (size_t)(p[i].n * p[i].n) * sizeof(float);
    for (int32_t j = 0; j < b->count; ++j) {
      const size_t bytes_j = (size_t)(p[j].n * p[j].n) * sizeof(float);
      if (overlap(p[i].C, bytes_i, p[j].A, bytes_j) || overlap(p[i].C, bytes_i, p[j].B, bytes_j))
        return SPAMM_ERR_INVALID_ARG;
      if (j != i && overlap(p[i].C, bytes_i, p[j].C, bytes_j)) return SPAMM_ERR_INVALID_ARG;
    }
  }
  return SPAMM_OK;
}

InstRef batch_ref(const spamm_batch_s* b) {
  return make_ref(b->eng.insts.data(), b->insts_dev, b->count);
}

// The whole batch on one stream: norm maps, plan, multiply (with phase
// events when timing is on).
cudaError_t enqueue(spamm_batch_s* b, cudaStream_t s, bool timing) {
  const InstRef ref = batch_ref(b);
  cudaError_t e = timing ? cudaEventRecord(b->phase[0], s) : cudaSuccess;
  if (e == cudaSuccess)
    e = launch_normmap_jobs(b->jobs_dev, b->n_vec_jobs, b->units_vec, 2 * b->count - b->n_vec_jobs,
                            b->units_other, b->eng.leaf, b->status, s, b->eng.side, b->eng.fork,
                            b->eng.join);
  if (e == cudaSuccess && timing) e = cudaEventRecord(b->phase[1], s);
  if (e == cudaSuccess)
    e = engine_plan_multiply(b->eng, ref, b->status, s, timing ? b->phase[2] : nullptr,
                             timing ? b->phase[3] : nullptr);
  if (e == cudaSuccess && timing) e = cudaEventRecord(b->phase[4], s);
  return e;
}

void destroy_graph(spamm_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void release(spamm_batch_s* b) {
  destroy_graph(b);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->upload_done) cudaEventDestroy(b->upload_done);
  for (cudaEvent_t& ev : b->phase)
    if (ev) cudaEventDestroy(ev);
  if (b->staging) cudaFreeHost(b->staging);
  engine_free(b->eng);
  delete b;
}

}  // namespace

extern "C" {

spamm_status_t spamm_batch_workspace_size(const int64_t* n, int32_t count, int32_t leaf,
                                          spamm_precision_t precision, size_t* bytes) {
  if (!bytes) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = check_shapes(n, count, leaf, precision);
  if (st != SPAMM_OK) return st;
  std::vector<Inst> v = shape_table(n, count, leaf);
  const size_t extra = batch_extra(v, nullptr, nullptr, nullptr);
  *bytes = engine_layout(v, leaf, precision, extra, nullptr, nullptr, nullptr);
  return SPAMM_OK;
}

spamm_status_t spamm_batch_create(spamm_batch_t* batch, const int64_t* n, int32_t count,
                                  int32_t leaf, spamm_precision_t precision, int32_t flags,
                                  void* workspace, size_t ws_bytes) {
  if (!batch) return SPAMM_ERR_INVALID_ARG;
  *batch = nullptr;
  spamm_status_t st = check_shapes(n, count, leaf, precision);
  if (st != SPAMM_OK) return st;
  if (flags & ~(SPAMM_BATCH_GRAPH | SPAMM_BATCH_DYNAMIC | SPAMM_BATCH_TIMING | SPAMM_BATCH_GROUPS))
    return SPAMM_ERR_INVALID_ARG;
  if ((flags & SPAMM_BATCH_DYNAMIC) && (flags & SPAMM_BATCH_GROUPS)) return SPAMM_ERR_INVALID_ARG;
  spamm_batch_s* b = new (std::nothrow) spamm_batch_s();
  if (!b) return SPAMM_ERR_NO_MEMORY;
  b->count = count;
  b->flags = flags;
  b->n.assign(n, n + count);
  std::vector<Inst> v = shape_table(n, count, leaf);
  size_t norm_bytes = 0;
  const size_t extra = batch_extra(v, &norm_bytes, &b->table_bytes, &b->insts_offset);
  st = engine_init(b->eng, std::move(v), leaf, precision, extra, workspace, ws_bytes);
  if (st != SPAMM_OK) {
    delete b;
    return st;
  }
  b->eng.schedule = (flags & SPAMM_BATCH_DYNAMIC)  ? kScheduleDynamic
                    : (flags & SPAMM_BATCH_GROUPS) ? kScheduleGroups
                                                   : kScheduleStatic;
  char* base = static_cast<char*>(b->eng.base);
  b->normA = reinterpret_cast<double*>(base);
  b->normB = reinterpret_cast<double*>(base + norm_bytes);
  b->jobs_dev = reinterpret_cast<NormJob*>(base + 2 * norm_bytes);
  b->insts_dev = reinterpret_cast<Inst*>(base + 2 * norm_bytes + b->insts_offset);
  // norm-map jobs: operands are 16-byte aligned, so rows are iff n % 4 == 0;
  // those jobs come first in the table, each part with its own unit count
  b->job_slot.resize(2 * (size_t)count);
  b->job_unit0.resize(2 * (size_t)count);
  int slot = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool vec_pass = pass == 0;
    int64_t units = 0;
    for (int32_t i = 0; i < count; ++i) {
      if (((n[i] % 4) == 0) != vec_pass) continue;
      for (int op = 0; op < 2; ++op) {
        NormJob j{};
        j.rows = j.cols = j.ld = n[i];
        j.vec = vec_pass ? 1 : 0;
        b->job_slot[2 * i + op] = slot++;
        b->job_unit0[2 * i + op] = (int)units;
        units += normjob_shape(j, leaf);
        if (units >= ((int64_t)1 << 31)) {
          release(b);
          return SPAMM_ERR_UNSUPPORTED;
        }
      }
    }
    if (vec_pass) {
      b->n_vec_jobs = slot;
      b->units_vec = (int)units;
    } else {
      b->units_other = (int)units;
    }
  }
  b->last.assign(b->table_bytes, 0);
  b->status = device_status_word();   // bounded waits of the norm map and the multiply
  if (!b->status) {
    release(b);
    return SPAMM_ERR_NO_MEMORY;
  }
  if (flags & SPAMM_BATCH_TIMING) {
    for (cudaEvent_t& ev : b->phase) {
      if (cudaEventCreate(&ev) != cudaSuccess) {
        (void)cudaGetLastError();
        release(b);
        return SPAMM_ERR_CUDA;
      }
    }
  }
  if (cudaMallocHost(&b->staging, b->table_bytes) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->upload_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    (void)cudaGetLastError();
    if (b->staging == nullptr) {
      release(b);
      return SPAMM_ERR_NO_MEMORY;
    }
    release(b);
    return SPAMM_ERR_CUDA;
  }
  *batch = b;
  return SPAMM_OK;
}

spamm_status_t spamm_batch_destroy(spamm_batch_t batch) {
  if (!batch) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = SPAMM_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) st = SPAMM_ERR_CUDA;
  release(batch);
  return st;
}

}  // extern "C"

namespace {

// Fills the instance and norm-map job tables for `problems` and uploads them
// when they changed.  targets (per instance, may be null) overrides
// target_rel_err for tau prediction.
spamm_status_t upload_tables(spamm_batch_s* b, const spamm_problem_t* problems,
                             double target_rel_err, const double* targets, cudaStream_t s) {
  Engine& e = b->eng;
  const bool split = uses_split_flags(e.precision);
  const double u = hi_unit(e.precision);
  std::vector<char> tab(b->table_bytes, 0);
  NormJob* jobs = reinterpret_cast<NormJob*>(tab.data());
  for (int32_t i = 0; i < b->count; ++i) {
    Inst& in = e.insts[i];
    in.A = problems[i].A;
    in.B = problems[i].B;
    in.C = problems[i].C;
    in.nA = b->normA + in.ablk0;
    in.nB = b->normB + in.bblk0;
    in.nC = nullptr;
    in.T = make_tau_screen(targets ? 0.0 : problems[i].tau);
    in.band = 0;
    in.split = split ? 1 : 0;
    in.quant = is_tensor_mode(e.precision) ? 1 : 0;
    in.target_rel = targets ? targets[i] : (split ? target_rel_err : 0.0);
    in.c1 = split ? 2.0 * u + u * u : 0.0;
    for (int op = 0; op < 2; ++op) {
      NormJob& j = jobs[b->job_slot[2 * i + op]];
      j.X = op ? in.B : in.A;
      j.out = op ? b->normB + in.bblk0 : b->normA + in.ablk0;
      j.rows = j.cols = j.ld = in.n;
      j.vec = (in.n % 4) == 0 ? 1 : 0;
      (void)normjob_shape(j, e.leaf);
      j.unit0 = b->job_unit0[2 * i + op];
    }
  }
  std::memcpy(tab.data() + b->insts_offset, e.insts.data(), (size_t)b->count * sizeof(Inst));
  // upload only what changed since the last run (the staging buffer is reused
  // once the previous copy has read it)
  if (!b->uploaded_once || std::memcmp(tab.data(), b->last.data(), b->table_bytes) != 0) {
    SPAMM_CUDA_TRY(cudaEventSynchronize(b->upload_done));
    std::memcpy(b->staging, tab.data(), b->table_bytes);
    SPAMM_CUDA_TRY(cudaMemcpyAsync(b->jobs_dev, b->staging, b->table_bytes,
                                   cudaMemcpyHostToDevice, s));
    SPAMM_CUDA_TRY(cudaEventRecord(b->upload_done, s));
    b->last.swap(tab);
    b->uploaded_once = true;
  }
  return SPAMM_OK;
}

}  // namespace

extern "C" {

spamm_status_t spamm_batch_run(spamm_batch_t b, const spamm_problem_t* problems,
                               double target_rel_err, void* stream) {
  if (!b) return SPAMM_ERR_INVALID_ARG;
  spamm_status_t st = check_problems(b, problems);
  if (st != SPAMM_OK) return st;
  Engine& e = b->eng;
  if (uses_split_flags(e.precision) && !(target_rel_err >= 0.0)) return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  st = upload_tables(b, problems, target_rel_err, nullptr, s);
  if (st != SPAMM_OK) return st;

  cudaError_t err = cudaSuccess;
  const bool timing = (b->flags & SPAMM_BATCH_TIMING) != 0;
  if ((b->flags & SPAMM_BATCH_GRAPH) && !timing) {
    // every kernel argument is a pointer into the workspace or a grid size
    // fixed at creation, so one capture serves every later run
    if (!b->exec) {
      err = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
      if (err == cudaSuccess) {
        const cudaError_t e1 = enqueue(b, b->main, false);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
        err = e1 != cudaSuccess ? e1 : e2;
        if (err == cudaSuccess) {
          b->graph = g;
          err = cudaGraphInstantiate(&b->exec, g, 0);
        } else if (g) {
          cudaGraphDestroy(g);
        }
      }
      if (err != cudaSuccess) destroy_graph(b);
    }
    if (err == cudaSuccess) err = cudaEventRecord(b->ev_in, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(b->main, b->ev_in, 0);
    if (err == cudaSuccess) err = cudaGraphLaunch(b->exec, b->main);
    if (err == cudaSuccess) err = cudaEventRecord(b->ev_out, b->main);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, b->ev_out, 0);
  } else {
    err = enqueue(b, s, timing);
    b->timed = timing && err == cudaSuccess;
  }
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  return SPAMM_OK;
}

spamm_status_t spamm_batch_tau_predict(spamm_batch_t b, const spamm_problem_t* problems,
                                       const double* targets, const float* weights,
                                       double* taus, void* stream) {
  if (!b || !problems || !targets || !weights || !taus) return SPAMM_ERR_INVALID_ARG;
  for (int32_t i = 0; i < b->count; ++i) {   // only A, B and n are read
    const spamm_problem_t& q = problems[i];
    if (q.n != b->n[i] || !q.A || !q.B || !aligned16(q.A) || !aligned16(q.B))
      return SPAMM_ERR_INVALID_ARG;
  }
  spamm_status_t st = SPAMM_OK;
  for (int32_t i = 0; i < b->count; ++i)
    if (!(targets[i] > 0.0) || std::isinf(targets[i])) return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  st = upload_tables(b, problems, 0.0, targets, s);
  if (st != SPAMM_OK) return st;
  const InstRef ref = batch_ref(b);
  cudaError_t err = launch_normmap_jobs(b->jobs_dev, b->n_vec_jobs, b->units_vec,
                                        2 * b->count - b->n_vec_jobs, b->units_other, b->eng.leaf,
                                        b->status, s);
  if (err == cudaSuccess) err = run_histogram(ref, b->eng.buf, s);
  if (err == cudaSuccess) err = launch_tau_from_hist(ref, weights, b->eng.feat_dev, b->eng.tau_dev, s);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    return SPAMM_ERR_CUDA;
  }
  SPAMM_CUDA_TRY(cudaMemcpyAsync(taus, b->eng.tau_dev, (size_t)b->count * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

spamm_status_t spamm_batch_stats(spamm_batch_t b, spamm_stats_t* stats, void* stream) {
  if (!b || !stats) return SPAMM_ERR_INVALID_ARG;
  std::vector<PlanDevice> h((size_t)b->count);
  const cudaStream_t s = (cudaStream_t)stream;
  SPAMM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->eng.buf.pd, h.size() * sizeof(PlanDevice),
                                 cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int32_t i = 0; i < b->count; ++i) fill_stats(h[i], b->eng.leaf, b->eng.insts[i].bm, &stats[i]);
  return SPAMM_OK;
}

spamm_status_t spamm_batch_export(spamm_batch_t b, int32_t index, double* normA, double* normB,
                                  int32_t* tile_ptr, uint16_t* k_idx, int64_t cap, void* stream) {
  if (!b || index < 0 || index >= b->count) return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  const Inst& in = b->eng.insts[index];
  const int64_t tiles = (int64_t)in.bm * in.bn;
  const PlanBuffers& pb = b->eng.buf;
  if (normA)
    SPAMM_CUDA_TRY(cudaMemcpyAsync(normA, b->normA + in.ablk0, (size_t)tiles * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
  if (normB)
    SPAMM_CUDA_TRY(cudaMemcpyAsync(normB, b->normB + in.bblk0, (size_t)tiles * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return export_queues(pb, in, tile_ptr, k_idx, cap, s);
}

spamm_status_t spamm_batch_timings(spamm_batch_t b, float* ms) {
  if (!b || !ms) return SPAMM_ERR_INVALID_ARG;
  if (!(b->flags & SPAMM_BATCH_TIMING) || !b->timed) return SPAMM_ERR_INVALID_ARG;
  SPAMM_CUDA_TRY(cudaEventSynchronize(b->phase[4]));
  for (int q = 0; q < 4; ++q)
    SPAMM_CUDA_TRY(cudaEventElapsedTime(&ms[q], b->phase[q], b->phase[q + 1]));
  return SPAMM_OK;
}

spamm_status_t spamm_batch_autotune(const spamm_problem_t* problems, int32_t count,
                                    spamm_precision_t precision, double target_rel_err,
                                    int32_t reps, void* stream, spamm_tune_t* best,
                                    spamm_tune_t* results, int32_t* nresults) {
  if (!problems || count < 1 || !best || reps < 1) return SPAMM_ERR_INVALID_ARG;
  std::vector<int64_t> n((size_t)count);
  for (int32_t i = 0; i < count; ++i) n[i] = problems[i].n;
  const cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> leaves = precision == SPAMM_FP32 ? std::vector<int32_t>{32, 64, 128}
                                                        : std::vector<int32_t>{64, 128};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return SPAMM_ERR_CUDA;
  }
  spamm_status_t st = SPAMM_OK;
  int32_t nres = 0;
  best->leaf = 0;
  best->flags = 0;
  best->ms = -1.0f;
  for (int32_t leaf : leaves) {
    for (int32_t sched : {0, SPAMM_BATCH_DYNAMIC, SPAMM_BATCH_GROUPS}) {
      // the grouped multiply exists for BF16 and FP16 at leaf 128 only
      if (sched == SPAMM_BATCH_GROUPS &&
          !(leaf == 128 && (precision == SPAMM_BF16 || precision == SPAMM_FP16)))
        continue;
      spamm_tune_t r{leaf, SPAMM_BATCH_GRAPH | sched, -1.0f};
      spamm_batch_t b = nullptr;
      spamm_status_t cs = spamm_batch_create(&b, n.data(), count, leaf, precision, r.flags,
                                             nullptr, 0);
      if (cs == SPAMM_OK) {
        std::vector<float> t;
        // first run captures the graph, second warms it; then `reps` timed runs
        for (int32_t q = 0; q < reps + 2 && cs == SPAMM_OK; ++q) {
          if (q >= 2 && cudaEventRecord(e0, s) != cudaSuccess) cs = SPAMM_ERR_CUDA;
          if (cs == SPAMM_OK) cs = spamm_batch_run(b, problems, target_rel_err, stream);
          if (q >= 2 && cs == SPAMM_OK) {
            float ms = 0.0f;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
              cs = SPAMM_ERR_CUDA;
            t.push_back(ms);
          }
        }
        if (cs == SPAMM_OK && !t.empty()) {
          std::sort(t.begin(), t.end());
          r.ms = t[t.size() / 2];
        }
        const spamm_status_t ds = spamm_batch_destroy(b);
        if (cs == SPAMM_OK) cs = ds;
      }
      if (cs != SPAMM_OK && cs != SPAMM_ERR_NO_MEMORY && cs != SPAMM_ERR_UNSUPPORTED) {
        st = cs;   // a real failure ends the search
      }
      if (results && nresults && nres < *nresults) results[nres] = r;
      ++nres;
      if (r.ms >= 0.0f && (best->ms < 0.0f || r.ms < best->ms)) *best = r;
      if (st != SPAMM_OK) break;
    }
    if (st != SPAMM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (nresults) *nresults = nres;
  if (st == SPAMM_OK && best->ms < 0.0f) st = SPAMM_ERR_NO_MEMORY;
  return st;
}

spamm_status_t spamm_multiply_batched(const spamm_problem_t* problems, int32_t count, int32_t leaf,
                                      spamm_precision_t precision, double target_rel_err,
                                      spamm_stats_t* stats, void* stream) {
  if (!problems || count < 1) return SPAMM_ERR_INVALID_ARG;
  std::vector<int64_t> n((size_t)count);
  for (int32_t i = 0; i < count; ++i) n[i] = problems[i].n;
  spamm_batch_t b = nullptr;
  spamm_status_t st = spamm_batch_create(&b, n.data(), count, leaf, precision, 0, nullptr, 0);
  if (st != SPAMM_OK) return st;
  st = spamm_batch_run(b, problems, target_rel_err, stream);
  if (st == SPAMM_OK && stats) st = spamm_batch_stats(b, stats, stream);
  if (st == SPAMM_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    st = SPAMM_ERR_CUDA;
  const spamm_status_t st2 = spamm_batch_destroy(b);
  return st != SPAMM_OK ? st : st2;
}

}  // extern "C"
