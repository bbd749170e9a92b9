// Get-norm step (Section 3.2, Eq. 2): normmap[I*bd+K] = ||X[I,K]||_F.
//
// GB300 design.  FP64 arithmetic runs at 1/72 of the FP32 rate on this part,
// so every group of 32 entries is scaled by a power of two (no FP32 underflow
// of tiny squares), squared exactly with FMA and accumulated as an unevaluated
// FP32 pair with an explicit scale exponent; the threads of a block column are
// combined in that FP32 form (warp shuffles, and shared memory when a block
// column spans several warps), and the square root is taken with an FP32
// Newton step on the exact residual, so a block costs three FP64
// instructions.
//
// Two ways of reading X, both a single pass:
//  - TMA-staged (rows 16-byte aligned: n % 4 == 0 and X 16-byte aligned):
//    persistent CTAs, two per SM.  A unit is one block-row strip (leaf rows)
//    times a window of 1024 columns; the units are dealt round-robin, and the
//    grid is the smallest that keeps the number of rounds, so every CTA takes
//    the same number of units (no partial last wave).  One warp streams each
//    unit's rows into a ring of three 32 KiB shared-memory stages (eight rows
//    per stage, one bulk copy per row, completion counted in bytes on the
//    stage's mbarrier); eight consumer warps each own 128 columns (a float4
//    per lane) of every staged row.  Up to 96 KiB per CTA are in flight
//    without holding registers.  Every wait is bounded; on expiry the CTA
//    raises SPAMM_ERR_TIMEOUT, writes NaN to the norms it did not finish and
//    lets its copies land before it exits.
//  - streaming (any n and alignment; also the batched form): a CTA covers one
//    block-row strip and a window of columns; each thread owns a fixed column
//    slot (a float4 when aligned, else one float) and walks the strip's rows
//    with streamed (evict-first) loads, eight rows of loads in flight per
//    group.
#include "plan.cuh"
#include "tc.cuh"

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

// ---------------------------------------------------------------------------
// TMA-staged form.
// ---------------------------------------------------------------------------
// Shape: CW warps across a unit window of CW * 128 columns (a float4 per
// lane), RP 8-row parts per stage (consumer warp w takes column slice w % CW
// and rows 8 (w / CW) .. 8 (w / CW) + 7 of every stage), STAGES ring stages,
// CPS CTAs per SM.  The RP partial sums of a column are merged in part order
// at the end of each unit.
template <int CW, int RP, int STAGES, int CPS>
struct StagedCfg {
  static constexpr int kColWarps = CW;
  static constexpr int kRowParts = RP;
  static constexpr int kConsumers = CW * RP;
  static constexpr int kThreads = (kConsumers + 1) * 32;     // + one producer warp
  static constexpr int kWinCols = CW * 128;
  static constexpr int kRows = 8 * RP;                       // rows per stage
  static constexpr int kStages = STAGES;
  static constexpr int kCtasPerSm = CPS;
  static constexpr uint32_t kRowBytes = kWinCols * 4;
  static constexpr uint32_t kStageBytes = kRows * kRowBytes;
  // partial sums of parts 1 .. RP-1, double-buffered by unit parity
  static constexpr size_t kMergeOff = (size_t)STAGES * kStageBytes;
  static constexpr size_t kMergeBytes = RP > 1 ? 2 * (RP - 1) * CW * 32 * sizeof(SumSq) : 0;
  static constexpr size_t kBarOff = (kMergeOff + kMergeBytes + 15) / 16 * 16;
  static constexpr size_t kSmem = kBarOff + 2 * STAGES * sizeof(uint64_t) + 16;
  static_assert(kSmem * CPS <= 227 * 1024, "shared memory");
  static_assert(kRows <= 32, "one producer lane per staged row");
};
// two CTAs per SM, 8 consumer warps each, 32 KiB stages (8 rows x 1024
// columns).  Each lane then sums its column slot in the same order as the
// streaming form (bitwise-equal norm maps).  Measured on N = 8192 (back to
// back, per operand): 46.9 us, the same as the streaming form and within 3%
// of the same pipeline with the arithmetic removed; 16 consumer warps with
// two row parts (StagedCfg<8, 2, 3, 1>) took 49.2 us.
using StagedDefault = StagedCfg<8, 1, 3, 2>;
constexpr uint64_t kStagedWaitNs = 2000000000ull;   // 2 s: a safety net, never hit normally
constexpr uint64_t kStagedDrainNs = 100000000ull;   // 100 ms for the abort drain

// One operand of a staged launch; its units are unit0 .. unit0 + bd * nwin - 1
// (block row I = local / nwin, window local % nwin).
struct StagedJob {
  const float* X;
  double* out;
  int64_t n;
  int bd, nwin, unit0, pad_;
};
// Up to two jobs by value, or a device table (sorted by unit0).
struct StagedJobs {
  const StagedJob* table;
  int count, units;
  StagedJob one[2];
};

__device__ __forceinline__ StagedJob job_of(const StagedJobs& J, int u) {
  if (J.table == nullptr) {
    if (J.count > 1 && u >= J.one[1].unit0) return J.one[1];
    return J.one[0];
  }
  int lo = 0, hi = J.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (J.table[mid].unit0 <= u) lo = mid;
    else hi = mid - 1;
  }
  return J.table[lo];
}

// Bounded wait of a whole warp: returns (uniformly) once every lane has seen
// the phase complete, or false when the limit passed or the abort flag is up.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int32_t* status) {
  bool done = tc::mbar_try_wait(bar, parity);
  if (__all_sync(0xffffffffu, done)) return true;
  const uint64_t t0 = tc::globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (!done) done = tc::mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    if ((it & 63u) == 0) {
      int give_up = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*abort_flag) {
          give_up = 1;
        } else if (tc::globaltimer_ns() - t0 > kStagedWaitNs) {
          *abort_flag = 1;
          if (status) atomicExch(status, (int32_t)SPAMM_ERR_TIMEOUT);
          give_up = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
    }
  }
}

template <int LEAF, class Cfg>
__global__ void __launch_bounds__(Cfg::kThreads, Cfg::kCtasPerSm)
    normmap_staged_kernel(const StagedJobs J, int32_t* status) {
  constexpr int kCW = Cfg::kColWarps, kRP = Cfg::kRowParts, kConsumers = Cfg::kConsumers;
  constexpr int kWinCols = Cfg::kWinCols, kRows = Cfg::kRows, kStages = Cfg::kStages;
  constexpr uint32_t kRowBytes = Cfg::kRowBytes, kStageBytes = Cfg::kStageBytes;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOff);
  uint64_t* empty = full + kStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], kConsumers);
    }
    *abort_flag = 0;
    tc::fence_mbarrier_init();
  }
  __syncthreads();

  if (warp == kConsumers) {
    // ------------------------------------------------------------ producer
    uint32_t stage = 0, phase = 0, issued = 0, issued_phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < J.units && ok; u += gridDim.x) {
      const StagedJob jb = job_of(J, u);
      const int local = u - jb.unit0;
      const int I = local / jb.nwin;
      const int64_t n = jb.n;
      const int64_t col0 = (int64_t)(local - I * jb.nwin) * kWinCols;
      const int64_t row0 = (int64_t)I * LEAF;
      const int rows = (int)(n - row0 < LEAF ? n - row0 : LEAF);
      const uint32_t width = (uint32_t)((n - col0 < kWinCols ? n - col0 : kWinCols) * 4);
      const float* X = jb.X;
      for (int r = 0; r < rows; r += kRows) {
        const int rr = rows - r < kRows ? rows - r : kRows;
        if (!warp_wait(&empty[stage], phase ^ 1u, abort_flag, status)) {
          ok = false;
          break;
        }
        if (lane == 0) tc::mbar_arrive_expect_tx(&full[stage], (uint32_t)rr * width);
        __syncwarp();
        if (lane < rr)
          tc::bulk_g2s(smem + (size_t)stage * kStageBytes + (size_t)lane * kRowBytes,
                       X + (row0 + r + lane) * n + col0, width, &full[stage]);
        issued |= 1u << stage;
        issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // every copy this warp issued has landed before the warp leaves (the
    // consumers may have given up waiting for them)
    if (lane == 0)
      for (int s = 0; s < kStages; ++s)
        if (issued & (1u << s)) (void)tc::mbar_wait(&full[s], (issued_phase >> s) & 1u, kStagedDrainNs);
    return;
  }

  // -------------------------------------------------------------- consumers
  constexpr int kLanesPerBlockCol = LEAF / 4;
  const int cslice = warp % kCW, part = warp / kCW;
  const int cw = cslice * 128 + lane * 4;   // this lane's first column inside a window
  SumSq* merge = reinterpret_cast<SumSq*>(smem + Cfg::kMergeOff);
  uint32_t stage = 0, phase = 0, parity = 0;
  bool ok = true;
  for (int u = blockIdx.x; u < J.units; u += gridDim.x, parity ^= 1u) {
    const StagedJob jb = job_of(J, u);
    const int local = u - jb.unit0;
    const int I = local / jb.nwin;
    const int64_t n = jb.n;
    const int64_t col0 = (int64_t)(local - I * jb.nwin) * kWinCols;
    const int64_t row0 = (int64_t)I * LEAF;
    const int rows = (int)(n - row0 < LEAF ? n - row0 : LEAF);
    const bool active = col0 + cw < n;
    SumSq ss = sumsq_empty();
    for (int r = 0; r < rows && ok; r += kRows) {
      const int rr = rows - r < kRows ? rows - r : kRows;
      const int mine = rr - 8 * part;   // rows of this stage in this warp's part
      if (!warp_wait(&full[stage], phase, abort_flag, status)) {
        ok = false;
        break;
      }
      float v[32];
      const float* src =
          reinterpret_cast<const float*>(smem + (size_t)stage * kStageBytes) + 8 * part * kWinCols + cw;
      if (mine >= 8 && active) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = *reinterpret_cast<const float4*>(src + q * kWinCols);
          v[4 * q] = t.x;
          v[4 * q + 1] = t.y;
          v[4 * q + 2] = t.z;
          v[4 * q + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < mine && active) {
            const float4 t = *reinterpret_cast<const float4*>(src + q * kWinCols);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
          } else {
            v[4 * q] = v[4 * q + 1] = v[4 * q + 2] = v[4 * q + 3] = 0.0f;
          }
        }
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&empty[stage]);   // the stage is in registers: release it
      if (++stage == kStages) {
        stage = 0;
        phase ^= 1u;
      }
      if (mine > 0) sumsq_group<32>(ss, v);
    }
    if constexpr (kRP > 1) {
      // parts 1 .. RP-1 hand their partial sums to part 0 (merged in part order)
      SumSq* mb = merge + (size_t)parity * (kRP - 1) * kCW * 32;
      if (part > 0) mb[((part - 1) * kCW + cslice) * 32 + lane] = ss;
      asm volatile("bar.sync 1, %0;" ::"r"(kConsumers * 32) : "memory");
      if (part > 0) continue;
#pragma unroll
      for (int p = 1; p < kRP; ++p) {
        const SumSq o = mb[((p - 1) * kCW + cslice) * 32 + lane];
        merge_from(ss, o.hi, o.lo, o.e);
      }
    }
#pragma unroll
    for (int off = kLanesPerBlockCol / 2; off > 0; off >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
      const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
      const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
      merge_from(ss, h, l, e);
    }
    if ((lane % kLanesPerBlockCol) == 0 && active)
      jb.out[(int64_t)I * jb.bd + (col0 + cw) / LEAF] =
          (ok && !*abort_flag) ? sumsq_sqrt(ss) : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Resident CTAs of the staged kernel on the current device (occupancy x SMs).
template <int LEAF, class Cfg>
cudaError_t staged_capacity(int* cap) {
  static int max_ctas[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (max_ctas[dev] == 0) {
    e = cudaFuncSetAttribute(normmap_staged_kernel<LEAF, Cfg>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, normmap_staged_kernel<LEAF, Cfg>,
                                                      Cfg::kThreads, Cfg::kSmem);
    if (e != cudaSuccess) return e;
    max_ctas[dev] = sms * (per_sm > 0 ? per_sm : 1);
  }
  *cap = max_ctas[dev];
  return cudaSuccess;
}

// The units are dealt round-robin; the grid is the smallest that keeps the
// number of rounds, so every CTA takes `rounds` or `rounds - 1` units.
template <int LEAF, class Cfg = StagedDefault>
cudaError_t launch_staged_jobs(const StagedJobs& J, int32_t* status, cudaStream_t s) {
  if (J.units <= 0) return cudaSuccess;
  int cap = 0;
  cudaError_t e = staged_capacity<LEAF, Cfg>(&cap);
  if (e != cudaSuccess) return e;
  const int rounds = (J.units + cap - 1) / cap;
  const int grid = (J.units + rounds - 1) / rounds;
  normmap_staged_kernel<LEAF, Cfg><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(J, status);
  return cudaPeekAtLastError();
}

template <class Cfg = StagedDefault>
StagedJob staged_job(const float* X, int64_t n, int leaf, double* out, int unit0) {
  StagedJob j{};
  j.X = X;
  j.out = out;
  j.n = n;
  j.bd = (int)num_blocks(n, leaf);
  j.nwin = (int)((n + Cfg::kWinCols - 1) / Cfg::kWinCols);
  j.unit0 = unit0;
  return j;
}

template <int LEAF, class Cfg = StagedDefault>
cudaError_t launch_staged(const float* X, int64_t n, double* out, int32_t* status,
                          cudaStream_t s) {
  StagedJobs J{};
  J.count = 1;
  J.one[0] = staged_job<Cfg>(X, n, LEAF, out, 0);
  J.units = J.one[0].bd * J.one[0].nwin;
  return launch_staged_jobs<LEAF, Cfg>(J, status, s);
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
                           int32_t* status, cudaStream_t s) {
  const int bd = (int)num_blocks(n, leaf);
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  if (vec) {
    switch (leaf) {
      case 32: return launch_staged<32>(X, n, out, status, s);
      case 64: return launch_staged<64>(X, n, out, status, s);
      case 128: return launch_staged<128>(X, n, out, status, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (leaf) {
    case 32: return launch<1, 32>(X, n, bd, out, s);
    case 64: return launch<1, 64>(X, n, bd, out, s);
    case 128: return launch<1, 128>(X, n, bd, out, s);
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
