// Get-norm step (Section 3.2, Eq. 2): normmap[I*bc+K] = ||X[I,K]||_F for a
// rows x cols operand (leading dimension ld) with bc = ceil(cols / leaf).
//
// GB300 design.  FP64 arithmetic runs at 1/72 of the FP32 rate on this part,
// so every group of 32 entries is scaled by a power of two (no FP32 underflow
// of tiny squares), squared exactly with FMA and accumulated as an unevaluated
// FP32 pair with an explicit scale exponent; the lanes of a block column are
// combined in that FP32 form (warp shuffles, and shared memory when a block
// column spans several warps), and the square root is taken with an FP32
// Newton step on the exact residual, so a block costs three FP64
// instructions.
//
// One streaming pass over X, staged through shared memory by the TMA engine.
// Persistent CTAs, two per SM.  A unit is one block-row strip (leaf rows)
// times a window of columns; the units (of one operand, or of every operand
// of a batch) are dealt round-robin, and the grid is the smallest that keeps
// the number of rounds, so every CTA takes the same number of units (no
// partial last wave).  One producer warp streams each unit's rows into a ring
// of three shared-memory stages (one bulk copy per row, completion counted in
// bytes on the stage's mbarrier); eight consumer warps read the staged rows
// and accumulate, each lane one column slot over the strip's rows in groups
// of 32 entries.  Up to ~100 KiB per CTA are in flight without holding
// registers.  A lane owns 4 adjacent columns and takes 8 rows per group;
// windows of 1024 columns.  A row segment's bulk copy starts at the 128-byte
// boundary at or below its first entry (never before X) and ends at the one
// at or above its last (never past the last 16-byte boundary inside X), so
// every copy moves whole cache lines even when rows are not line-aligned (a
// copy at an odd offset ran at about 60% of the line-aligned rate); the
// producer records each row's offset into its copy, and the entries the copy
// carries from neighbouring rows are not read.  Rows 16-byte aligned
// (ld % 4 == 0): float4 reads.  Any other ld: scalar reads, each lane taking its
// 4 columns in a lane-dependent rotation so that the warp's reads hit 32
// different banks, and the matrix's last few entries past the last 16-byte
// boundary inside X read from global memory directly.
// Every wait is bounded; on expiry the CTA raises SPAMM_ERR_TIMEOUT, writes
// NaN to the norms it did not finish and lets its copies land before it exits.
#include <algorithm>

#include "plan.cuh"
#include "tc.cuh"

namespace spamm {
namespace {

__device__ __forceinline__ void merge_from(SumSq& a, float h, float l, int e) {
  if (e == kSumSqEmpty) {
    if (h != h) a.hi = h;   // NaN from an otherwise empty partner
  } else {
    sumsq_merge(a, h, l, e);
  }
}

// Shape of the staged kernel: ALIGNED (rows 16-byte aligned) or not, CW
// consumer warps across a window of CW * 128 columns (4 per lane), RP parts of
// 8 rows per stage (consumer warp w takes column slice w % CW and part w / CW
// of every stage; the parts' sums of a column are merged in part order at the
// end of a unit), STAGES ring stages, CPS CTAs per SM.
template <bool ALIGNED, int CW, int RP, int STAGES, int CPS>
struct StagedCfg {
  static constexpr bool kAligned = ALIGNED;
  static constexpr int kColWarps = CW;
  static constexpr int kRowParts = RP;
  static constexpr int kConsumers = CW * RP;
  static constexpr int kThreads = (kConsumers + 1) * 32;     // + one producer warp
  static constexpr int kWinCols = CW * 128;
  static constexpr int kRowsPerPart = 8;                     // one 32-entry group per lane
  static constexpr int kRows = kRowsPerPart * RP;            // rows per stage
  static constexpr int kStages = STAGES;
  static constexpr int kCtasPerSm = CPS;
  // a row copy spans up to 31 extra entries on each side (128-byte lines)
  static constexpr int kRowFloats = kWinCols + 64;
  static constexpr uint32_t kRowBytes = kRowFloats * 4;
  static constexpr uint32_t kStageBytes = kRows * kRowBytes;
  // partial sums of the other row parts, double-buffered by unit parity
  static constexpr size_t kMergeOff = (size_t)STAGES * kStageBytes;
  static constexpr size_t kMergeBytes = RP > 1 ? 2 * (size_t)kConsumers * 32 * sizeof(SumSq) : 0;
  static constexpr size_t kBarOff = (kMergeOff + kMergeBytes + 15) / 16 * 16;
  // per stage and row: the row's first entry's offset (in floats) into its copy
  static constexpr size_t kOffOff = kBarOff + 2 * STAGES * sizeof(uint64_t) + 16;
  static constexpr size_t kSmem = kOffOff + (size_t)STAGES * kRows * sizeof(int);
  static_assert(kSmem * CPS <= 227 * 1024, "shared memory");
  static_assert(kRows <= 32, "one producer lane per staged row");
  static_assert(kRowBytes % 16 == 0, "bulk-copy destinations 16-byte aligned");
};
// Two CTAs per SM, 8 consumer warps each, three stages of ~32 KiB.  Measured on
// N = 8192 (back to back, per operand): 46.9 us, the same as a plain float4
// streaming kernel and within 3% of the same pipeline with the arithmetic
// removed; 16 consumer warps with two row parts (StagedCfg<true, 8, 2, 3, 1>)
// took 49.2 us.  For rows not 16-byte aligned a plain streaming kernel with one
// column per thread took 74 us on N = 8191, a staged one-column-per-lane
// mapping 64-86 us (its per-block lane merges cost as much as the sums).
using StagedAligned = StagedCfg<true, 8, 1, 3, 2>;
using StagedUnaligned = StagedCfg<false, 8, 1, 3, 2>;
constexpr uint64_t kStagedWaitNs = 2000000000ull;   // 2 s: a safety net, never hit normally
constexpr uint64_t kStagedDrainNs = 100000000ull;   // 100 ms for the abort drain

// Up to two jobs by value, or a device table (sorted by unit0).
struct StagedJobs {
  const NormJob* table;
  int count, units;
  NormJob one[2];
};

__device__ __forceinline__ NormJob job_of(const StagedJobs& J, int u) {
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
                                          int32_t* status, uint64_t limit_ns = kStagedWaitNs) {
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
        } else if (tc::globaltimer_ns() - t0 > limit_ns) {
          *abort_flag = 1;
          if (status) atomicExch(status, (int32_t)SPAMM_ERR_TIMEOUT);
          give_up = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
    }
  }
}

// Position of one unit: block row I, first row and column, rows in the strip
// and the window's width in entries.
struct UnitPos {
  int I;
  int64_t row0, col0;
  int rows, width;
};

template <int LEAF, class Cfg>
__device__ __forceinline__ UnitPos unit_pos(const NormJob& jb, int u) {
  UnitPos p;
  const int local = u - jb.unit0;
  p.I = local / jb.nwin;
  p.col0 = (int64_t)(local - p.I * jb.nwin) * Cfg::kWinCols;
  p.row0 = (int64_t)p.I * LEAF;
  p.rows = (int)(jb.rows - p.row0 < LEAF ? jb.rows - p.row0 : LEAF);
  p.width = (int)(jb.cols - p.col0 < Cfg::kWinCols ? jb.cols - p.col0 : Cfg::kWinCols);
  return p;
}

// Entries X spans: from its first to its last entry, (rows - 1) * ld + cols.
__device__ __forceinline__ int64_t job_span(const NormJob& jb) {
  return (jb.rows - 1) * jb.ld + jb.cols;
}

template <int LEAF, class Cfg>
__global__ void __launch_bounds__(Cfg::kThreads, Cfg::kCtasPerSm)
    normmap_staged_kernel(const StagedJobs J, int32_t* status) {
  constexpr bool ALIGNED = Cfg::kAligned;
  constexpr int kCW = Cfg::kColWarps, kRP = Cfg::kRowParts, kConsumers = Cfg::kConsumers;
  constexpr int kRows = Cfg::kRows, kRowsPerPart = Cfg::kRowsPerPart, kStages = Cfg::kStages;
  constexpr int kRowFloats = Cfg::kRowFloats;
  constexpr uint32_t kRowBytes = Cfg::kRowBytes, kStageBytes = Cfg::kStageBytes;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOff);
  uint64_t* empty = full + kStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);
  int* offs = reinterpret_cast<int*>(smem + Cfg::kOffOff);
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
      const NormJob jb = job_of(J, u);
      const UnitPos p = unit_pos<LEAF, Cfg>(jb, u);
      const int64_t ld = jb.ld;
      const float* X = jb.X;
      for (int r = 0; r < p.rows; r += kRows) {
        const int rr = p.rows - r < kRows ? p.rows - r : kRows;
        if (!warp_wait(&empty[stage], phase ^ 1u, abort_flag, status)) {
          ok = false;
          break;
        }
        // lane q < rr copies row row0 + r + q: whole 128-byte lines, clipped
        // to X's first byte and to its last 16-byte boundary
        const uintptr_t xb = reinterpret_cast<uintptr_t>(X);
        const uintptr_t xend = xb + (uintptr_t)((job_span(jb) & ~(int64_t)3) * 4);
        uintptr_t a0 = 0, a1 = 0;
        if (lane < rr) {
          const uintptr_t b0 = xb + (uintptr_t)(((p.row0 + r + lane) * ld + p.col0) * 4);
          const uintptr_t b1 = b0 + (uintptr_t)p.width * 4u;
          a0 = b0 & ~(uintptr_t)127;
          if (a0 < xb) a0 = xb;
          a1 = (b1 + 127) & ~(uintptr_t)127;
          if (a1 > xend) a1 = xend;
          if (a1 < a0) a1 = a0;
          offs[stage * kRows + lane] = (int)((b0 - a0) >> 2);
        }
        const uint32_t bytes = (uint32_t)(a1 - a0);
        const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
        __syncwarp();   // the offsets are written before lane 0's arrive releases them
        if (lane == 0) tc::mbar_arrive_expect_tx(&full[stage], total);
        __syncwarp();
        if (bytes)
          tc::bulk_g2s(smem + (size_t)stage * kStageBytes + (size_t)lane * kRowBytes,
                       reinterpret_cast<const void*>(a0), bytes, &full[stage]);
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
  constexpr int kLanesPerBlockCol = LEAF / 4;   // <= 32: a block column is inside a warp
  const int cslice = warp % kCW, part = warp / kCW;
  const int cw = (cslice * 32 + lane) * 4;   // this lane's first column inside a window
  // unaligned rows: this lane reads its 4 columns in the order c0, c1, c2, c3
  // (rotated by lane / 8), so every scalar read of the warp hits 32 banks
  const int l8 = lane >> 3;
  const int c0 = l8 & 3, c1 = (l8 + 1) & 3, c2 = (l8 + 2) & 3, c3 = (l8 + 3) & 3;
  SumSq* merge = reinterpret_cast<SumSq*>(smem + Cfg::kMergeOff);
  uint32_t stage = 0, phase = 0, parity = 0;
  bool ok = true;
  for (int u = blockIdx.x; u < J.units; u += gridDim.x, parity ^= 1u) {
    const NormJob jb = job_of(J, u);
    const UnitPos p = unit_pos<LEAF, Cfg>(jb, u);
    const int64_t ld = jb.ld, cols = jb.cols;
    const bool active = p.col0 + cw < cols;
    SumSq ss = sumsq_empty();
    for (int r = 0; r < p.rows && ok; r += kRows) {
      const int rr = p.rows - r < kRows ? p.rows - r : kRows;
      const int mine = rr - kRowsPerPart * part;   // rows of this stage in this warp's part
      if (!warp_wait(&full[stage], phase, abort_flag, status)) {
        ok = false;
        break;
      }
      float v[32];
      const float* src = reinterpret_cast<const float*>(smem + (size_t)stage * kStageBytes) +
                         kRowsPerPart * part * kRowFloats + cw;
      const int* so = offs + stage * kRows + kRowsPerPart * part;   // the rows' offsets
      if constexpr (ALIGNED) {
        // rows 16-byte aligned: the offsets are multiples of 4 floats (zero
        // when every row starts on a line)
        if (mine >= kRowsPerPart && active && jb.lines) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(src + q * kRowFloats);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
          }
        } else if (mine >= kRowsPerPart && active) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(src + q * kRowFloats + so[q]);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (q < mine && active) {
              const float4 t = *reinterpret_cast<const float4*>(src + q * kRowFloats + so[q]);
              v[4 * q] = t.x;
              v[4 * q + 1] = t.y;
              v[4 * q + 2] = t.z;
              v[4 * q + 3] = t.w;
            } else {
              v[4 * q] = v[4 * q + 1] = v[4 * q + 2] = v[4 * q + 3] = 0.0f;
            }
          }
        }
      } else {
        const int64_t row_first = p.row0 + r + kRowsPerPart * part;
        const int64_t lim = job_span(jb) & ~(int64_t)3;   // entries past it: read from global
        const bool tail = p.row0 + r + rr == jb.rows && (jb.rows - 1) * ld + p.col0 + p.width > lim;
        // columns of this lane inside the matrix (4 except at its right edge)
        const int64_t left = cols - (p.col0 + cw);
        const int nv = left >= 4 ? 4 : (left > 0 ? (int)left : 0);
        if (mine >= kRowsPerPart && nv == 4 && !tail) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float* rp = src + q * kRowFloats + so[q];
            v[4 * q] = rp[c0];
            v[4 * q + 1] = rp[c1];
            v[4 * q + 2] = rp[c2];
            v[4 * q + 3] = rp[c3];
          }
        } else if (!tail) {   // a partial stage or the lane at the right edge: masked reads
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float* rp = src + q * kRowFloats + (q < mine ? so[q] : 0);
            v[4 * q] = (q < mine && c0 < nv) ? rp[c0] : 0.0f;
            v[4 * q + 1] = (q < mine && c1 < nv) ? rp[c1] : 0.0f;
            v[4 * q + 2] = (q < mine && c2 < nv) ? rp[c2] : 0.0f;
            v[4 * q + 3] = (q < mine && c3 < nv) ? rp[c3] : 0.0f;
          }
        } else {   // the matrix's last stage: its last entries come from global memory
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float* rp = src + q * kRowFloats + (q < mine ? so[q] : 0);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int c = (l8 + jj) & 3;
              float x = 0.0f;
              if (q < mine && c < nv) {
                const int64_t e = (row_first + q) * ld + p.col0 + cw + c;
                x = e < lim ? rp[c] : __ldg(jb.X + e);
              }
              v[4 * q + jj] = x;
            }
          }
        }
      }
      if constexpr (ALIGNED) {
        // a rectangular operand whose width is not a multiple of 4: the lane at the right
        // edge read entries past the last column (the gap up to the leading dimension), and
        // the matrix's last few entries, past its last 16-byte boundary, were not copied:
        // those come from global memory
        const int64_t left = cols - (p.col0 + cw);
        if (left < 4 && active) {
          const int64_t lim = job_span(jb) & ~(int64_t)3;
          const int64_t row_first = p.row0 + r + kRowsPerPart * part;
#pragma unroll
          for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              if (c >= left) {
                v[4 * q + c] = 0.0f;
              } else if (q < mine) {
                const int64_t e = (row_first + q) * ld + p.col0 + cw + c;
                if (e >= lim) v[4 * q + c] = __ldg(jb.X + e);
              }
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
    // the lanes of a block column (inside this warp)
#pragma unroll
    for (int off = kLanesPerBlockCol / 2; off > 0; off >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
      const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
      const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
      merge_from(ss, h, l, e);
    }
    if constexpr (kRP > 1) {
      // the other row parts hand their sums to part 0 (merged in part order)
      SumSq* mb = merge + (size_t)parity * kConsumers * 32;
      mb[warp * 32 + lane] = ss;
      asm volatile("bar.sync 1, %0;" ::"r"(kConsumers * 32) : "memory");
      if (part > 0) continue;
#pragma unroll
      for (int pp = 1; pp < kRP; ++pp) {
        const SumSq o = mb[(pp * kCW + cslice) * 32 + lane];
        merge_from(ss, o.hi, o.lo, o.e);
      }
    }
    if ((lane % kLanesPerBlockCol) == 0 && active)
      jb.out[(int64_t)p.I * jb.bc + (p.col0 + cw) / LEAF] =
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
// share in (0, 1]: the fraction of the resident CTAs this launch may take (the
// rest go to a launch running beside it).
template <int LEAF, class Cfg>
cudaError_t launch_staged_jobs(const StagedJobs& J, int32_t* status, cudaStream_t s,
                               double share = 1.0) {
  if (J.units <= 0) return cudaSuccess;
  int cap = 0;
  cudaError_t e = staged_capacity<LEAF, Cfg>(&cap);
  if (e != cudaSuccess) return e;
  cap = std::max(1, (int)(cap * share));
  const int rounds = (J.units + cap - 1) / cap;
  const int grid = (J.units + rounds - 1) / rounds;
  normmap_staged_kernel<LEAF, Cfg><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(J, status);
  return cudaPeekAtLastError();
}

template <class Cfg>
cudaError_t launch_leaf(int leaf, const StagedJobs& J, int32_t* status, cudaStream_t s,
                        double share = 1.0) {
  switch (leaf) {
    case 32: return launch_staged_jobs<32, Cfg>(J, status, s, share);
    case 64: return launch_staged_jobs<64, Cfg>(J, status, s, share);
    case 128: return launch_staged_jobs<128, Cfg>(J, status, s, share);
    default: return cudaErrorInvalidValue;
  }
}

// Self-test of the norm map's warp-wide bounded wait: one warp waits, with a
// short limit, on an mbarrier phase that nothing completes.  out[0] = 1 if the
// wait returned false, out[1] = the abort flag, out[2] = elapsed nanoseconds.
__global__ void normmap_wait_selftest_kernel(int32_t* status, uint64_t limit_ns, long long* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);   // phase 0 completes only on an arrival, which never comes
    abort_flag = 0;
    tc::fence_mbarrier_init();
  }
  __syncwarp();
  const uint64_t t0 = tc::globaltimer_ns();
  const bool ok = warp_wait(&bar, 0u, &abort_flag, status, limit_ns);
  const uint64_t t1 = tc::globaltimer_ns();
  if (threadIdx.x == 0) {
    out[0] = ok ? 0 : 1;
    out[1] = abort_flag;
    out[2] = (long long)(t1 - t0);
  }
}

}  // namespace

cudaError_t launch_normmap_wait_selftest(int32_t* status, uint64_t limit_ns, long long* out,
                                         cudaStream_t s) {
  normmap_wait_selftest_kernel<<<1, 32, 0, s>>>(status, limit_ns, out);
  return cudaPeekAtLastError();
}

int normjob_shape(NormJob& j, int leaf) {
  j.br = (int)num_blocks(j.rows, leaf);
  j.bc = (int)num_blocks(j.cols, leaf);
  j.lines = (j.ld % 32) == 0 && (reinterpret_cast<uintptr_t>(j.X) % 128) == 0 ? 1 : 0;
  const int win = j.vec ? StagedAligned::kWinCols : StagedUnaligned::kWinCols;
  j.nwin = (int)((j.cols + win - 1) / win);
  return j.br * j.nwin;
}

cudaError_t launch_normmap_rect(const float* X, int64_t rows, int64_t cols, int64_t ld,
                                int32_t leaf, double* out, int32_t* status, cudaStream_t s) {
  if (reinterpret_cast<uintptr_t>(X) % 16) return cudaErrorMisalignedAddress;   // bulk copies
  StagedJobs J{};
  J.count = 1;
  NormJob& j = J.one[0];
  j.X = X;
  j.out = out;
  j.rows = rows;
  j.cols = cols;
  j.ld = ld;
  j.vec = (ld % 4) == 0;
  j.unit0 = 0;
  J.units = normjob_shape(j, leaf);
  return j.vec ? launch_leaf<StagedAligned>(leaf, J, status, s)
               : launch_leaf<StagedUnaligned>(leaf, J, status, s);
}

cudaError_t launch_normmap(const float* X, int64_t n, int32_t leaf, double* out, int32_t* status,
                           cudaStream_t s) {
  return launch_normmap_rect(X, n, n, n, leaf, out, status, s);
}

cudaError_t launch_normmap_pair(const float* A, const float* B, int64_t n, int32_t leaf,
                                double* outA, double* outB, int32_t* status, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16)
    return cudaErrorMisalignedAddress;   // bulk copies
  StagedJobs J{};
  J.count = 2;
  const bool vec = (n % 4) == 0;
  int units = 0;
  for (int q = 0; q < 2; ++q) {
    NormJob& j = J.one[q];
    j.X = q ? B : A;
    j.out = q ? outB : outA;
    j.rows = j.cols = j.ld = n;
    j.vec = vec;
    j.unit0 = units;
    units += normjob_shape(j, leaf);
  }
  J.units = units;
  return vec ? launch_leaf<StagedAligned>(leaf, J, status, s)
             : launch_leaf<StagedUnaligned>(leaf, J, status, s);
}

cudaError_t launch_normmap_jobs(const NormJob* dev_jobs, int n_vec, int units_vec, int n_other,
                                int units_other, int leaf, int32_t* status, cudaStream_t s,
                                cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  StagedJobs Jv{}, Jo{};
  Jv.table = dev_jobs;
  Jv.count = n_vec;
  Jv.units = units_vec;
  Jo.table = dev_jobs + n_vec;
  Jo.count = n_other;
  Jo.units = units_other;
  cudaError_t e = cudaSuccess;
  if (n_vec > 0 && n_other > 0 && side && fork && join) {
    // both kinds at once, on two streams, the resident CTAs shared in proportion
    // to the units: they end together instead of one after the other
    const double fv = (double)units_vec / ((double)units_vec + (double)units_other);
    e = cudaEventRecord(fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
    if (e == cudaSuccess) e = launch_leaf<StagedUnaligned>(leaf, Jo, status, side, 1.0 - fv);
    if (e == cudaSuccess) e = cudaEventRecord(join, side);
    if (e == cudaSuccess) e = launch_leaf<StagedAligned>(leaf, Jv, status, s, fv);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
    return e;
  }
  if (n_vec > 0) e = launch_leaf<StagedAligned>(leaf, Jv, status, s);
  if (e == cudaSuccess && n_other > 0) e = launch_leaf<StagedUnaligned>(leaf, Jo, status, s);
  return e;
}

}  // namespace spamm
