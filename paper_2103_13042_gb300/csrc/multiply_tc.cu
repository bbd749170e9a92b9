// Tensor-core multiply (Section 3.3 / Algorithm 3, rebuilt for tcgen05):
//   C[i,j] = sum over listed k of 2^(ea[i,k] + eb[k,j]) * (Ahi Bhi [+ 2^-s (Ahi Blo + Alo Bhi)])
// over the plan's non-empty tiles, most survivors first.
//
// One persistent CTA per SM, warps with fixed roles:
//   warp 2   scheduler: takes the CTA's tiles 32 at a time (one descriptor
//            per lane), flattens their surviving k into one list and loads
//            it 32 entries per round (k, then the exponent sum ea + eb),
//            marks run starts and tile ends with warp shuffles, and publishes
//            the records into a shared-memory ring of 32-entry groups.
//   warp 0   TMA producer: reads the records, waits for a free shared-memory
//            stage and copies the operand image chunks (A hi, B hi, and the
//            lo parts of split triples) with one bulk copy each; per-stage
//            metadata marks run starts, tile ends and split triples.
//   warp 1   allocates tensor memory and issues the MMAs from one thread:
//            consecutive k of a tile with the same exponent sum (and split
//            flag) form a run accumulated in one TMEM accumulator; runs
//            rotate over as many accumulators as TMEM holds (2 to 8), so
//            the epilogue of one overlaps the MMAs of the next ones.  Each stage is released by
//            tcgen05.commit when its MMAs have read it.
//   warps 3+  epilogue (4 warps per 64 output columns): for each run, load
//            the accumulator rows (one TMEM lane per output row, 64 columns
//            per warp), rescale by 2^(ea+eb) in FP32 and add to the tile's
//            register accumulator; at a tile's last run store the rows to C.
// Every wait is bounded in wall time; on expiry the CTA raises an abort flag
// (and SPAMM_ERR_TIMEOUT in the status word), the roles leave their loops,
// outstanding copies and MMAs are drained with bounded waits, and TMEM is
// released.
#include "tc_common.cuh"

namespace spamm {
namespace {

using namespace tc;

constexpr int kRunRing = 16;
constexpr int kGroups = 4;           // scheduler ring: groups of 32 entry records
constexpr int kFirstEpiWarp = 3;

struct StageMeta {
  int32_t flags;   // 1: first chunk of a run, 2: last chunk of a tile, 4: split, 8: end of work
  int32_t s;       // exponent sum of the run
  int32_t tile;
  int32_t pad;
};

struct RunRec {
  int32_t tile, s, split, last;
};

// Entry record published by the scheduler: x = global block of A_ik, y =
// global block of B_kj, z = exponent sum * 16 + flags (1: first of a run,
// 2: last of its tile, 4: split), w = global tile.  A group holds up to 32
// records; its count sits in the misc area (0 count = end of work).
enum : int { kEntFirst = 1, kEntLast = 2, kEntSplit = 4 };

struct TcParams {
  InstRef R;
  PlanBuffers Bf;
  OperandImages img;
  int32_t* status;
  int dynamic;   // take 32-slot chunks of the order from Bf.bdev->mul_ticket
};

template <uint32_t FMT, int LEAF, int SPLITMODE>
struct TcCfg {
  using L = TcLayout<FMT, LEAF>;
  static constexpr bool kHasLo = SPLITMODE != 0;
  static constexpr int M = LEAF, N = LEAF;
  static constexpr int kEpiWarps = 4 * (N / 64);          // 64 columns per epilogue warp
  static constexpr int kThreads = 32 * kFirstEpiWarp + 32 * kEpiWarps;
  // chunks of K per pipeline stage: without lo parts a whole block pair (when
  // it fits in 72 KB), so one barrier wait serves 4 * kNch MMAs; split modes
  // already issue 3 MMAs per K step and keep one chunk per stage
  static constexpr int kCPS =
      (!kHasLo && L::kNch > 1 && L::kChunkBytes * 2 * L::kNch <= 72 * 1024) ? L::kNch : 1;
  static constexpr uint32_t kStageBytes = L::kChunkBytes * 2 * (kHasLo ? 2 : 1) * kCPS;
  static constexpr int kStagesFit =
      (216 * 1024 - kEpiWarps * (M == 64 ? 16 : 0) * (64 * 4 + 16)) / kStageBytes;
  static constexpr int kStages = kStagesFit > 16 ? 16 : kStagesFit;
  static constexpr int kAccCols = N * (kHasLo ? 2 : 1);
  // as many run accumulators as the 512 TMEM columns hold (2 to 8): the MMA
  // issuer runs that many runs ahead of the epilogue
  static constexpr int kNumAcc = 512 / kAccCols;
  static constexpr uint32_t kTmemCols = kNumAcc * kAccCols;          // 512
  static constexpr uint32_t kIdesc = idesc(FMT, M, N);
  // every region starts on a 16-byte boundary (128-bit shared-memory accesses)
  static constexpr size_t up16(size_t x) { return (x + 15) / 16 * 16; }
  static constexpr size_t kBarOffset = (size_t)kStages * kStageBytes;
  static constexpr int kNumBars = 2 * kStages + 2 * kNumAcc + 2 * kRunRing + 1 + 2 * kGroups;
  static constexpr size_t kMetaOffset = up16(kBarOffset + (size_t)kNumBars * 8);
  static constexpr size_t kRunOffset = up16(kMetaOffset + (size_t)kStages * sizeof(StageMeta));
  static constexpr size_t kEntOffset = up16(kRunOffset + (size_t)kRunRing * sizeof(RunRec));
  // epilogue staging for the bulk stores of C (M = 64): per epilogue warp its
  // 16 rows of 64 columns, rows 272 bytes apart.  At M = 128 the shared
  // memory goes to pipeline stages instead and rows are stored directly.
  static constexpr bool kBulkEpilogue = M == 64;
  static constexpr int kEpiRows = kBulkEpilogue ? 16 : 0;
  static constexpr int kEpiRowBytes = 64 * 4 + 16;
  static constexpr size_t kEpiOffset =
      up16(kEntOffset + (size_t)kGroups * 32 * sizeof(int4) + kGroups * sizeof(int));
  static constexpr size_t kMiscOffset =
      up16(kEpiOffset + (size_t)kEpiWarps * kEpiRows * kEpiRowBytes);
  static_assert(kMetaOffset % 16 == 0 && kRunOffset % 16 == 0 && kEntOffset % 16 == 0 &&
                    kEpiOffset % 16 == 0 && kMiscOffset % 16 == 0 && kBarOffset % 1024 == 0 &&
                    kEpiRowBytes % 16 == 0,
                "shared-memory regions aligned");
  static constexpr size_t kSmemBytes = kMiscOffset + 64 + 1024;     // + alignment slack
  static_assert(kStages >= 2, "at least two pipeline stages");
  static_assert(!kHasLo || kCPS == 1, "lo parts are staged one chunk at a time");
  static_assert(kTmemCols >= 32 && kTmemCols <= 512 && kNumAcc >= 2, "TMEM columns");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};


template <uint32_t FMT, int LEAF, int SPLITMODE>
__global__ void __launch_bounds__(TcCfg<FMT, LEAF, SPLITMODE>::kThreads, 1)
    tc_multiply_kernel(TcParams p) {
  using Cfg = TcCfg<FMT, LEAF, SPLITMODE>;
  using L = typename Cfg::L;
  constexpr int S = Cfg::kStages, N = Cfg::N;
  constexpr uint32_t CH = L::kChunkBytes;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOffset);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  constexpr int NA = Cfg::kNumAcc;
  uint64_t* acc_full = bars + 2 * S;
  uint64_t* acc_empty = acc_full + NA;
  uint64_t* run_full = acc_empty + NA;
  uint64_t* run_empty = run_full + kRunRing;
  uint64_t* drain = run_empty + kRunRing;
  uint64_t* ent_full = drain + 1;
  uint64_t* ent_empty = ent_full + kGroups;
  StageMeta* meta = reinterpret_cast<StageMeta*>(smem + Cfg::kMetaOffset);
  RunRec* runs = reinterpret_cast<RunRec*>(smem + Cfg::kRunOffset);
  int4* ents = reinterpret_cast<int4*>(smem + Cfg::kEntOffset);
  int* ent_count = reinterpret_cast<int*>(smem + Cfg::kEntOffset + kGroups * 32 * sizeof(int4));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::kMiscOffset);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + Cfg::kMiscOffset + 4);

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NA; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], Cfg::kEpiWarps);
    }
    for (int r = 0; r < kRunRing; ++r) {
      mbar_init(&run_full[r], 1);
      mbar_init(&run_empty[r], Cfg::kEpiWarps);
    }
    mbar_init(drain, 1);
    for (int g = 0; g < kGroups; ++g) {
      mbar_init(&ent_full[g], 1);
      mbar_init(&ent_empty[g], 1);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // the set-up above (barriers, tensor memory) overlaps the previous kernel's
  // tail; everything below reads what it wrote
  pdl_wait();
  const int ne = p.Bf.bdev->nonempty;

  if (warp == 2) {
    // ------------------------------------------------------------ scheduler
    uint32_t grp = 0, gphase = 0;
    int gfill = 0;            // records already in the current group
    bool ok = wait_ab(&ent_empty[0], 1u, abort_flag, p.status);
    auto publish = [&]() -> bool {   // hands the current group to the producer
      __threadfence_block();
      __syncwarp();
      if (lane == 0) {
        ent_count[grp] = gfill;
        mbar_arrive(&ent_full[grp]);
      }
      if (++grp == kGroups) {
        grp = 0;
        gphase ^= 1u;
      }
      gfill = 0;
      return wait_ab(&ent_empty[grp], gphase ^ 1u, abort_flag, p.status);
    };
    // static: this CTA's slots are blockIdx.x + (32 m + lane) * gridDim.x;
    // dynamic: consecutive 32-slot chunks from the global counter
    auto next_base = [&](int prev) -> int {
      if (!p.dynamic) return prev < 0 ? (int)blockIdx.x : prev + 32 * (int)gridDim.x;
      int b = 0;
      if (lane == 0) b = atomicAdd(&p.Bf.bdev->mul_ticket, 32);
      return __shfl_sync(0xffffffffu, b, 0);
    };
    for (int base = next_base(-1); base < ne && ok; base = next_base(base)) {
      const int w = p.dynamic ? base + lane : base + lane * (int)gridDim.x;
      const bool valid = w < ne;
      int t = 0, beg = 0, end = 0, bkl = 1, bnl = 1;
      int64_t t0 = 0, a0 = 0, b0 = 0;
      if (valid) {
        t = p.Bf.order[w];                       // global tile
        const Inst& in = p.R.at(inst_of(p.R, p.Bf, t));
        t0 = in.tile0;
        a0 = in.ablk0;
        b0 = in.bblk0;
        bkl = in.bk;
        bnl = in.bn;
        beg = p.Bf.tile_beg[t];
        end = beg + p.Bf.cnt[t];
      }
      const int cnt = end - beg;
      int incl = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
      }
      const int excl = incl - cnt;
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      int32_t carry_key = 0;
      int carry_tile = -1;
      for (int f0 = 0; f0 < total && ok; f0 += 32) {
        const int f = f0 + lane;
        const bool act = f < total;
        // owning tile slot: the last lane u with excl[u] <= f
        int u = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = u + step;
          const int ex = __shfl_sync(0xffffffffu, excl, cand & 31);
          if (cand < 32 && ex <= f) u = cand;
        }
        const int tu = __shfl_sync(0xffffffffu, t, u);
        const int bu = __shfl_sync(0xffffffffu, beg, u);
        const int xu = __shfl_sync(0xffffffffu, excl, u);
        const int iu = __shfl_sync(0xffffffffu, incl, u);
        const int bku = __shfl_sync(0xffffffffu, bkl, u);
        const int bnu = __shfl_sync(0xffffffffu, bnl, u);
        const int64_t t0u = __shfl_sync(0xffffffffu, t0, u);
        const int64_t a0u = __shfl_sync(0xffffffffu, a0, u);
        const int64_t b0u = __shfl_sync(0xffffffffu, b0, u);
        const int q = bu + (f - xu);
        uint32_t ent = 0;
        if (act) ent = p.Bf.k_idx[q];
        const int k = (int)(ent & 0x3ffu);
        const int64_t lt = (int64_t)tu - t0u;
        const int i = (int)(lt / bnu), j = (int)(lt % bnu);
        const int ga = (int)(a0u + (int64_t)i * bku + k), gb = (int)(b0u + (int64_t)k * bnu + j);
        int32_t sexp = 0;
        if (act) sexp = p.img.ea[ga] + p.img.eb[gb];
        const bool split = SPLITMODE == 2 || (SPLITMODE == 1 && (ent & 0x8000u));
        const int32_t key = sexp * 2 + (split ? 1 : 0);
        int32_t pkey = __shfl_up_sync(0xffffffffu, key, 1);
        int ptile = __shfl_up_sync(0xffffffffu, tu, 1);
        if (lane == 0) {
          pkey = carry_key;
          ptile = carry_tile;
        }
        const bool first = ptile != tu || pkey != key;
        const bool last = f == iu - 1;
        carry_key = __shfl_sync(0xffffffffu, key, 31);
        carry_tile = __shfl_sync(0xffffffffu, tu, 31);
        const int nact = min(32, total - f0);
        if (gfill + nact > 32) ok = publish();
        if (!ok) break;
        if (act)
          ents[grp * 32 + gfill + lane] =
              make_int4(ga, gb,
                        sexp * 16 + ((first ? kEntFirst : 0) | (last ? kEntLast : 0) |
                                     (split ? kEntSplit : 0)),
                        tu);
        gfill += nact;
      }
    }
    if (ok && gfill > 0) ok = publish();
    if (ok) publish();   // an empty group: end of work
  } else if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, grp = 0, gphase = 0;
      uint32_t issued = 0, issued_phase = 0;   // bit s: stage s has a copy in flight / its parity
      bool ok = true;
      for (;;) {
        if (!wait_ab(&ent_full[grp], gphase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const int nrec = ent_count[grp];
        if (nrec == 0) break;
        for (int r = 0; r < nrec && ok; ++r) {
          const int4 rec = ents[grp * 32 + r];
          const int flags = rec.z & 15, sexp = rec.z >> 4;   // arithmetic shift
          const bool split = (flags & kEntSplit) != 0;
          const int64_t oa = (int64_t)rec.x * L::kBlockBytes;
          const int64_t ob = (int64_t)rec.y * L::kBlockBytes;
          constexpr int CPS = Cfg::kCPS;
          for (int c = 0; c < L::kNch; c += CPS) {
            if (!wait_ab(&empty[stage], phase ^ 1u, abort_flag, p.status)) {
              ok = false;
              break;
            }
            StageMeta m;
            m.flags = ((flags & kEntFirst) && c == 0 ? 1 : 0) |
                      ((flags & kEntLast) && c + CPS == L::kNch ? 2 : 0) | (split ? 4 : 0);
            m.s = sexp;
            m.tile = rec.w;
            m.pad = 0;
            meta[stage] = m;
            mbar_arrive_expect_tx(&full[stage], CH * CPS * 2 * (split ? 2 : 1));
            uint8_t* sb = smem + (size_t)stage * Cfg::kStageBytes;
            // the image's chunks are consecutive: CPS chunks are one copy
            bulk_g2s(sb, p.img.a_hi + oa + c * CH, CH * CPS, &full[stage]);
            bulk_g2s(sb + CH * CPS, p.img.b_hi + ob + c * CH, CH * CPS, &full[stage]);
            if constexpr (Cfg::kHasLo) {
              if (split) {
                bulk_g2s(sb + 2 * CH, p.img.a_lo + oa + c * CH, CH, &full[stage]);
                bulk_g2s(sb + 3 * CH, p.img.b_lo + ob + c * CH, CH, &full[stage]);
              }
            }
            issued |= 1u << stage;
            issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        mbar_arrive(&ent_empty[grp]);
        if (++grp == kGroups) {
          grp = 0;
          gphase ^= 1u;
        }
      }
      if (ok && wait_ab(&empty[stage], phase ^ 1u, abort_flag, p.status)) {
        meta[stage].flags = 8;   // end of work
        mbar_arrive(&full[stage]);
      }
      if (*abort_flag) {   // let every copy this thread issued land before the CTA exits
        for (int s = 0; s < S; ++s)
          if (issued & (1u << s)) (void)mbar_wait(&full[s], (issued_phase >> s) & 1u, kDrainLimitNs);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, slot = 0, slot_phase = 0;
      int run = -1, runs_opened = 0;
      bool open = false, split_run = false, ok = true;
      int32_t run_s = 0, run_tile = 0;
      uint32_t acc_hh = 0, acc_x = 0, d_hh = tmem, d_x = tmem + N;
      auto close_run = [&](int last) -> bool {
        if (!wait_ab(&run_empty[slot], slot_phase ^ 1u, abort_flag, p.status)) return false;
        runs[slot] = RunRec{run_tile, run_s, split_run ? 1 : 0, last};
        mbar_arrive(&run_full[slot]);
        if (++slot == kRunRing) {
          slot = 0;
          slot_phase ^= 1u;
        }
        mma_commit(&acc_full[run % NA]);
        open = false;
        return true;
      };
      for (;;) {
        if (!wait_ab(&full[stage], phase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const StageMeta m = meta[stage];
        if (m.flags & 8) break;
        // (the operands were written by bulk copies whose completion the
        // mbarrier reported: no tcgen05 fence is needed before reading them)
        if (m.flags & 1) {
          if (open && !close_run(0)) {
            ok = false;
            break;
          }
          run = runs_opened++;
          const int buf = run % NA;
          if (!wait_ab(&acc_empty[buf], (((uint32_t)(run / NA)) & 1u) ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          fence_after_sync();
          d_hh = tmem + (uint32_t)(buf * Cfg::kAccCols);
          d_x = d_hh + N;
          acc_hh = 0;
          acc_x = 0;
          open = true;
          split_run = (m.flags & 4) != 0;
          run_s = m.s;
          run_tile = m.tile;
        }
        // descriptors of the stage's chunks; a 32-byte K step adds 2 to the
        // start-address field (addresses stay below 256 KB: no carry)
        constexpr int CPS = Cfg::kCPS;
        const uint32_t a0 = smem_u32(smem + (size_t)stage * Cfg::kStageBytes);
        const uint64_t da = sdesc_k_sw128(a0), db = sdesc_k_sw128(a0 + CPS * CH);
#pragma unroll
        for (int cc = 0; cc < CPS; ++cc) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t step = (uint64_t)(cc * CH >> 4) + 2u * ks;
            const uint64_t ad = da + step, bdsc = db + step;
            mma<FMT>(d_hh, ad, bdsc, Cfg::kIdesc, acc_hh);
            acc_hh = 1;
            if constexpr (Cfg::kHasLo) {   // CPS == 1 here: lo parts at 2 CH and 3 CH
              if (split_run) {
                mma<FMT>(d_x, ad, db + (uint64_t)(2 * CH >> 4) + 2u * ks, Cfg::kIdesc, acc_x);
                acc_x = 1;
                mma<FMT>(d_x, da + (uint64_t)(2 * CH >> 4) + 2u * ks, bdsc, Cfg::kIdesc, 1);
              }
            }
          }
        }
        mma_commit(&empty[stage]);
        if ((m.flags & 2) && !close_run(1)) {
          ok = false;
          break;
        }
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (ok && wait_ab(&run_empty[slot], slot_phase ^ 1u, abort_flag, p.status)) {
        runs[slot] = RunRec{-1, 0, 0, 1};   // end of work
        mbar_arrive(&run_full[slot]);
      }
      mma_commit(drain);   // every MMA this thread issued has finished before TMEM is freed
      (void)mbar_wait(drain, 0, kDrainLimitNs);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int NC = 64;                       // columns owned by this warp
    const int quarter = warp & 3;
    const int col0 = ((warp - kFirstEpiWarp) / 4) * NC;
    const int row = Cfg::M == 128 ? quarter * 32 + lane : quarter * 16 + lane;
    const bool lane_has_row = Cfg::M == 128 || lane < 16;
    const float lo_w = 1.0f / (float)(1 << L::kLoShift);
    uint8_t* stage_row = smem + Cfg::kEpiOffset +
                         ((size_t)(warp - kFirstEpiWarp) * Cfg::kEpiRows + lane) * Cfg::kEpiRowBytes;
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
    uint32_t slot = 0, slot_phase = 0;
    int run = 0;
    for (;;) {
      if (!wait_ab(&run_full[slot], slot_phase, abort_flag, p.status)) break;
      const RunRec r = runs[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&run_empty[slot]);
      if (++slot == kRunRing) {
        slot = 0;
        slot_phase ^= 1u;
      }
      if (r.tile < 0) break;
      const int buf = run % NA;
      if (!wait_ab(&acc_full[buf], ((uint32_t)(run / NA)) & 1u, abort_flag, p.status)) break;
      fence_after_sync();
      // 2^s in one factor when it is a normal float, else in two (coarse
      // BF16/TF32 exponents can put s outside [-126, 127] for representable C)
      const bool one = r.s >= -126 && r.s <= 127;
      const int s1 = one ? r.s : r.s / 2;
      const float scale = ldexpf(1.0f, s1), scale2 = ldexpf(1.0f, r.s - s1);
      const uint32_t base = tmem + (uint32_t)(buf * Cfg::kAccCols + col0) +
                            ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += 32) {
        float v[32];
        tmem_ld32(base + c0, v);
        if constexpr (Cfg::kHasLo) {
          if (r.split) {
            float x[32];
            tmem_ld32(base + N + c0, x);
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = fmaf(x[q], lo_w, v[q]);
          }
        }
        if (one) {
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[c0 + q] = fmaf(v[q], scale, acc[c0 + q]);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[c0 + q] = fmaf(v[q] * scale, scale2, acc[c0 + q]);
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      ++run;
      if (r.last) {
        const Inst& in = p.R.at(inst_of(p.R, p.Bf, r.tile));
        const int bn = in.bn;
        const int64_t m = in.m, n = in.n, ldc = in.ldc, lt = (int64_t)r.tile - in.tile0;
        const int i = (int)(lt / bn), j = (int)(lt % bn);
        const int64_t gr = (int64_t)i * LEAF + row;
        const int64_t cols = n - (int64_t)j * LEAF - col0;
        const bool row_in = lane_has_row && gr < m;
        float* dst = in.C + gr * ldc + (int64_t)j * LEAF + col0;
        // C = alpha * acc + beta * C (the old C is read only when beta != 0)
        const float alpha = in.alpha, beta = in.beta;
        if (beta != 0.0f && row_in) {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            acc[c] = c < cols ? __fmaf_rn(beta, dst[c], __fmul_rn(alpha, acc[c])) : 0.0f;
        } else if (alpha != 1.0f) {
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = __fmul_rn(alpha, acc[c]);
        }
        if (in.nC) {
          // C's norm map for a chained product: this warp's part of the tile's
          // sum of squares (its rows x its 64 columns) goes to the tile's slot
          float v[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] = (row_in && c < cols) ? acc[c] : 0.0f;
          SumSq ss = sumsq_empty();
          sumsq_group<NC>(ss, v);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
            const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
            const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
            sumsq_merge_any(ss, h, l, e);
          }
          if (lane == 0)
            reinterpret_cast<NormPart*>(p.Bf.norm_part)[(int64_t)r.tile * kMaxEpiWarps +
                                                        (warp - kFirstEpiWarp)] =
                NormPart{ss.hi, ss.lo, ss.e, 0};
        }
        if (row_in) {
          if (Cfg::kBulkEpilogue && (ldc & 3) == 0 && (n & 3) == 0) {
            // the row goes through shared memory and leaves as one bulk copy
            // (ldc % 4 == 0: 16-byte aligned; n % 4 == 0: whole 16-byte pieces)
            if (cols > 0) {
              bulk_wait_read0();   // this lane's previous row has left the buffer
#pragma unroll
              for (int c = 0; c < NC; c += 4)
                *reinterpret_cast<float4*>(stage_row + 4 * c) =
                    make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
              fence_proxy_async_smem();
              bulk_s2g(dst, smem_u32(stage_row), (uint32_t)(cols < NC ? cols : NC) * 4u);
              bulk_commit();
            }
          } else if ((ldc & 3) == 0 && cols >= NC) {
#pragma unroll
            for (int c = 0; c < NC; c += 4)
              *reinterpret_cast<float4*>(dst + c) =
                  make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c)
              if (c < cols) dst[c] = acc[c];
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
      }
    }
  }

  if (warp >= kFirstEpiWarp) bulk_wait0();   // C rows written before the kernel ends
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, Cfg::kTmemCols);
  }
}

// One tile without survivors, written by a whole warp: C = beta * C, which
// for beta = 0 is zeros (16-byte streaming stores when the rows are 16-byte
// aligned: lane l owns float4 column l % (leaf/4) and every (32 / (leaf/4))-th
// row, so a warp store covers whole 128-byte row segments) and for beta = 1
// leaves C as it is; with an output norm map the tile's norm is written too.
template <int LEAF>
__device__ __forceinline__ void empty_tile(const Inst& in, int64_t lt, int lane) {
  constexpr int kPerRow = LEAF / 4;                          // float4 per tile row
  constexpr int kRowsPerStore = kPerRow >= 32 ? 1 : 32 / kPerRow;
  constexpr int kColSteps = kPerRow >= 32 ? kPerRow / 32 : 1;
  const int bn = in.bn;
  const int ti = (int)(lt / bn), tj = (int)(lt - (int64_t)ti * bn);
  const int64_t r0 = (int64_t)ti * LEAF, c0 = (int64_t)tj * LEAF;
  const int rows = (int)min((int64_t)LEAF, in.m - r0), cols = (int)min((int64_t)LEAF, in.n - c0);
  const int64_t ldc = in.ldc;
  float* C = in.C;
  const float beta = in.beta;
  if (beta == 0.0f) {
    const int my_c4 = kPerRow >= 32 ? lane : lane % kPerRow;
    const int my_r = kPerRow >= 32 ? 0 : lane / kPerRow;
    const bool vec = (ldc & 3) == 0 && (in.n & 3) == 0;   // then cols % 4 == 0
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec && rows == LEAF && cols == LEAF) {   // aligned full tile: unrolled stores
#pragma unroll
      for (int cs = 0; cs < kColSteps; ++cs) {
        float4* p = reinterpret_cast<float4*>(C + (r0 + my_r) * ldc + c0) + my_c4 + 32 * cs;
        const int64_t step = (int64_t)kRowsPerStore * ldc / 4;
#pragma unroll 8
        for (int r = 0; r < LEAF / kRowsPerStore; ++r) __stcs(p + r * step, z);
      }
    } else if (vec) {   // aligned ragged tile
      for (int cs = 0; cs < kColSteps; ++cs) {
        const int c4 = my_c4 + 32 * cs;
        if (4 * c4 >= cols) continue;
        float4* p = reinterpret_cast<float4*>(C + (r0 + my_r) * ldc + c0 + 4 * c4);
        const int64_t step = (int64_t)kRowsPerStore * ldc / 4;
        for (int r = my_r; r < rows; r += kRowsPerStore, p += step) __stcs(p, z);
      }
    } else {   // rows not 16-byte aligned: row by row, the lanes over the columns
               // (coalesced 4-byte streaming stores, no index division)
      for (int r = 0; r < rows; ++r) {
        float* p = C + (r0 + r) * ldc + c0;
        for (int c = lane; c < cols; c += 32) __stcs(p + c, 0.f);
      }
    }
    if (in.nC && lane == 0) in.nC[lt] = 0.0;
    return;
  }
  if (beta == 1.0f && !in.nC) return;
  SumSq ss = sumsq_empty();
  for (int u0 = 0; u0 < rows * cols; u0 += 32 * 32) {
    float v[32];
#pragma unroll 4
    for (int q = 0; q < 32; ++q) {
      const int u = u0 + q * 32 + lane;
      float x = 0.0f;
      if (u < rows * cols) {
        float* p = C + (r0 + u / cols) * ldc + c0 + u % cols;
        x = __fmul_rn(beta, *p);
        if (beta != 1.0f) *p = x;
      }
      v[q] = x;
    }
    if (in.nC) sumsq_group<32>(ss, v);
  }
  if (in.nC) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
      const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
      const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
      sumsq_merge_any(ss, h, l, e);
    }
    if (lane == 0) in.nC[lt] = sumsq_sqrt(ss);
  }
}

// Every tile without survivors: the plan lists them after the non-empty tiles
// in `order`.  One warp per tile (many independent warps keep enough stores in
// flight for the HBM write rate).
template <int LEAF>
__global__ void __launch_bounds__(256)
    zero_tiles_kernel(InstRef R, PlanBuffers Bf) {
  const int lane = threadIdx.x & 31;
  const int ne = Bf.bdev->nonempty;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t e = ne + ((int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32); e < Bf.tiles;
       e += nw) {
    const int64_t g = Bf.order[e];
    const Inst& in = R.at(inst_of(R, Bf, g));
    empty_tile<LEAF>(in, g - in.tile0, lane);
  }
}

// The same from the per-tile counts alone (may run as soon as the plan's
// counting half has finished).  Every CTA takes an equal contiguous range of
// global tiles (so every SM writes about the same number of bytes); warp 0
// lists the range's empty tiles in shared memory (coalesced count loads,
// ballots), then each warp takes whole empty tiles (list entries warp,
// warp + 8, ...), so the tile's address arithmetic is paid once per
// leaf*leaf*4 bytes.
constexpr int kZeroThreads = 256;
constexpr int kZeroMaxRange = 64;   // tiles per CTA at most (the grid grows beyond that)

template <int LEAF>
__global__ void __launch_bounds__(kZeroThreads)
    zero_scan_kernel(InstRef R, PlanBuffers Bf) {
  constexpr int kWarps = kZeroThreads / 32;
  __shared__ int s_list[kZeroMaxRange];
  __shared__ int s_count;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t lo = Bf.tiles * blockIdx.x / gridDim.x;
  const int64_t hi = Bf.tiles * (blockIdx.x + 1) / gridDim.x;   // hi - lo <= kZeroMaxRange
  if (warp == 0) {
    int count = 0;
    for (int64_t g0 = lo; g0 < hi; g0 += 32) {
      const int64_t gl = g0 + lane;
      const bool empty = gl < hi && Bf.cnt[gl] == 0;
      const unsigned mask = __ballot_sync(0xffffffffu, empty);
      if (empty) s_list[count + __popc(mask & ((1u << lane) - 1u))] = (int)(gl - lo);
      count += __popc(mask);
    }
    if (lane == 0) s_count = count;
  }
  __syncthreads();
  const int count = s_count;
  for (int e = warp; e < count; e += kWarps) {
    const int64_t g = lo + s_list[e];
    const Inst& in = R.at(inst_of(R, Bf, g));
    empty_tile<LEAF>(in, g - in.tile0, lane);
  }
}

// Output norm maps of the tensor-core multiply: each non-empty tile's
// epilogue warps left their partial sums of squares in the tile's slot; one
// thread per tile merges them (in warp order) and writes the norm.
__global__ void __launch_bounds__(256)
    norm_out_finish_kernel(InstRef R, PlanBuffers Bf, int parts) {
  pdl_wait();
  const int ne = Bf.bdev->nonempty;
  const NormPart* np = reinterpret_cast<const NormPart*>(Bf.norm_part);
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < ne;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = Bf.order[w];
    const Inst& in = R.at(inst_of(R, Bf, g));
    if (!in.nC) continue;
    SumSq ss = sumsq_empty();
    for (int q = 0; q < parts; ++q) {
      const NormPart x = np[g * kMaxEpiWarps + q];
      sumsq_merge_any(ss, x.hi, x.lo, x.e);
    }
    in.nC[g - in.tile0] = sumsq_sqrt(ss);
  }
}

// Self-test of the bounded wait: one CTA waits, with the multiply's own wait
// routine and a short limit, on an mbarrier phase that nothing completes; the
// wait must give up, raise the abort flag and latch SPAMM_ERR_TIMEOUT.
// out[0] = 1 if the wait returned false, out[1] = the abort flag, out[2] =
// elapsed nanoseconds.
__global__ void wait_selftest_kernel(int32_t* status, uint64_t limit_ns, long long* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);   // phase 0 completes only on an arrival, which never comes
    abort_flag = 0;
    fence_mbarrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer_ns();
    const bool ok = wait_ab(&bar, 0u, &abort_flag, status, limit_ns);
    out[0] = ok ? 0 : 1;
    out[1] = abort_flag;
    out[2] = (long long)(globaltimer_ns() - t0);
  }
}

template <uint32_t FMT, int LEAF, int SPLITMODE>
cudaError_t launch_tc(const TcParams& prm, cudaStream_t s) {
  using Cfg = TcCfg<FMT, LEAF, SPLITMODE>;
  auto kern = tc_multiply_kernel<FMT, LEAF, SPLITMODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return launch_pdl(kern, dim3(sms), dim3(Cfg::kThreads), Cfg::kSmemBytes, s, prm);
}

}  // namespace

cudaError_t launch_zero_empty_tiles(const InstRef& ref, const PlanBuffers& b, int leaf,
                                    cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one wave of warps (the number of empty tiles is known on the device only)
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((b.tiles + 7) / 8, (int64_t)sms * 8));
  switch (leaf) {
    case 32: zero_tiles_kernel<32><<<grid, 256, 0, s>>>(ref, b); break;
    case 64: zero_tiles_kernel<64><<<grid, 256, 0, s>>>(ref, b); break;
    case 128: zero_tiles_kernel<128><<<grid, 256, 0, s>>>(ref, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaPeekAtLastError();
}

cudaError_t launch_wait_selftest(int32_t* status, uint64_t limit_ns, long long* out,
                                 cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(status, limit_ns, out);
  return cudaPeekAtLastError();
}

cudaError_t launch_zero_empty_tiles_scan(const InstRef& ref, const PlanBuffers& b, int leaf,
                                         cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // four CTAs per SM, each an equal range of at most kZeroMaxRange tiles
  const int64_t want = std::max<int64_t>((int64_t)sms * 4, (b.tiles + kZeroMaxRange - 1) / kZeroMaxRange);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(b.tiles, want));
  switch (leaf) {
    case 32: zero_scan_kernel<32><<<grid, kZeroThreads, 0, s>>>(ref, b); break;
    case 64: zero_scan_kernel<64><<<grid, kZeroThreads, 0, s>>>(ref, b); break;
    case 128: zero_scan_kernel<128><<<grid, kZeroThreads, 0, s>>>(ref, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaPeekAtLastError();
}

cudaError_t launch_norm_out_finish(const InstRef& ref, const PlanBuffers& b, int leaf,
                                   cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((b.tiles + 255) / 256, (int64_t)sms * 4));
  return launch_pdl(norm_out_finish_kernel, dim3(grid), dim3(256), 0, s, ref, b,
                    4 * (leaf / 64));
}

cudaError_t launch_multiply_tc(spamm_precision_t prec, int leaf, const InstRef& ref,
                               const PlanBuffers& b, const OperandImages& img, int32_t* status,
                               int schedule, cudaStream_t s) {
  if (schedule == kScheduleGroups && multiply_tc_groups_supported(prec, leaf, ref))
    return launch_multiply_tc_groups(prec, ref, b, img, status, s);
  TcParams prm{ref, b, img, status, schedule == kScheduleDynamic ? 1 : 0};
  const bool l64 = leaf == 64;
  switch (prec) {
    case SPAMM_BF16:
      return l64 ? launch_tc<kFmtBF16, 64, 0>(prm, s) : launch_tc<kFmtBF16, 128, 0>(prm, s);
    case SPAMM_FP16:
      return l64 ? launch_tc<kFmtF16, 64, 0>(prm, s) : launch_tc<kFmtF16, 128, 0>(prm, s);
    case SPAMM_BF16_SPLIT:
      return l64 ? launch_tc<kFmtBF16, 64, 1>(prm, s) : launch_tc<kFmtBF16, 128, 1>(prm, s);
    case SPAMM_FP16_SPLIT:
      return l64 ? launch_tc<kFmtF16, 64, 1>(prm, s) : launch_tc<kFmtF16, 128, 1>(prm, s);
    case SPAMM_TF32X3:
      return l64 ? launch_tc<kFmtTF32, 64, 2>(prm, s) : launch_tc<kFmtTF32, 128, 2>(prm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spamm
