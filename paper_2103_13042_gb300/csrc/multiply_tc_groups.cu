// Grouped tensor-core multiply: the tiles of one block row in groups of four
// consecutive block columns (i, 4g .. 4g + 3) share their A operands.
//
// The per-tile multiply stages A_ik and B_kj for every surviving triple
// (2 x 32 KB at leaf 128 in BF16/FP16).  Here a CTA walks the union of the
// four tiles' surviving k in increasing order; for each k it stages A_ik once
// and B_kj for every tile of the group that keeps the triple, and issues each
// tile's MMAs into that tile's own TMEM accumulator (4 x 128 columns: all of
// TMEM).  On a dense-ish skip set (near-sparse inputs at a 50% valid ratio)
// two or three of the four tiles keep a given k, so the bytes staged per
// product fall from 64 KB to about 45 KB: the multiply there is bound by the
// rate at which an SM takes operands in from L2, not by the tensor pipe.
//
// Roles, as in the per-tile kernel:
//   warp 2   scheduler: takes groups in column panels of kPanelGroups groups
//            (row-major inside a panel: the SMs work down a narrow band of
//            block columns, sharing its B blocks in L2; measured best among
//            panel widths 1 to 64 at N = 8192 to 32768), reads the four
//            tiles' survivor bitmasks, and publishes one record per k of
//            the union: A block, the B block of the
//            group's first column, the mask of tiles that keep k, which of
//            them start an accumulator run (a change of the exponent sum
//            ea + eb) and which end their tile, and the four exponent sums.
//   warp 0   producer: per record one 32 KB slot of the A ring (three slots),
//            then one slot of the B ring (four) per kept B, each filled by
//            one bulk copy.  Separate rings: an A slot is held while its
//            record's B slots are multiplied, and must not hold up the reuse
//            of B slots that are already free.
//   warp 1   MMA issuer: holds the record's A slot until its last B slot has
//            been multiplied (then releases both); opens and closes the runs
//            of each tile's accumulator.
//   warps 3+ epilogue: for each closed run, loads the accumulator rows (one
//            TMEM lane per row, 64 columns per warp), frees the accumulator,
//            scales by 2^(ea+eb) and adds to C.  A tile with one run is
//            stored once; earlier runs of a tile with several leave their
//            partial sum in C, which the next run of the same thread reads
//            back (the same FMA chain as a register accumulator).
// Instances must have alpha = 1, beta = 0 and no output norm map (the batch
// form); the host falls back to the per-tile kernel otherwise.  Every wait is
// bounded as in the per-tile kernel: on expiry the abort flag is raised and
// SPAMM_ERR_TIMEOUT latched, the roles leave their loops, copies and MMAs are
// drained and TMEM is released.
#include "tc_common.cuh"

namespace spamm {
namespace {

using namespace tc;

constexpr int kG = kGroupTiles;      // tiles per group
// Seven 32 KB operand slots (all of shared memory but the bookkeeping): three
// for A blocks (one is held per record), four for B blocks (the B ring bounds
// the bytes in flight); groups in column panels two groups wide.  Measured at
// near-sparse N = 8192 to 32768: splits 1/5 to 4/3 of six and seven slots,
// panel widths 1 to 64.
constexpr int kSlots = 7;
constexpr int kASlots = 3;
constexpr int kBSlots = kSlots - kASlots;
constexpr int kRecGroups = 2;        // record ring: groups of 32 records
// run ring: a closed run waits here for the epilogue (at most one per
// accumulator is open); kept short so that seven slots fit in shared memory
constexpr int kRuns = 4;
constexpr int kPanelGroups = 2;      // groups per panel row of the group order
constexpr int kEpi0 = 3;             // first epilogue warp

// One k of a group's union: A block ga, B block gb0 + q for tile q; flags:
// bits 0-3 tiles that keep k, 4-7 tiles whose run starts here, 8-11 tiles
// whose last k this is; tile0 = global tile of q = 0; s[q] = ea + eb.
struct GRec {
  int ga, gb0, flags, tile0;
  short s[kG];
};

// B-slot flags: the record's first B (take the next A slot), the tile's run
// starts / the tile ends here, the record's last B (release its A slot), end.
enum : int { kSlotNewA = 1, kSlotFirst = 2, kSlotLast = 4, kSlotLastB = 8, kSlotEnd = 16 };

struct GMeta {
  int flags, s, tile, q;
};

struct GRun {
  int tile, s, q, last;   // tile < 0: end of work
};

struct GParams {
  InstRef R;
  PlanBuffers Bf;
  OperandImages img;
  int32_t* status;
};

template <uint32_t FMT>
struct GCfg {
  using L = TcLayout<FMT, 128>;
  static constexpr int M = 128, N = 128;
  static constexpr int kEpiWarps = 8;                       // 4 row quarters x 2 column halves
  static constexpr int kThreads = 32 * kEpi0 + 32 * kEpiWarps;
  static constexpr uint32_t kSlotBytes = L::kBlockBytes;    // one block image, 32 KB
  static constexpr uint32_t kIdesc = idesc(FMT, M, N);
  static constexpr uint32_t kTmemCols = kG * N;             // 512
  static constexpr size_t up16(size_t x) { return (x + 15) / 16 * 16; }
  static constexpr size_t kBarOffset = (size_t)kSlots * kSlotBytes;
  static constexpr int kNumBars = 2 * kSlots + 2 * kG + 2 * kRuns + 1 + 2 * kRecGroups;
  static constexpr size_t kMetaOffset = up16(kBarOffset + (size_t)kNumBars * 8);
  static constexpr size_t kRunOffset = up16(kMetaOffset + (size_t)kSlots * sizeof(GMeta));
  static constexpr size_t kRecOffset = up16(kRunOffset + (size_t)kRuns * sizeof(GRun));
  static constexpr size_t kMiscOffset =
      up16(kRecOffset + (size_t)kRecGroups * 32 * sizeof(GRec) + kRecGroups * sizeof(int));
  static constexpr size_t kSmemBytes = kMiscOffset + 16 + 1024;   // + alignment slack
  static_assert(kSlotBytes == 32768 && kBarOffset % 1024 == 0, "slot layout");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory");
  static_assert(kTmemCols == 512, "four 128-column accumulators");
};

// Group number lg of an instance -> block row i and group column jg: column
// panels of kPanelGroups groups (the last narrower), row-major inside.
__device__ __forceinline__ void group_at(const Inst& in, int64_t lg, int& i, int& jg) {
  const int ng = (in.bn + kG - 1) / kG;
  const int64_t full = (int64_t)in.bm * kPanelGroups;
  const int64_t p = lg / full;
  const int64_t r = lg - p * full;
  const int w = min(kPanelGroups, ng - (int)p * kPanelGroups);
  i = (int)(r / w);
  jg = (int)(p * kPanelGroups + r % w);
}

template <uint32_t FMT>
__global__ void __launch_bounds__(GCfg<FMT>::kThreads, 1) tc_group_kernel(GParams p) {
  using Cfg = GCfg<FMT>;
  using L = typename Cfg::L;
  constexpr uint32_t SB = Cfg::kSlotBytes, CH = L::kChunkBytes;
  constexpr unsigned kAll = 0xffffffffu;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOffset);
  uint64_t* full = bars;
  uint64_t* empty = full + kSlots;
  uint64_t* acc_full = empty + kSlots;
  uint64_t* acc_empty = acc_full + kG;
  uint64_t* run_full = acc_empty + kG;
  uint64_t* run_empty = run_full + kRuns;
  uint64_t* drain = run_empty + kRuns;
  uint64_t* rec_full = drain + 1;
  uint64_t* rec_empty = rec_full + kRecGroups;
  GMeta* meta = reinterpret_cast<GMeta*>(smem + Cfg::kMetaOffset);
  GRun* runs = reinterpret_cast<GRun*>(smem + Cfg::kRunOffset);
  GRec* recs = reinterpret_cast<GRec*>(smem + Cfg::kRecOffset);
  int* rec_count = reinterpret_cast<int*>(smem + Cfg::kRecOffset + kRecGroups * 32 * sizeof(GRec));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::kMiscOffset);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + Cfg::kMiscOffset + 4);

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < kG; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], Cfg::kEpiWarps);
    }
    for (int r = 0; r < kRuns; ++r) {
      mbar_init(&run_full[r], 1);
      mbar_init(&run_empty[r], Cfg::kEpiWarps);
    }
    mbar_init(drain, 1);
    for (int g = 0; g < kRecGroups; ++g) {
      mbar_init(&rec_full[g], 1);
      mbar_init(&rec_empty[g], 1);
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

  if (warp == 2) {
    // ------------------------------------------------------------ scheduler
    uint32_t grp = 0, gphase = 0;
    int gfill = 0;
    bool ok = wait_ab(&rec_empty[0], 1u, abort_flag, p.status);
    auto publish = [&]() -> bool {
      __threadfence_block();
      __syncwarp();
      if (lane == 0) {
        rec_count[grp] = gfill;
        mbar_arrive(&rec_full[grp]);
      }
      if (++grp == kRecGroups) {
        grp = 0;
        gphase ^= 1u;
      }
      gfill = 0;
      return wait_ab(&rec_empty[grp], gphase ^ 1u, abort_flag, p.status);
    };
    for (int64_t G = blockIdx.x; G < p.Bf.groups && ok; G += gridDim.x) {
      const Inst& in = p.R.at(inst_of_group(p.R, G));
      int i, jg;
      group_at(in, G - in.grp0, i, jg);
      const int bk = in.bk, bn = in.bn;
      const int nch = (bk + 31) >> 5;                     // <= 32 (bk <= 1024)
      const int64_t lt0 = (int64_t)i * bn + (int64_t)jg * kG;
      // lane c holds word c of each tile's survivor bitmask (zero for a tile
      // past the last block column)
      uint32_t w[kG];
#pragma unroll
      for (int q = 0; q < kG; ++q) {
        const bool tq = jg * kG + q < bn;
        w[q] = (tq && lane < nch) ? p.Bf.surv_mask[in.mask0 + (lt0 + q) * nch + lane] : 0u;
      }
      // last surviving k of each tile (-1: none)
      int lastk[kG];
      bool any = false;
#pragma unroll
      for (int q = 0; q < kG; ++q) {
        const unsigned nz = __ballot_sync(kAll, w[q] != 0u);
        lastk[q] = -1;
        if (nz) {
          const int cl = 31 - __clz(nz);
          const uint32_t wl = __shfl_sync(kAll, w[q], cl);
          lastk[q] = 32 * cl + 31 - __clz(wl);
          any = true;
        }
      }
      if (!any) continue;
      const int64_t ga0 = in.ablk0 + (int64_t)i * bk;
      const int64_t gbb = in.bblk0 + (int64_t)jg * kG;
      const int gtile0 = (int)(in.tile0 + lt0);
      int prev_s[kG];
      bool has_prev[kG];
#pragma unroll
      for (int q = 0; q < kG; ++q) {
        prev_s[q] = 0;
        has_prev[q] = false;
      }
      for (int c = 0; c < nch && ok; ++c) {
        const int k = 32 * c + lane;
        int jm = 0;
#pragma unroll
        for (int q = 0; q < kG; ++q) jm |= (int)((__shfl_sync(kAll, w[q], c) >> lane) & 1u) << q;
        const bool act = jm != 0;
        const int ga = (int)(ga0 + k);
        const int gb0 = (int)(gbb + (int64_t)k * bn);
        const int ea = act ? p.img.ea[ga] : 0;
        int s[kG];
        int first = 0, last = 0;
#pragma unroll
        for (int q = 0; q < kG; ++q) {
          const bool kq = (jm >> q) & 1;
          s[q] = kq ? ea + p.img.eb[gb0 + q] : 0;
          // the previous k of tile q: the nearest lower lane that keeps it,
          // else the last one of the earlier chunks
          const unsigned mq = __ballot_sync(kAll, kq);
          const unsigned below = mq & ((1u << lane) - 1u);
          const int pl = below ? 31 - __clz(below) : 0;
          const int ps = __shfl_sync(kAll, s[q], pl);
          const bool hp = below ? true : has_prev[q];
          const int pv = below ? ps : prev_s[q];
          if (kq) {
            if (!hp || pv != s[q]) first |= 1 << q;
            if (k == lastk[q]) last |= 1 << q;
          }
          if (mq) {
            prev_s[q] = __shfl_sync(kAll, s[q], 31 - __clz(mq));
            has_prev[q] = true;
          }
        }
        const unsigned am = __ballot_sync(kAll, act);
        const int nact = __popc(am);
        if (nact == 0) continue;
        if (gfill + nact > 32) ok = publish();
        if (!ok) break;
        if (act) {
          GRec r;
          r.ga = ga;
          r.gb0 = gb0;
          r.flags = jm | (first << 4) | (last << 8);
          r.tile0 = gtile0;
#pragma unroll
          for (int q = 0; q < kG; ++q) r.s[q] = (short)s[q];   // |ea + eb| <= 512
          recs[grp * 32 + gfill + __popc(am & ((1u << lane) - 1u))] = r;
        }
        gfill += nact;
      }
    }
    if (ok && gfill > 0) ok = publish();
    if (ok) publish();   // an empty group: end of work
  } else if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t as = 0, aph = 0, bs = 0, bph = 0, grp = 0, gphase = 0;
      uint32_t issued = 0, issued_phase = 0;   // bit s: slot s has a copy in flight / its parity
      bool ok = true;
      // one bulk copy of a block image into slot `slot` (phase `ph`), after it is free
      auto copy = [&](int slot, uint32_t ph, const uint8_t* src) -> bool {
        if (!wait_ab(&empty[slot], ph ^ 1u, abort_flag, p.status)) return false;
        mbar_arrive_expect_tx(&full[slot], SB);
        bulk_g2s(smem + (size_t)slot * SB, src, SB, &full[slot]);
        issued |= 1u << slot;
        issued_phase = (issued_phase & ~(1u << slot)) | (ph << slot);
        return true;
      };
      for (;;) {
        if (!wait_ab(&rec_full[grp], gphase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const int nrec = rec_count[grp];
        if (nrec == 0) break;
        for (int r = 0; r < nrec && ok; ++r) {
          const GRec rec = recs[grp * 32 + r];
          const int jm = rec.flags & 15, first = (rec.flags >> 4) & 15, last = (rec.flags >> 8) & 15;
          const int firstq = __ffs(jm) - 1, lastq = 31 - __clz((unsigned)jm);
          ok = copy((int)as, aph, p.img.a_hi + (int64_t)rec.ga * SB);
          if (++as == kASlots) {
            as = 0;
            aph ^= 1u;
          }
          for (int q = 0; q < kG && ok; ++q) {
            if (!((jm >> q) & 1)) continue;
            const int slot = kASlots + (int)bs;
            // the slot is free once copy() has waited: its metadata may be written
            if (!wait_ab(&empty[slot], bph ^ 1u, abort_flag, p.status)) {
              ok = false;
              break;
            }
            meta[slot] = GMeta{(q == firstq ? kSlotNewA : 0) | (((first >> q) & 1) ? kSlotFirst : 0) |
                                   (((last >> q) & 1) ? kSlotLast : 0) | (q == lastq ? kSlotLastB : 0),
                               rec.s[q], rec.tile0 + q, q};
            ok = copy(slot, bph, p.img.b_hi + (int64_t)(rec.gb0 + q) * SB);
            if (++bs == kBSlots) {
              bs = 0;
              bph ^= 1u;
            }
          }
        }
        if (!ok) break;
        mbar_arrive(&rec_empty[grp]);
        if (++grp == kRecGroups) {
          grp = 0;
          gphase ^= 1u;
        }
      }
      const int slot = kASlots + (int)bs;
      if (ok && wait_ab(&empty[slot], bph ^ 1u, abort_flag, p.status)) {
        meta[slot].flags = kSlotEnd;
        mbar_arrive(&full[slot]);
      }
      if (*abort_flag) {   // let every copy this thread issued land before the CTA exits
        for (int q = 0; q < kSlots; ++q)
          if (issued & (1u << q)) (void)mbar_wait(&full[q], (issued_phase >> q) & 1u, kDrainLimitNs);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t as = 0, aph = 0, bs = 0, bph = 0, rslot = 0, rphase = 0;
      uint32_t opened = 0;        // bit q: parity of the runs opened on accumulator q
      uint32_t open = 0, started = 0;
      int run_s[kG], run_tile[kG];
#pragma unroll
      for (int q = 0; q < kG; ++q) run_s[q] = run_tile[q] = 0;
      bool ok = true;
      auto close_run = [&](int q, int last) -> bool {
        if (!wait_ab(&run_empty[rslot], rphase ^ 1u, abort_flag, p.status)) return false;
        runs[rslot] = GRun{run_tile[q], run_s[q], q, last};
        mbar_arrive(&run_full[rslot]);
        if (++rslot == kRuns) {
          rslot = 0;
          rphase ^= 1u;
        }
        mma_commit(&acc_full[q]);
        open &= ~(1u << q);
        return true;
      };
      for (;;) {
        const int slot = kASlots + (int)bs;
        if (!wait_ab(&full[slot], bph, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const GMeta m = meta[slot];
        if (m.flags & kSlotEnd) break;
        // the record's A block (held until its last B block has been multiplied)
        if ((m.flags & kSlotNewA) && !wait_ab(&full[as], aph, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const int q = m.q & (kG - 1);
        if (m.flags & kSlotFirst) {
          if (((open >> q) & 1) && !close_run(q, 0)) {
            ok = false;
            break;
          }
          // the epilogue has taken the previous run of this accumulator
          if (!wait_ab(&acc_empty[q], ((opened >> q) & 1u) ^ 1u, abort_flag, p.status)) {
            ok = false;
            break;
          }
          opened ^= 1u << q;
          fence_after_sync();
          open |= 1u << q;
          started &= ~(1u << q);
          run_s[q] = m.s;
          run_tile[q] = m.tile;
        }
        const uint32_t d = tmem + (uint32_t)(q * Cfg::N);
        const uint64_t da = sdesc_k_sw128(smem_u32(smem + (size_t)as * SB));
        const uint64_t db = sdesc_k_sw128(smem_u32(smem + (size_t)slot * SB));
        uint32_t acc = (started >> q) & 1u;
#pragma unroll
        for (int cc = 0; cc < L::kNch; ++cc) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // a 32-byte K step adds 2 to the start-address field (below 256 KB: no carry)
            const uint64_t step = (uint64_t)(cc * CH >> 4) + 2u * ks;
            mma<FMT>(d, da + step, db + step, Cfg::kIdesc, acc);
            acc = 1;
          }
        }
        started |= 1u << q;
        mma_commit(&empty[slot]);
        if (m.flags & kSlotLastB) {
          mma_commit(&empty[as]);
          if (++as == kASlots) {
            as = 0;
            aph ^= 1u;
          }
        }
        if ((m.flags & kSlotLast) && !close_run(q, 1)) {
          ok = false;
          break;
        }
        if (++bs == kBSlots) {
          bs = 0;
          bph ^= 1u;
        }
      }
      if (ok && wait_ab(&run_empty[rslot], rphase ^ 1u, abort_flag, p.status)) {
        runs[rslot] = GRun{-1, 0, 0, 1};   // end of work
        mbar_arrive(&run_full[rslot]);
      }
      mma_commit(drain);   // every MMA this thread issued has finished before TMEM is freed
      (void)mbar_wait(drain, 0, kDrainLimitNs);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int NC = 64;                       // columns owned by this warp
    const int quarter = warp & 3;                // TMEM lanes 32 * (warp % 4) ...
    const int col0 = ((warp - kEpi0) / 4) * NC;
    const int row = quarter * 32 + lane;
    uint32_t rslot = 0, rphase = 0;
    uint32_t taken = 0;     // bit q: parity of the runs taken from accumulator q
    uint32_t partial = 0;   // bit q: C holds this thread's partial sum of tile q's earlier runs
    for (;;) {
      // waits are decided for the whole warp: tcgen05.ld below needs all 32 lanes
      if (!__all_sync(kAll, wait_ab(&run_full[rslot], rphase, abort_flag, p.status))) break;
      const GRun r = runs[rslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&run_empty[rslot]);
      if (++rslot == kRuns) {
        rslot = 0;
        rphase ^= 1u;
      }
      if (r.tile < 0) break;
      const int q = r.q & (kG - 1);
      if (!__all_sync(kAll, wait_ab(&acc_full[q], (taken >> q) & 1u, abort_flag, p.status))) break;
      taken ^= 1u << q;
      fence_after_sync();
      float v[NC];
      {
        float h[32];
        const uint32_t base =
            tmem + (uint32_t)(q * Cfg::N + col0) + ((uint32_t)(quarter * 32) << 16);
        tmem_ld32(base, h);
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = h[c];
        tmem_ld32(base + 32, h);
#pragma unroll
        for (int c = 0; c < 32; ++c) v[32 + c] = h[c];
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[q]);   // the accumulator is free again
      // 2^s in one factor when it is a normal float, else in two
      const bool one = r.s >= -126 && r.s <= 127;
      const int s1 = one ? r.s : r.s / 2;
      const float scale = ldexpf(1.0f, s1), scale2 = ldexpf(1.0f, r.s - s1);
      const Inst& in = p.R.at(inst_of(p.R, p.Bf, r.tile));
      const int bn = in.bn;
      const int64_t lt = (int64_t)r.tile - in.tile0;
      const int ti = (int)(lt / bn), tj = (int)(lt % bn);
      const int64_t gr = (int64_t)ti * 128 + row;
      const int64_t cols = in.n - (int64_t)tj * 128 - col0;
      const bool had = (partial >> q) & 1u;
      if (r.last) partial &= ~(1u << q);
      else partial |= 1u << q;
      if (gr >= in.m || cols <= 0) continue;
      float* dst = in.C + gr * in.ldc + (int64_t)tj * 128 + col0;
      const bool vec = (in.ldc & 3) == 0 && cols >= NC;
      float acc[NC];
      if (had) {
        if (vec) {
#pragma unroll
          for (int c = 0; c < NC; c += 4) {
            const float4 x = *reinterpret_cast<const float4*>(dst + c);
            acc[c] = x.x;
            acc[c + 1] = x.y;
            acc[c + 2] = x.z;
            acc[c + 3] = x.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = c < cols ? dst[c] : 0.0f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
      }
      if (one) {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(v[c], scale, acc[c]);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(v[c] * scale, scale2, acc[c]);
      }
      if (vec) {
#pragma unroll
        for (int c = 0; c < NC; c += 4)
          *reinterpret_cast<float4*>(dst + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < cols) dst[c] = acc[c];
      }
    }
  }

  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, Cfg::kTmemCols);
  }
}

template <uint32_t FMT>
cudaError_t launch_group(const GParams& prm, cudaStream_t s) {
  using Cfg = GCfg<FMT>;
  auto kern = tc_group_kernel<FMT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return launch_pdl(kern, dim3(sms), dim3(Cfg::kThreads), Cfg::kSmemBytes, s, prm);
}

}  // namespace

bool multiply_tc_groups_supported(spamm_precision_t prec, int leaf, const InstRef& ref) {
  return leaf == 128 && (prec == SPAMM_BF16 || prec == SPAMM_FP16) && !ref.any_scaled &&
         !ref.any_norm_out && !ref.any_band;
}

cudaError_t launch_multiply_tc_groups(spamm_precision_t prec, const InstRef& ref,
                                      const PlanBuffers& b, const OperandImages& img,
                                      int32_t* status, cudaStream_t s) {
  const GParams prm{ref, b, img, status};
  switch (prec) {
    case SPAMM_BF16: return launch_group<kFmtBF16>(prm, s);
    case SPAMM_FP16: return launch_group<kFmtF16>(prm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spamm
